"""Configuration-size parity: the library's proofs and quotients equal the
oracle's byte for byte at the workload sizes (Plonk n = 22 and 24, the
product gate at n = 22 for every degree of the sweep d = 2..32, the served
mix's n = 24 shapes, the sweep's 2N, 3N and 5N domains and the
eq-factored proof at n = 22, two of the paper's polynomials at n = 22,
the commitment of the bench's n = 22 columns), both forms.

The oracle's outputs at these sizes take it minutes, so they are stored as
SHA-256 digests in ``golden/oracle_digests.jsonl``, written by
``golden/make_oracle_digests.py`` from ``oracle/`` alone; the test hashes
the GPU output of the same seeded witness and compares."""
import hashlib
import os
import sys

import pytest

from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_oracle_digests as digests  # noqa: E402

RECORDS = digests.load()


def _ids(case):
    form, gate, n, d, lb, seed = case
    return f"{ {1: 'sc', 2: 'ntt', 3: 'sceq', 5: 'pcs'}[form]}-g{gate}-n{n}-d{d}" + (f"-lb{lb}" if lb else "")


@pytest.fixture(scope="module")
def ctx():
    c = zc.Context(0, max_n=24, max_d=32)
    yield c
    c.close()


@pytest.mark.parametrize("case", digests.CASES, ids=_ids)
def test_config_size_matches_oracle(ctx, case):
    import torch
    assert case in RECORDS, f"no oracle record for {case}: run tests/golden/make_oracle_digests.py"
    rec = RECORDS[case]
    form, gate, n, d, lb, seed = case
    cols = to_device(witness.generate(gate, n, d, seed))
    try:
        if form == 5:  # the commitment: root and opening (t queries in the log_blowup slot)
            com = ctx.pcs_commit(n, cols, lb)
            try:
                assert com.root.hex() == rec["root"], "commitment root differs from the oracle's"
                alpha, values = digests.pcs_point(n, len(cols))
                p = com.open(alpha, values)
            finally:
                com.close()
        elif form in (zc.ZC_FORM_SUMCHECK, zc.ZC_FORM_SUMCHECK_EQ):
            p = proof_bytes(ctx.prove_sumcheck(gate, n, d, cols, eq_factored=form == zc.ZC_FORM_SUMCHECK_EQ))
        else:
            q = torch.zeros(rec["q_len"], dtype=torch.uint8, device="cuda")
            p, _ = ctx.prove_ntt(gate, n, d, cols, q_out=q, log_blowup=lb)
            p = proof_bytes(p)
            qd = hashlib.sha256(q.cpu().numpy().tobytes()).hexdigest()
            del q
            assert qd == rec["q_sha256"], "quotient differs from the oracle's"
        assert len(p) == rec["proof_len"]
        assert hashlib.sha256(p).hexdigest() == rec["proof_sha256"], "proof differs from the oracle's"
    finally:
        del cols
        torch.cuda.empty_cache()
