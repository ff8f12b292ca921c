"""The paper's workload family (Sec. 5, Table poly_examples) through the sum
gate ZC_GATE_SUM_OF(m): f = g_1 ... g_d + g_{d+1} + ... + g_{d+m}.  Both
forms' proofs (and the NTT quotient) equal the oracle's byte for byte, from
one-element-pair tables through several tiles, the fused small rounds and the
large rounds; tampered witnesses give the oracle's bytes and are rejected;
batched proofs equal single ones."""
import numpy as np
import pytest

import oracle
from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu

# (name, gate word, d)
FAMILY = [("g1g2", zc.gate_sum(0), 2), ("g1g2+g3", zc.gate_sum(1), 2),
          ("g1g2+g3+g4", zc.gate_sum(2), 2), ("g1g2+g3+g4+g5", zc.gate_sum(3), 2),
          ("g1g2g3", zc.gate_sum(0), 3), ("g1g2g3g4", zc.gate_sum(0), 4)]
IDS = [f[0] for f in FAMILY]


@pytest.fixture(scope="module")
def ctx():
    c = zc.Context(0, max_n=24, max_d=32)
    yield c
    c.close()


def _q_bytes(q):
    import torch
    if isinstance(q, torch.Tensor):
        return q.cpu().numpy().tobytes()
    return np.asarray(q).tobytes()


@pytest.mark.parametrize("name,gate,d", FAMILY, ids=IDS)
@pytest.mark.parametrize("n", [1, 2, 5, 9, 14])
def test_sumcheck_matches_oracle(ctx, name, gate, d, n):
    cols = witness.generate(gate, n, d, 3000 + 7 * n + d + (gate >> 8))
    want = oracle.prove_sumcheck(gate, n, d, cols)
    assert proof_bytes(ctx.prove_sumcheck(gate, n, d, to_device(cols))) == want


@pytest.mark.parametrize("name,gate,d", FAMILY, ids=IDS)
@pytest.mark.parametrize("n", [1, 3, 8, 13])
def test_ntt_matches_oracle(ctx, name, gate, d, n):
    cols = witness.generate(gate, n, d, 4000 + 7 * n + d + (gate >> 8))
    want_p, want_q = oracle.prove_ntt(gate, n, d, cols)
    p, q = ctx.prove_ntt(gate, n, d, to_device(cols))
    assert _q_bytes(q) == want_q.tobytes()
    assert proof_bytes(p) == want_p


@pytest.mark.parametrize("name,gate,d", [FAMILY[3], FAMILY[5]], ids=[IDS[3], IDS[5]])
def test_large_rounds_match_oracle(ctx, name, gate, d):
    # n = 18: the separate fold + evaluation rounds (more than 2^16 pairs) run too
    n = 18
    cols = witness.generate(gate, n, d, 5000 + d)
    assert proof_bytes(ctx.prove_sumcheck(gate, n, d, to_device(cols))) == \
        oracle.prove_sumcheck(gate, n, d, cols)
    want_p, want_q = oracle.prove_ntt(gate, n, d, cols)
    p, q = ctx.prove_ntt(gate, n, d, to_device(cols))
    assert _q_bytes(q) == want_q.tobytes() and proof_bytes(p) == want_p


@pytest.mark.parametrize("name,gate,d", [FAMILY[1], FAMILY[4]], ids=[IDS[1], IDS[4]])
def test_tampered_rejected(ctx, name, gate, d):
    n = 10
    bad = witness.generate(gate, n, d, 61, tamper=True)
    ps = proof_bytes(ctx.prove_sumcheck(gate, n, d, to_device(bad)))
    assert ps == oracle.prove_sumcheck(gate, n, d, bad)
    assert not zc.verify(gate, n, d, zc.ZC_FORM_SUMCHECK, bad, ps)
    p, q = ctx.prove_ntt(gate, n, d, to_device(bad))
    assert not zc.verify(gate, n, d, zc.ZC_FORM_NTT, bad, proof_bytes(p), q=_q_bytes(q))


def test_batch_mixes_family_members(ctx):
    import torch
    forms, params, cols, proofs = [], [], [], []
    for i, (name, gate, d) in enumerate(FAMILY):
        n = 6 + 2 * i
        form = zc.ZC_FORM_SUMCHECK if i % 2 == 0 else zc.ZC_FORM_NTT
        c = witness.generate(gate, n, d, 6000 + i)
        forms.append(form)
        params.append((gate, n, d, 0))
        cols.append(to_device(c))
        proofs.append(torch.zeros(zc.proof_size(gate, n, d, form), dtype=torch.uint8, device="cuda"))
    ctx.prove_batch(forms, params, cols, proofs)
    torch.cuda.synchronize()
    for form, (gate, n, d, _), c, pr in zip(forms, params, cols, proofs):
        if form == zc.ZC_FORM_SUMCHECK:
            single = proof_bytes(ctx.prove_sumcheck(gate, n, d, c))
        else:
            single = proof_bytes(ctx.prove_ntt(gate, n, d, c)[0])
        assert proof_bytes(pr) == single
