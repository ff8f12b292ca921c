"""The persistent round kernel (the Plonk rounds with at most 2^14 pairs
before the tail, in one cooperative launch with bounded grid-wide
hand-offs): its proofs equal the oracle's and those of the per-round
kernels; when its hand-off waits are made to run out (a poll limit of one,
set from the host), the launch still ends, the call returns
ZC_ERR_TIMEOUT, and the context proves correctly afterwards."""
import pytest

import oracle
from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [8, 12, 16, 20])
def test_persistent_and_per_round_kernels_agree(monkeypatch, n):
    gate, d = 1, 3
    cols = witness.generate(gate, n, d, 9600 + n)
    want = oracle.prove_sumcheck(gate, n, d, cols)
    dc = to_device(cols)
    for flag in ("1", "0"):
        monkeypatch.setenv("ZC_SC_PERSISTENT", flag)
        ctx = zc.Context(0, max_n=20, max_d=8)
        try:
            assert proof_bytes(ctx.prove_sumcheck(gate, n, d, dc)) == want, flag
            assert proof_bytes(ctx.prove_sumcheck(gate, n, d, dc, eq_factored=True)) == \
                oracle.prove_sumcheck_eq(gate, n, d, cols), flag
        finally:
            ctx.close()


def test_handoff_timeout_is_reported_and_recovered(monkeypatch):
    gate, n, d = 1, 16, 3
    cols = witness.generate(gate, n, d, 9700)
    dc = to_device(cols)
    ctx = zc.Context(0, max_n=16, max_d=8)
    try:
        monkeypatch.setenv("ZC_SPIN_LIMIT", "1")
        with pytest.raises(zc.ZCError) as e:
            ctx.prove_sumcheck(gate, n, d, dc)
        assert e.value.status == 4                      # ZC_ERR_TIMEOUT
        monkeypatch.delenv("ZC_SPIN_LIMIT")
        assert proof_bytes(ctx.prove_sumcheck(gate, n, d, dc)) == oracle.prove_sumcheck(gate, n, d, cols)
    finally:
        ctx.close()
