"""Eq-factored SumCheck proofs on the GPU (rounds carry H_i(0..d), where
G_i = c_i l_i H_i; transcript v2): byte-identical to the oracle's across
sizes that span every round kernel band, both gates and the sum gate,
satisfying, tampered and edge-value witnesses, host and device buffers, and
inside batches."""
import pytest

import oracle
from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = zc.Context(0, max_n=20, max_d=16)
    yield c
    c.close()


def _check(ctx, gate, n, d, cols, device=True):
    want = oracle.prove_sumcheck_eq(gate, n, d, cols)
    got = proof_bytes(ctx.prove_sumcheck(gate, n, d, to_device(cols) if device else cols, eq_factored=True))
    assert got == want
    return got


@pytest.mark.parametrize("n", [1, 2, 5, 8, 11, 14, 17, 20])
@pytest.mark.parametrize("gate,d", [(1, 3), (2, 2), (2, 5), (2, 8), (witness.gate_sum(1), 2)])
def test_eq_factored_matches_oracle(ctx, gate, n, d):
    if n == 20 and gate != 1 and d > 2:
        pytest.skip("n = 20 runs the Plonk and degree-2 gates")
    cols = witness.generate(gate, n, d, 9100 + n + d)
    pb = _check(ctx, gate, n, d, cols)
    if n <= 14:
        assert zc.verify(gate, n, d, zc.ZC_FORM_SUMCHECK_EQ, cols, pb)


@pytest.mark.parametrize("gate,n,d", [(1, 9, 3), (2, 12, 4), (witness.gate_sum(0), 7, 3)])
def test_eq_factored_tampered_and_edge(ctx, gate, n, d):
    bad = witness.generate(gate, n, d, 9200 + n, tamper=True)
    pb = _check(ctx, gate, n, d, bad, device=False)
    assert not zc.verify(gate, n, d, zc.ZC_FORM_SUMCHECK_EQ, bad, pb)
    _check(ctx, gate, n, d, witness.generate_edge(gate, n, d, 9300 + n))


def test_eq_factored_in_a_batch(ctx):
    import torch
    shapes = [(1, 10, 3, 1), (2, 12, 8, 3), (1, 13, 3, 3), (2, 9, 2, 1), (1, 11, 3, 2)]
    cols = [witness.generate(g, n, d, 9400 + i) for i, (g, n, d, _) in enumerate(shapes)]
    forms = [f for *_, f in shapes]
    params = [(g, n, d, 0) for g, n, d, _ in shapes]
    proofs = [torch.zeros(zc.proof_size(g, n, d, f), dtype=torch.uint8, device="cuda") for g, n, d, f in shapes]
    ctx.prove_batch(forms, params, [to_device(c) for c in cols], proofs, None)
    torch.cuda.synchronize()
    for (g, n, d, f), c, p in zip(shapes, cols, proofs):
        if f == zc.ZC_FORM_SUMCHECK_EQ:
            want = oracle.prove_sumcheck_eq(g, n, d, c)
        elif f == zc.ZC_FORM_SUMCHECK:
            want = oracle.prove_sumcheck(g, n, d, c)
        else:
            want = oracle.prove_ntt(g, n, d, c)[0]
        assert proof_bytes(p) == want, (g, n, d, f)
