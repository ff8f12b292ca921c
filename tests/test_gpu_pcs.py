"""The hash-based commitment around the ZeroCheck on the GPU (stages (1)
and (3) of Sec. 3.1, Ligero-style): the root and the opening bytes equal the
oracle's, from one-row matrices to many rows; the whole flow (commit, prove
the ZeroCheck with the commitment as every column's root, recover the point
from the proof, open there) verifies on the host without the columns."""
import pytest

import oracle
from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = zc.Context(0, max_n=20, max_d=8)
    yield c
    c.close()


@pytest.mark.parametrize("gate,n,d,nc,t,eqf", [(1, 3, 3, 0, 5, False), (2, 8, 4, 3, 9, True),
                                                (1, 13, 3, 0, 16, False), (2, 16, 2, 10, 32, True),
                                                (witness.gate_sum(1), 12, 2, 6, 12, False), (1, 20, 3, 0, 24, True)])
def test_commit_prove_open_verify(ctx, gate, n, d, nc, t, eqf):
    cols = witness.generate(gate, n, d, 9800 + n)
    c = len(cols)
    dc = to_device(cols)
    com = ctx.pcs_commit(n, dc, t, nc)
    try:
        assert com.root == oracle.pcs_commit(n, cols, nc=nc or None)
        form = zc.ZC_FORM_SUMCHECK_EQ if eqf else zc.ZC_FORM_SUMCHECK
        pb = proof_bytes(ctx.prove_sumcheck(gate, n, d, dc, roots=[com.root] * c, eq_factored=eqf))
        alpha, vals, ok = zc.sumcheck_point(gate, n, d, form, [com.root] * c, pb)
        assert ok
        pr = com.open(alpha, vals)
        assert pr == oracle.pcs_open(n, cols, alpha, vals, t, nc=nc or None)
        assert zc.pcs_verify(n, c, t, com.root, alpha, vals, pr, nc)
        # an opening to values the columns do not have is rejected
        v2 = list(vals)
        v2[-1] = bytes([vals[-1][0] ^ 4]) + vals[-1][1:]
        assert not zc.pcs_verify(n, c, t, com.root, alpha, v2, com.open(alpha, v2), nc)
    finally:
        com.close()


def test_host_and_device_columns_commit_alike(ctx):
    gate, n, d, t = 2, 11, 5, 4
    cols = witness.generate(gate, n, d, 9900)
    a = ctx.pcs_commit(n, cols, t)
    b = ctx.pcs_commit(n, to_device(cols), t)
    try:
        assert a.root == b.root == oracle.pcs_commit(n, cols)
        alpha = [oracle.ints_to_bytes([x]).tobytes() for x in range(3, 3 + n)]
        vals = [oracle.ints_to_bytes([7 + j]).tobytes() for j in range(len(cols))]
        assert a.open(alpha, vals) == b.open(alpha, vals) == oracle.pcs_open(n, cols, alpha, vals, t)
    finally:
        a.close()
        b.close()
