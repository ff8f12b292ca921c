"""Boundary field values through both GPU forms: columns drawn from 0, 1, 2,
r-1, r-2, r-2^k, 2^k, 2^k - 1, 2^256 mod r, (r +- 1)/2, ... (mixed with
uniform values, or nothing else), gate not satisfied.  The proof of either
form is defined for any canonical input (Sec. 3.2, 3.3), so the library's
bytes must equal the oracle's; these inputs put values next to the modulus
and all-zero or all-one limbs through every carry chain, conditional
subtraction and Montgomery-level conversion of the kernels."""
import numpy as np
import pytest

import oracle
from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu

SHAPES = [(1, 3), (2, 2), (2, 4), (2, 7), (witness.gate_sum(2), 2), (witness.gate_sum(0), 3)]


@pytest.fixture(scope="module")
def ctx():
    c = zc.Context(0, max_n=20, max_d=16)
    yield c
    c.close()


@pytest.mark.parametrize("only_edges", [True, False])
@pytest.mark.parametrize("n", [1, 5, 12, 17])
@pytest.mark.parametrize("gate,d", SHAPES)
def test_edge_values_sumcheck(ctx, gate, d, n, only_edges):
    cols = witness.generate_edge(gate, n, d, 9000 + 10 * n + d, only_edges=only_edges)
    want = oracle.prove_sumcheck(gate, n, d, cols)
    got = proof_bytes(ctx.prove_sumcheck(gate, n, d, to_device(cols)))
    assert got == want


@pytest.mark.parametrize("only_edges", [True, False])
@pytest.mark.parametrize("n", [1, 5, 12, 17])
@pytest.mark.parametrize("gate,d", SHAPES)
def test_edge_values_ntt(ctx, gate, d, n, only_edges):
    cols = witness.generate_edge(gate, n, d, 9500 + 10 * n + d, only_edges=only_edges)
    want_p, want_q = oracle.prove_ntt(gate, n, d, cols)
    p, q = ctx.prove_ntt(gate, n, d, to_device(cols))
    assert np.asarray(q).tobytes() == want_q.tobytes(), "quotient differs"
    assert proof_bytes(p) == want_p, "proof differs"


@pytest.mark.parametrize("n", [3, 12])
def test_edge_values_quotient_sized_domain(ctx, n):
    gate, d = 1, 3
    cols = witness.generate_edge(gate, n, d, 9900 + n)
    want_p, want_q = oracle.prove_ntt(gate, n, d, cols, log_blowup=1)
    p, q = ctx.prove_ntt(gate, n, d, to_device(cols), log_blowup=1)
    assert np.asarray(q).tobytes() == want_q.tobytes()
    assert proof_bytes(p) == want_p
