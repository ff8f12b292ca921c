"""Step-radix NTT domains on the GPU (Sec. 4, "Degree scaling": a quotient
transform of 2^k N + N points, e.g. 3N = 2N + N for degree 4 and 5N = 4N +
N for degree 6): proofs and quotients equal the oracle's byte for byte, from
one-pass sizes through the two-pass four-step sizes, host and device
buffers, satisfying, tampered and edge-value witnesses; the library's own
verifier accepts them."""
import numpy as np
import pytest

import oracle
from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu

W3N = zc.domain_word(1, 0)   # 2N + N
W5N = zc.domain_word(2, 0)   # 4N + N


@pytest.fixture(scope="module")
def ctx():
    c = zc.Context(0, max_n=22, max_d=16)
    yield c
    c.close()


def _check(ctx, gate, n, d, w, cols, q_device=False, device=True):
    import torch
    want_p, want_q = oracle.prove_ntt(gate, n, d, cols, log_blowup=w)
    q_out = torch.zeros(len(want_q), dtype=torch.uint8, device="cuda") if q_device else None
    p, q = ctx.prove_ntt(gate, n, d, to_device(cols) if device else cols, q_out=q_out, log_blowup=w)
    qb = q.cpu().numpy().tobytes() if q_device else np.asarray(q).tobytes()
    assert len(qb) == zc.domain_size(n, d, w) * 32
    assert qb == want_q.tobytes(), "quotient differs"
    assert proof_bytes(p) == want_p, "proof differs"
    return proof_bytes(p), qb


@pytest.mark.parametrize("n", [3, 9, 14, 20])
@pytest.mark.parametrize("gate,d,w", [(1, 3, W3N), (2, 4, W3N), (2, 6, W5N), (witness.gate_sum(0), 4, W3N)])
def test_step_radix_matches_oracle(ctx, gate, n, d, w):
    cols = witness.generate(gate, n, d, 8100 + n + d)
    pb, qb = _check(ctx, gate, n, d, w, cols, q_device=n >= 14)
    assert zc.verify(gate, n, d, zc.ZC_FORM_NTT, cols, pb, q=qb, log_blowup=w)


@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_step_radix_small_and_edge(ctx, n):
    for gate, d, w in [(1, 3, W3N), (2, 4, W3N), (2, 5, W5N)]:
        _check(ctx, gate, n, d, w, witness.generate_edge(gate, n, d, 8300 + n))


def test_step_radix_tampered_and_host_buffers(ctx):
    gate, n, d = 2, 11, 4
    cols = witness.generate(gate, n, d, 8400, tamper=True)
    pb, qb = _check(ctx, gate, n, d, W3N, cols, device=False)
    assert not zc.verify(gate, n, d, zc.ZC_FORM_NTT, cols, pb, q=qb, log_blowup=W3N)


def test_step_radix_rejects_bad_words(ctx):
    cols = to_device(witness.generate(2, 8, 6, 1))
    for w in (zc.domain_word(1, 0),     # 3N cannot hold a degree-6 quotient (5N - 5)
              zc.domain_word(1, 1),     # the small part must be smaller
              zc.domain_word(0, 0)):    # a step domain needs a big part of 2N at least
        with pytest.raises(zc.ZCError) as e:
            ctx.prove_ntt(2, 8, 6, cols, log_blowup=w)
        assert e.value.status == 1
    with pytest.raises(zc.ZCError) as e:    # s > 0 is not built on the GPU
        ctx.prove_ntt(2, 8, 6, cols, log_blowup=zc.domain_word(3, 1))
    assert e.value.status == 5
