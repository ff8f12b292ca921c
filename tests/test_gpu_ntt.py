"""NTT-form proofs and quotients from the CUDA library equal the oracle's,
byte for byte (Fig. side-by-side-zc left; Sec. 3.2), from one-pass sizes
through the two-pass four-step sizes, both gates, host and device buffers,
satisfying and tampered witnesses.  The configuration sizes (n = 22, 24)
are compared with stored oracle digests in test_gpu_configs.py."""
import numpy as np
import pytest

import oracle
from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu


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


def _check(ctx, gate, n, d, seed, tamper=False, device=True, roots=False, q_device=False):
    import torch
    cols = witness.generate(gate, n, d, seed, tamper=tamper)
    want_p, want_q = oracle.prove_ntt(gate, n, d, cols)
    rts = [oracle.root(c) for c in cols] if roots else None
    q_out = None
    if q_device:
        q_out = torch.zeros(len(want_q), dtype=torch.uint8, device="cuda")
    p, q = ctx.prove_ntt(gate, n, d, to_device(cols) if device else cols, roots=rts, q_out=q_out)
    assert _q_bytes(q) == want_q.tobytes(), "quotient differs"
    assert proof_bytes(p) == want_p, "proof differs"
    return cols, proof_bytes(p), _q_bytes(q)


@pytest.mark.parametrize("n", list(range(1, 16)))
def test_plonk_sizes(ctx, n):
    _check(ctx, 1, n, 3, 1000 + n)


@pytest.mark.parametrize("d", [2, 3, 4, 5, 8, 16])
@pytest.mark.parametrize("n", [2, 7, 13])
def test_product_gate(ctx, n, d):
    _check(ctx, 2, n, d, 2000 + d + n)


@pytest.mark.parametrize("gate,n,d", [(1, 9, 3), (2, 13, 4)])
def test_tampered_witness(ctx, gate, n, d):
    cols, p, q = _check(ctx, gate, n, d, 55, tamper=True)
    assert not zc.verify(gate, n, d, 2, cols, p, q=q)


@pytest.mark.parametrize("device,roots,q_device", [(False, False, False), (True, True, True),
                                                   (False, True, True), (True, False, False)])
def test_buffers(ctx, device, roots, q_device):
    _check(ctx, 1, 14, 3, 14, device=device, roots=roots, q_device=q_device)


@pytest.mark.parametrize("gate,n,d,seed", [(1, 18, 3, 1018), (2, 17, 5, 2017)])
def test_host_columns_pipelined(ctx, gate, n, d, seed):
    """Host columns at two-pass sizes: each column's N1 passes start as soon as
    that column has been copied; the bytes equal the oracle's."""
    _check(ctx, gate, n, d, seed, device=False, roots=True)


@pytest.mark.parametrize("where", [0, -1])
def test_noncanonical_rejected_two_pass(ctx, where):
    """A value >= r in the first or the last host column at a two-pass size
    (the check rides in N1's first pass)."""
    gate, n, d = 1, 14, 3
    cols = [np.array(c, copy=True) for c in witness.generate(gate, n, d, 4)]
    cols[where][32 * 100 + 31] = 0xf3
    with pytest.raises(zc.ZCError) as e:
        ctx.prove_ntt(gate, n, d, cols)
    assert e.value.status == 1


def test_noncanonical_rejected(ctx):
    gate, n, d = 1, 6, 3
    cols = witness.generate(gate, n, d, 3)
    cols[5] = np.array(cols[5], copy=True)
    cols[5][32 * 7 + 31] = 0xf0
    with pytest.raises(zc.ZCError) as e:
        ctx.prove_ntt(gate, n, d, cols)
    assert e.value.status == 1


@pytest.mark.parametrize("n", [20])
def test_plonk_config_sizes(ctx, n):
    """Plonk gate at n = 20 (seed 1000 + n), 4N coset; n = 22 in test_gpu_configs."""
    _check(ctx, 1, n, 3, 1000 + n, q_device=True)


def test_product_degree32_mid(ctx):
    _check(ctx, 2, 16, 32, 2032)


@pytest.mark.parametrize("gate,n,d", [(1, 2, 3), (1, 9, 3), (1, 14, 3), (2, 10, 3),
                                      (witness.gate_sum(0), 12, 3), (witness.gate_sum(1), 5, 2)])
def test_quotient_sized_domain(ctx, gate, n, d):
    # |D| = 2N for degree 3 and 2: the smallest power-of-two domain that
    # holds the quotient (Sec. 4, degree scaling); same bytes as the oracle
    lb = 1
    cols = witness.generate(gate, n, d, 8000 + n)
    want_p, want_q = oracle.prove_ntt(gate, n, d, cols, log_blowup=lb)
    p, q = ctx.prove_ntt(gate, n, d, to_device(cols), log_blowup=lb)
    assert _q_bytes(q) == want_q.tobytes()
    assert proof_bytes(p) == want_p
    assert zc.verify(gate, n, d, zc.ZC_FORM_NTT, cols, proof_bytes(p), q=_q_bytes(q), log_blowup=lb)
