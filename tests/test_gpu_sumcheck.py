"""SumCheck-form proofs from the CUDA library equal the oracle's, byte for
byte (Fig. side-by-side-zc right; Sec. 3.3), across sizes that span several
tiles and a ragged tail, both gates, host and device inputs, satisfying and
tampered witnesses, and the configuration sizes."""
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


def _check(ctx, gate, n, d, seed, tamper=False, device=True, roots=False):
    cols = witness.generate(gate, n, d, seed, tamper=tamper)
    want = oracle.prove_sumcheck(gate, n, d, cols)
    rts = [oracle.root(c) for c in cols] if roots else None
    got = ctx.prove_sumcheck(gate, n, d, to_device(cols) if device else cols, roots=rts)
    assert proof_bytes(got) == want


@pytest.mark.parametrize("n", list(range(1, 15)))
def test_plonk_small_sizes(ctx, n):
    _check(ctx, 1, n, 3, 1000 + n)


@pytest.mark.parametrize("d", [2, 3, 4, 5, 7, 8, 16, 32])
@pytest.mark.parametrize("n", [1, 3, 9])
def test_product_gate_small(ctx, n, d):
    _check(ctx, 2, n, d, 2000 + d + n)


@pytest.mark.parametrize("gate,n,d", [(1, 10, 3), (2, 8, 4), (2, 11, 3)])
def test_tampered_witness_bytes_and_rejection(ctx, gate, n, d):
    cols = witness.generate(gate, n, d, 77, tamper=True)
    want = oracle.prove_sumcheck(gate, n, d, cols)
    got = proof_bytes(ctx.prove_sumcheck(gate, n, d, to_device(cols)))
    assert got == want
    assert not zc.verify(gate, n, d, 1, cols, got)


@pytest.mark.parametrize("device", [False, True])
@pytest.mark.parametrize("roots", [False, True])
def test_host_device_inputs_and_given_roots(ctx, device, roots):
    _check(ctx, 1, 13, 3, 5, device=device, roots=roots)
    _check(ctx, 2, 12, 5, 6, device=device, roots=roots)


@pytest.mark.parametrize("gate,n,d,seed,tamper", [(1, 18, 3, 1018, False), (1, 20, 3, 1020, False),
                                                   (2, 18, 2, 2102, False), (2, 19, 5, 2105, False),
                                                   (1, 18, 3, 91, True)])
def test_host_columns_in_ranges(ctx, gate, n, d, seed, tamper):
    """Host columns from n = 18 on, with their roots given, are copied in
    pair ranges while round 1 runs on the ranges already copied (one
    round-1 launch per range): the bytes equal the oracle's."""
    _check(ctx, gate, n, d, seed, tamper=tamper, device=False, roots=True)


def test_host_columns_in_ranges_eq_factored_and_rejection(ctx):
    gate, n, d = 1, 18, 3
    cols = witness.generate(gate, n, d, 1018)
    rts = [oracle.root(c) for c in cols]
    got = ctx.prove_sumcheck(gate, n, d, cols, roots=rts, eq_factored=True)
    assert proof_bytes(got) == oracle.prove_sumcheck_eq(gate, n, d, cols)
    bad = [np.array(c, copy=True) for c in cols]
    bad[6][32 * ((1 << n) - 3) + 31] = 0xf7          # a value >= r in the last range
    with pytest.raises(zc.ZCError) as e:
        ctx.prove_sumcheck(gate, n, d, bad, roots=rts)
    assert e.value.status == 1


def test_device_proof_buffer_async(ctx):
    import torch
    gate, n, d = 1, 12, 3
    cols = witness.generate(gate, n, d, 1012)
    want = oracle.prove_sumcheck(gate, n, d, cols)
    out = torch.zeros(zc.proof_size(gate, n, d, 1), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    dc = to_device(cols)
    torch.cuda.synchronize()
    ctx.prove_sumcheck(gate, n, d, dc, stream=s, proof_out=out)
    s.synchronize()
    assert proof_bytes(out) == want
    assert zc.verify(gate, n, d, 1, cols, want)


def test_noncanonical_input_rejected(ctx):
    gate, n, d = 1, 6, 3
    cols = witness.generate(gate, n, d, 3)
    cols[2] = np.array(cols[2], copy=True)
    cols[2][32 * 5 + 31] = 0xff            # element 5 of qM >= r
    with pytest.raises(zc.ZCError) as e:
        ctx.prove_sumcheck(gate, n, d, cols)
    assert e.value.status == 1


def test_derived_point_switch(monkeypatch):
    """Deriving H(0) instead of H(1) from the round identity gives the same bytes."""
    monkeypatch.setenv("ZC_SUMCHECK_DERIVED_POINT", "0")
    c2 = zc.Context(0, max_n=16, max_d=8)
    try:
        for gate, n, d in [(1, 11, 3), (2, 9, 5), (2, 6, 2)]:
            _check(c2, gate, n, d, 31)
    finally:
        c2.close()


@pytest.mark.parametrize("n", [20])
def test_plonk_config_sizes(ctx, n):
    """configs: Plonk gate, n = 20, seed 1000 + n; n = 22 in test_gpu_configs."""
    _check(ctx, 1, n, 3, 1000 + n)


@pytest.mark.parametrize("d", [4, 8, 16])
def test_product_gate_mid_degrees(ctx, d):
    _check(ctx, 2, 16, d, 2000 + d)
