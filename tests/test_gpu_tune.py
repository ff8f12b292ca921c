"""Launch tuning changes speed only: every SumCheck round split / tail
threshold and every NTT pass tile proves the oracle's bytes, and the
autotuner stores the fastest candidate."""
import pytest

import oracle
from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import tune, witness, zc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = zc.Context(0, max_n=24, max_d=32)
    yield c
    c.close()


@pytest.mark.parametrize("gate,n,d", [(1, 12, 3), (2, 11, 8)])
def test_sumcheck_candidates_same_bytes(ctx, gate, n, d):
    cols = witness.generate(gate, n, d, 8100 + n)
    want = oracle.prove_sumcheck(gate, n, d, cols)
    dc = to_device(cols)
    cands = [{k: v} for k, vals in tune.SC_SPACE.items() for v in vals]
    cands += [{zc.ZC_TUNE_SC_GRID: 1, zc.ZC_TUNE_SC_TAIL_LOG: 1, zc.ZC_TUNE_SC_SMALL_LOG: 1},
              {zc.ZC_TUNE_SC_GRID: 3, zc.ZC_TUNE_SC_TAIL_LOG: 24},
              {zc.ZC_TUNE_SC_GRID: 5, zc.ZC_TUNE_SC_SMALL_LOG: 24, zc.ZC_TUNE_SC_TAIL_LOG: 3,
               zc.ZC_TUNE_SC_MINB: 2},
              {zc.ZC_TUNE_SC_SMALL_LOG: 1, zc.ZC_TUNE_SC_CHUNK_LOG: 24, zc.ZC_TUNE_SC_TAIL_LOG: 2},
              {zc.ZC_TUNE_SC_SMALL_LOG: 1, zc.ZC_TUNE_SC_CHUNK_LOG: 1, zc.ZC_TUNE_SC_PROD_PPT: 1}]
    for cand in cands:
        for k in tune.SC_SPACE:
            ctx.tune_set(zc.ZC_FORM_SUMCHECK, n, k, cand.get(k, 0))
        assert proof_bytes(ctx.prove_sumcheck(gate, n, d, dc)) == want, cand
    for k in tune.SC_SPACE:
        ctx.tune_set(zc.ZC_FORM_SUMCHECK, n, k, 0)


@pytest.mark.parametrize("gate,n,d", [(1, 14, 3), (2, 13, 5), (1, 9, 3), (2, 6, 8)])
def test_ntt_candidates_same_bytes(ctx, gate, n, d):
    cols = witness.generate(gate, n, d, 8200 + n)
    want_p, want_q = oracle.prove_ntt(gate, n, d, cols)
    dc = to_device(cols)
    cands = [{zc.ZC_TUNE_NTT_TILE_LOG: t, zc.ZC_TUNE_NTT_MINB: m} for t in (10, 11, 12) for m in (1, 2)]
    cands += [{zc.ZC_TUNE_NTT_TWO_LOG: v} for v in (2, 4, 6, 9, 13, 24)]
    for cand in cands:
        for k in (zc.ZC_TUNE_NTT_TILE_LOG, zc.ZC_TUNE_NTT_MINB, zc.ZC_TUNE_NTT_TWO_LOG):
            ctx.tune_set(zc.ZC_FORM_NTT, n, k, cand.get(k, 0))
        p, q = ctx.prove_ntt(gate, n, d, dc)
        assert proof_bytes(p) == want_p, cand
        assert proof_bytes(q) == want_q.tobytes(), cand
    for k in (zc.ZC_TUNE_NTT_TILE_LOG, zc.ZC_TUNE_NTT_MINB, zc.ZC_TUNE_NTT_TWO_LOG):
        ctx.tune_set(zc.ZC_FORM_NTT, n, k, 0)


def test_tune_values_checked(ctx):
    ctx.tune_set(zc.ZC_FORM_NTT, 0, zc.ZC_TUNE_NTT_TILE_LOG, 11)
    assert ctx.tune_get(zc.ZC_FORM_NTT, 17, zc.ZC_TUNE_NTT_TILE_LOG) == 11
    ctx.tune_set(zc.ZC_FORM_NTT, 17, zc.ZC_TUNE_NTT_TILE_LOG, 12)
    assert ctx.tune_get(zc.ZC_FORM_NTT, 17, zc.ZC_TUNE_NTT_TILE_LOG) == 12
    assert ctx.tune_get(zc.ZC_FORM_NTT, 16, zc.ZC_TUNE_NTT_TILE_LOG) == 11
    ctx.tune_set(zc.ZC_FORM_NTT, 17, zc.ZC_TUNE_NTT_TILE_LOG, 0)
    ctx.tune_set(zc.ZC_FORM_NTT, 0, zc.ZC_TUNE_NTT_TILE_LOG, 0)
    for form, n, key, v in [(zc.ZC_FORM_NTT, 0, zc.ZC_TUNE_NTT_TILE_LOG, 13),
                            (zc.ZC_FORM_NTT, 0, zc.ZC_TUNE_NTT_MINB, 3),
                            (zc.ZC_FORM_SUMCHECK, 0, zc.ZC_TUNE_NTT_TILE_LOG, 11),
                            (zc.ZC_FORM_SUMCHECK, 29, zc.ZC_TUNE_SC_GRID, 8),
                            (zc.ZC_FORM_SUMCHECK, 0, zc.ZC_TUNE_SC_GRID, 5000),
                            (3, 0, zc.ZC_TUNE_SC_GRID, 8),
                            (zc.ZC_FORM_SUMCHECK, 12, zc.ZC_TUNE_BATCH_LANES, 8),
                            (zc.ZC_FORM_NTT, 0, zc.ZC_TUNE_BATCH_LANES, 65)]:
        with pytest.raises(zc.ZCError):
            ctx.tune_set(form, n, key, v)


def test_autotuner_picks_fastest(ctx):
    gate, n, d = 1, 16, 3
    dc = to_device(witness.generate(gate, n, d, 8300))
    for form in (zc.ZC_FORM_SUMCHECK, zc.ZC_FORM_NTT):
        r = tune.tune_shape(ctx, form, gate, n, d, dc, reps=2)
        assert r["ms"] <= min(ms for _, _, ms in r["trials"]) + 1e-9
        for k, v in r["best"].items():
            assert ctx.tune_get(form, n, k) == v
        for k in tune.space(form):
            ctx.tune_set(form, n, k, 0)


def test_batch_tuner_keeps_bytes(ctx):
    import torch
    mix = [(1, 1, 9, 3), (2, 2, 8, 8), (1, 2, 10, 8), (2, 1, 11, 3)]
    forms, params, cols, dcols, proofs = [], [], [], [], []
    for i, (form, gate, n, d) in enumerate(mix):
        c = witness.generate(gate, n, d, 8400 + i)
        forms.append(form)
        params.append((gate, n, d, 0))
        cols.append(c)
        dcols.append(to_device(c))
        proofs.append(torch.zeros(zc.proof_size(gate, n, d, form), dtype=torch.uint8, device="cuda"))
    r = tune.tune_batch(ctx, forms, params, dcols, proofs, None, reps=1)
    assert r["ms"] > 0 and len(r["trials"]) > 1
    ctx.prove_batch(forms, params, dcols, proofs, None)
    torch.cuda.synchronize()
    for (form, gate, n, d), c, p in zip(mix, cols, proofs):
        want = (oracle.prove_sumcheck(gate, n, d, c) if form == 1 else oracle.prove_ntt(gate, n, d, c)[0])
        assert proof_bytes(p) == want
    for form in (zc.ZC_FORM_SUMCHECK, zc.ZC_FORM_NTT):
        for n in range(8, 12):
            for k in tune.space(form):
                ctx.tune_set(form, n, k, 0)
    ctx.tune_set(zc.ZC_FORM_SUMCHECK, 0, zc.ZC_TUNE_BATCH_LANES, 0)


@pytest.mark.parametrize("small,chunk,quad", [(14, 10, 1), (10, 14, 1), (16, 16, 1), (1, 1, 1),
                                              (14, 10, 15), (10, 12, 16), (1, 1, 24), (15, 8, 12)])
def test_full_and_derived_rounds_mix(ctx, small, chunk, quad):
    """Rounds that derive a point and rounds that evaluate all points, in
    either kernel, interleave correctly (claims kept exactly when needed)."""
    gate, n, d = 1, 17, 3
    cols = witness.generate(gate, n, d, 8500)
    want = oracle.prove_sumcheck(gate, n, d, cols)
    ctx.tune_set(zc.ZC_FORM_SUMCHECK, n, zc.ZC_TUNE_SC_SMALL_LOG, small)
    ctx.tune_set(zc.ZC_FORM_SUMCHECK, n, zc.ZC_TUNE_SC_CHUNK_LOG, chunk)
    ctx.tune_set(zc.ZC_FORM_SUMCHECK, n, zc.ZC_TUNE_SC_QUAD_LOG, quad)
    try:
        assert proof_bytes(ctx.prove_sumcheck(gate, n, d, to_device(cols))) == want
    finally:
        ctx.tune_set(zc.ZC_FORM_SUMCHECK, n, zc.ZC_TUNE_SC_SMALL_LOG, 0)
        ctx.tune_set(zc.ZC_FORM_SUMCHECK, n, zc.ZC_TUNE_SC_CHUNK_LOG, 0)
        ctx.tune_set(zc.ZC_FORM_SUMCHECK, n, zc.ZC_TUNE_SC_QUAD_LOG, 0)
