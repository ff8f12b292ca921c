"""Autotuner for the launch shapes (zc_tune_set keys).

Every setting gives byte-identical proofs; only time changes.  The search
is coordinate descent: one key at a time, every candidate value timed with
the others held, the fastest kept, then the next key.  Two modes:

* ``tune_shape``: one proof of (form, gate, n, d) alone on the GPU; the
  winners are stored for that n.
* ``tune_batch``: a whole batch (``zc_batch_create`` graph), timed as one
  graph launch; the winners are stored for every size in the batch.
  Concurrent lanes favour smaller round grids than a proof alone does.

Times are CUDA-event medians on the launching stream after one untimed run.
"""
from __future__ import annotations

from . import zc

SC_SPACE = {
    zc.ZC_TUNE_SC_GRID: (152, 304, 456, 608, 912),
    zc.ZC_TUNE_SC_MINB: (1, 2),
    zc.ZC_TUNE_SC_PROD_PPT: (1, 3),
    zc.ZC_TUNE_SC_PROD_FUSE: (1, 10, 14, 18, 24),
    zc.ZC_TUNE_SC_QUAD_LOG: (13, 15, 16, 17, 18),
    zc.ZC_TUNE_SC_CHUNK_LOG: (12, 13, 14, 16),
    zc.ZC_TUNE_SC_SMALL_LOG: (10, 12, 13, 14, 16),
    zc.ZC_TUNE_SC_TAIL_LOG: (4, 5, 6, 7),
}
BATCH_LANES = (8, 16, 32, 64)
NTT_SPACE = {
    zc.ZC_TUNE_NTT_TWO_LOG: (6, 8, 10, 12, 13),
    zc.ZC_TUNE_NTT_TILE_LOG: (10, 11, 12),
    zc.ZC_TUNE_NTT_MINB: (1, 2),
}


def space(form: int) -> dict:
    return SC_SPACE if form == zc.ZC_FORM_SUMCHECK else NTT_SPACE


def _time(fn, stream, reps):
    import torch
    fn()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return sorted(ts)[len(ts) // 2]


def _descend(ctx, keys, ns, run, stream, reps):
    """keys: [(form, key, values)].  Sets the winners; returns (best_ms, settings, trials)."""
    trials = []
    best_ms = _time(run, stream, reps)
    trials.append(("start", None, best_ms))
    settings = {}
    for form, key, values in keys:
        cur = ctx.tune_get(form, ns[0], key)
        best_v = cur
        for v in values:
            if v == cur:
                continue
            for n in ns:
                ctx.tune_set(form, n, key, v)
            ms = _time(run, stream, reps)
            trials.append(((form, key), v, ms))
            if ms < best_ms:
                best_ms, best_v = ms, v
        for n in ns:
            ctx.tune_set(form, n, key, best_v)
        settings[(form, key)] = best_v
    return best_ms, settings, trials


def tune_shape(ctx, form, gate, n, d, dcols, reps: int = 3) -> dict:
    """Tune every key of `form` on one proof of (gate, n, d); winners stored for n."""
    import torch
    stream = torch.cuda.Stream()
    proof = torch.empty(zc.proof_size(gate, n, d, form), dtype=torch.uint8, device="cuda")
    if form == zc.ZC_FORM_SUMCHECK:
        def run():
            ctx.prove_sumcheck(gate, n, d, dcols, stream=stream, proof_out=proof)
    else:
        def run():
            ctx.prove_ntt(gate, n, d, dcols, stream=stream, proof_out=proof, want_q=False)
    keys = [(form, k, v) for k, v in space(form).items()]
    best_ms, settings, trials = _descend(ctx, keys, [n], run, stream, reps)
    return {"ms": best_ms, "best": {k: v for (_, k), v in settings.items()}, "trials": trials}


def tune_batch(ctx, forms, params, cols, proofs, q_outs=None, reps: int = 3) -> dict:
    """Tune the keys of the forms present in a batch by the time of its graph."""
    import torch
    stream = torch.cuda.Stream()
    keys, ns_of = [], {}
    for form in (zc.ZC_FORM_SUMCHECK, zc.ZC_FORM_NTT):
        ns = sorted({p[1] for f, p in zip(forms, params) if f == form})
        if ns:
            ns_of[form] = ns
            keys += [(form, k, v) for k, v in space(form).items()]
    # the lane count is one value per context (n = 0), tried first
    keys.insert(0, ("lanes", zc.ZC_TUNE_BATCH_LANES, BATCH_LANES))
    ns_of["lanes"] = [0]
    state = {"g": None}

    def run():
        if state["g"] is None:
            state["g"] = ctx.batch_graph(forms, params, cols, proofs, q_outs)
        state["g"].launch(stream)

    def reset():
        if state["g"] is not None:
            state["g"].close()
            state["g"] = None

    # a new graph per setting: the launch shapes are fixed at capture
    trials, settings = [], {}
    best_ms = _time(run, stream, reps)
    trials.append(("start", None, best_ms))
    for form, key, values in keys:
        ns = ns_of[form]
        f = zc.ZC_FORM_SUMCHECK if form == "lanes" else form
        cur = ctx.tune_get(f, ns[0], key)
        best_v = cur
        for v in values:
            if v == cur:
                continue
            for n in ns:
                ctx.tune_set(f, n, key, v)
            reset()
            ms = _time(run, stream, reps)
            trials.append(((form, key), v, ms))
            if ms < best_ms:
                best_ms, best_v = ms, v
        for n in ns:
            ctx.tune_set(f, n, key, best_v)
        settings[(form, key)] = best_v
        reset()
    reset()
    return {"ms": best_ms, "best": {f"{f}:{k}": v for (f, k), v in settings.items()}, "trials": trials}
