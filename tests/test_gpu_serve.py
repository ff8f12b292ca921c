"""Served proving: requests of mixed shape and form arriving over time are
admitted as slots and pool space free up, overlap on the device, and each
proof equals the proof of the same request alone (the oracle's bytes)."""
import pytest

import oracle
from gpu_util import proof_bytes
from paper_2606_16146_gb300 import serve, workloads, zc
from paper_2606_16146_gb300.workloads import Shape

pytestmark = pytest.mark.gpu

SHAPES = [Shape(1, 9, 3), Shape(2, 8, 8), Shape(1, 12, 3), Shape(2, 11, 16), Shape(2, 6, 4),
          Shape(1, 13, 3), Shape(2, 10, 8), Shape(1, 3, 3)]


@pytest.fixture(scope="module")
def ctx():
    c = zc.Context(0, max_n=24, max_d=32)
    yield c
    c.close()


@pytest.fixture(scope="module")
def expected():
    cache = {}

    def get(s, form):
        key = (s, form)
        if key not in cache:
            from paper_2606_16146_gb300 import witness
            cols = witness.generate(s.gate, s.n, s.d, workloads.shape_seed(s))
            if form == zc.ZC_FORM_SUMCHECK:
                cache[key] = oracle.prove_sumcheck(s.gate, s.n, s.d, cols)
            else:
                cache[key] = oracle.prove_ntt(s.gate, s.n, s.d, cols)[0]
        return cache[key]
    return get


def _timed(count, spacing):
    return [(i * spacing, SHAPES[(3 * i + 1) % len(SHAPES)]) for i in range(count)]


def _check(reqs, results, expected):
    for q, r in zip(reqs, results):
        assert r["status"] == 0
        assert r["done_s"] >= r["admit_s"] >= q["arrival_s"] - 1e-6
        assert proof_bytes(q["proof"]) == expected(q["shape"], q["form"]), (q["shape"], q["form"])


def test_mixed_requests_equal_alone(ctx, expected):
    srv = serve.Server(ctx, slots=4, hbm_budget_bytes=4 << 30)
    timed = _timed(24, 0.002)
    srv.load_pool([s for _, s in timed])
    forms = [zc.ZC_FORM_SUMCHECK if i % 3 else zc.ZC_FORM_NTT for i in range(len(timed))]
    reqs = srv.build(timed, forms=forms)
    results = srv.run(reqs, timeout_s=120)
    _check(reqs, results, expected)
    rep = serve.report(reqs, results)
    assert rep["completed"] == len(reqs)


def test_burst_overlaps_on_the_device(ctx, expected):
    srv = serve.Server(ctx, slots=8, hbm_budget_bytes=4 << 30)
    timed = [(0.0, SHAPES[i % len(SHAPES)]) for i in range(16)]
    srv.load_pool([s for _, s in timed])
    reqs = srv.build(timed, forms=[zc.ZC_FORM_SUMCHECK] * 16)
    results = srv.run(reqs, timeout_s=120)
    _check(reqs, results, expected)
    # continuous batching: some request was admitted while another was in flight
    iv = [(r["admit_s"], r["done_s"]) for r in results]
    assert any(a2 < d1 and a1 < d2 for i, (a1, d1) in enumerate(iv) for (a2, d2) in iv[i + 1:])
    assert len({r["slot"] for r in results}) > 1


@pytest.mark.parametrize("in_order", [True, False])
def test_memory_bound_admission(ctx, expected, in_order):
    big = Shape(1, 13, 3)
    fp = ctx.scratch_bytes(big.gate, big.n, big.d, zc.ZC_FORM_NTT)
    budget = int(fp * 1.5)
    srv = serve.Server(ctx, slots=6, hbm_budget_bytes=budget, in_order=in_order)
    timed = [(0.0, big), (0.0, big), (0.0, Shape(1, 9, 3)), (0.0, big), (0.001, Shape(2, 8, 8))]
    srv.load_pool([s for _, s in timed])
    reqs = srv.build(timed, forms=[zc.ZC_FORM_NTT] * len(timed))
    results = srv.run(reqs, timeout_s=120)
    _check(reqs, results, expected)
    assert any(r["waited_for_memory"] for r in results)
    # never more scratch in flight than the pool
    events = sorted([(r["admit_s"], r["scratch_bytes"]) for r in results] +
                    [(r["done_s"], -r["scratch_bytes"]) for r in results], key=lambda e: (e[0], e[1]))
    live = 0
    for _, b in events:
        live += b
        assert live <= budget + (2 << 20) * len(results)


def test_oversize_request_fails_alone(ctx, expected):
    small = Shape(1, 9, 3)
    fp = ctx.scratch_bytes(small.gate, small.n, small.d, zc.ZC_FORM_SUMCHECK)
    srv = serve.Server(ctx, slots=2, hbm_budget_bytes=fp + (4 << 20))
    timed = [(0.0, small), (0.0, Shape(1, 16, 3)), (0.0, small)]
    srv.load_pool([s for _, s in timed])
    reqs = srv.build(timed, forms=[zc.ZC_FORM_SUMCHECK] * 3)
    with pytest.raises(zc.ZCError) as ei:
        srv.run(reqs, timeout_s=60)
    res = ei.value.results
    assert res[1]["status"] == zc.ZC_ERR_OOM
    _check([reqs[0], reqs[2]], [res[0], res[2]], expected)


def test_routed_by_measured_cost(ctx, expected):
    from paper_2606_16146_gb300.router import CostModel
    m = CostModel()
    m.calibrate(ctx, [(1, 3), (2, 8)], ns=[8, 10], reps=2)
    assert all(v > 0 for v in m.table.values())
    srv = serve.Server(ctx, model=m, slots=4, hbm_budget_bytes=4 << 30)
    timed = _timed(10, 0.001)
    srv.load_pool([s for _, s in timed if s.d in (3, 8)])
    timed = [(t, s) for t, s in timed if s.d in (3, 8)]
    reqs = srv.build(timed)
    for q in reqs:
        s = q["shape"]
        want = min((zc.ZC_FORM_SUMCHECK, zc.ZC_FORM_NTT), key=lambda f: m.predict(f, s.gate, s.n, s.d))
        assert q["form"] == want
    results = srv.run(reqs, timeout_s=60)
    _check(reqs, results, expected)


def test_distinct_witnesses_equal_alone(ctx):
    """Every request has its own witness (seed 4000 + i), so no two requests
    share inputs; served concurrently with arrivals that overlap, each proof
    equals the oracle's proof of that request alone."""
    import torch
    from paper_2606_16146_gb300 import witness
    shapes = [Shape(1, 10, 3), Shape(2, 9, 8), Shape(1, 14, 3), Shape(2, 11, 4), Shape(2, 8, 16),
              Shape(1, 11, 3), Shape(2, 13, 8), Shape(1, 9, 3)]
    reqs, want = [], []
    for i in range(24):
        s = shapes[(5 * i + 2) % len(shapes)]
        form = zc.ZC_FORM_NTT if i % 4 == 1 else (zc.ZC_FORM_SUMCHECK_EQ if i % 4 == 3 else zc.ZC_FORM_SUMCHECK)
        cols = witness.generate(s.gate, s.n, s.d, 4000 + i)
        if form == zc.ZC_FORM_NTT:
            want.append(oracle.prove_ntt(s.gate, s.n, s.d, cols)[0])
        elif form == zc.ZC_FORM_SUMCHECK_EQ:
            want.append(oracle.prove_sumcheck_eq(s.gate, s.n, s.d, cols))
        else:
            want.append(oracle.prove_sumcheck(s.gate, s.n, s.d, cols))
        reqs.append({"arrival_s": 0.00005 * i, "gate": s.gate, "n": s.n, "d": s.d, "form": form,
                     "cols": [torch.from_numpy(c).cuda() for c in cols],
                     "proof": torch.zeros(zc.proof_size(s.gate, s.n, s.d, form), dtype=torch.uint8,
                                          device="cuda")})
    # footprints are admitted in 2 MiB granules: the threshold is the second
    # smallest granule count, so both classes of request occur
    gran = 2 << 20
    fps = sorted({-(-ctx.scratch_bytes(q["gate"], q["n"], q["d"], q["form"]) // gran) * gran for q in reqs})
    assert len(fps) >= 2
    for prio in (0, fps[1]):
        for q in reqs:
            q["proof"].zero_()
        res = ctx.serve(reqs, slots=6, hbm_budget_bytes=2 << 30, timeout_s=120, priority_bytes=prio)
        assert all(r["status"] == 0 for r in res)
        assert max(r["slot"] for r in res) >= 2            # requests overlapped on several slots
        for q, r, w in zip(reqs, res, want):
            assert proof_bytes(q["proof"]) == w
            if prio:                                     # large requests only on slot 0, small ones never
                assert (r["slot"] == 0) == (r["scratch_bytes"] >= prio)
