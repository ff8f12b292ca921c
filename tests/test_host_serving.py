"""Host-side logic of the batched and served modes (no GPU): the seeded
workload lists, the cost model's prediction and routing, and the serving
report."""
import json

import numpy as np
import pytest

from paper_2606_16146_gb300 import costs, serve, workloads, zc
from paper_2606_16146_gb300.router import CostModel


def test_batched_instances_follow_the_recipe():
    a = workloads.batched_instances()
    assert a == workloads.batched_instances()
    assert len(a) == 64
    assert [seed for _, seed in a] == list(range(3000, 3064))
    ns = [s.n for s, _ in a]
    assert min(ns) >= 10 and max(ns) <= 20 and len(set(ns)) >= 8
    for s, _ in a:
        assert (s.gate, s.d) in ((1, 3), (2, 8))
    assert 16 <= sum(1 for s, _ in a if s.d == 3) <= 48


def test_served_requests_are_poisson():
    r = workloads.served_requests(rate=500.0, count=4000, seed=11)
    t = np.array([x for x, _ in r])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 500) < 0.1 / 500          # mean 1/rate
    assert abs(gaps.std() / gaps.mean() - 1) < 0.1          # exponential: cv = 1
    ns = [s.n for _, s in r]
    assert min(ns) == 12 and max(ns) == 24
    assert {s.d for _, s in r} == {3, 8, 16}
    assert all((s.gate == 1) == (s.d == 3) for _, s in r)


def test_cost_model_scales_by_work_and_routes():
    m = CostModel({(1, 1, 3, 20): 2.0, (2, 1, 3, 20): 10.0, (1, 2, 8, 18): 5.0, (2, 2, 8, 18): 1.0})
    assert m.predict(1, 1, 20, 3) == 2.0
    want = 2.0 * costs.algorithmic_mulmods("sumcheck", 22, 3, 1) / costs.algorithmic_mulmods("sumcheck", 20, 3, 1)
    assert m.predict(1, 1, 22, 3) == pytest.approx(want)
    assert m.route(1, 21, 3) == zc.ZC_FORM_SUMCHECK
    assert m.route(2, 18, 8) == zc.ZC_FORM_NTT
    assert m.route(2, 18, 8, fits=lambda f: f == zc.ZC_FORM_SUMCHECK) == zc.ZC_FORM_SUMCHECK
    with pytest.raises(ValueError):
        m.route(2, 18, 16)
    again = CostModel.from_json(m.to_json())
    assert again.table == m.table
    json.loads(m.to_json())


def test_serving_report():
    reqs = [{"arrival_s": 0.0, "form": 1}, {"arrival_s": 0.001, "form": 2}, {"arrival_s": 0.002, "form": 1},
            {"arrival_s": 0.003, "form": 1}]
    res = [{"admit_s": 0.0, "done_s": 0.010, "status": 0, "waited_for_memory": False, "slot": 0},
           {"admit_s": 0.001, "done_s": 0.021, "status": 0, "waited_for_memory": False, "slot": 1},
           {"admit_s": 0.010, "done_s": 0.030, "status": 0, "waited_for_memory": True, "slot": 0},
           {"admit_s": 0.003, "done_s": 0.003, "status": 2, "waited_for_memory": False, "slot": 0}]
    rep = serve.report(reqs, res)
    assert rep["completed"] == 3 and rep["failed"] == 1
    assert rep["p50_ms"] == pytest.approx(20.0)
    assert rep["proofs_per_s"] == pytest.approx(3 / 0.030)
    assert rep["waited_for_memory"] == 1
    assert rep["forms"] == {"sumcheck": 2, "ntt": 1}
    assert rep["admitted_on_arrival"] == 2
