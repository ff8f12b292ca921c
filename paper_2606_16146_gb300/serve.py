"""Served proving: witness pool on the device, routing, the request loop.

``Server`` keeps one device copy of the columns of every request shape (the
witness pool), routes each request to the SumCheck or NTT form with a
measured ``router.CostModel``, and hands the timed request list to the
native loop (``zc_serve``): admission by free slot and device-pool space,
continuous batching over streams, completion by event polling.  ``report``
turns the per-request times into latency percentiles and throughput.
"""
from __future__ import annotations

import numpy as np

from . import witness, workloads, zc
from .router import CostModel


class Server:
    def __init__(self, ctx: "zc.Context", model: CostModel | None = None, slots: int = 8,
                 hbm_budget_bytes: int = 180 << 30, in_order: bool = False, priority_bytes: int = 0):
        self.ctx = ctx
        self.model = model
        self.slots = slots
        self.budget = hbm_budget_bytes
        self.in_order = in_order
        self.priority_bytes = priority_bytes
        self.pool: dict[workloads.Shape, list] = {}

    def load_pool(self, shapes, seed_of=workloads.shape_seed) -> None:
        """Generate each shape's witness once and keep its columns on the device."""
        import torch
        for s in sorted(set(shapes), key=lambda s: (s.n, s.d)):
            if s in self.pool:
                continue
            cols = witness.generate(s.gate, s.n, s.d, seed_of(s))
            self.pool[s] = [torch.from_numpy(c).cuda() for c in cols]

    def route(self, s: workloads.Shape) -> int:
        if self.model is None:
            return zc.ZC_FORM_SUMCHECK

        def fits(form):
            return self.ctx.scratch_bytes(s.gate, s.n, s.d, form) <= self.budget
        return self.model.route(s.gate, s.n, s.d, fits=fits)

    def build(self, timed_shapes, forms=None) -> list[dict]:
        """Request records for zc_serve: [(arrival_s, Shape)] -> dicts with device buffers."""
        import torch
        reqs = []
        for i, (t, s) in enumerate(timed_shapes):
            form = forms[i] if forms is not None else self.route(s)
            proof = torch.zeros(zc.proof_size(s.gate, s.n, s.d, form), dtype=torch.uint8, device="cuda")
            reqs.append({"arrival_s": t, "gate": s.gate, "n": s.n, "d": s.d, "form": form,
                         "cols": self.pool[s], "proof": proof, "shape": s})
        return reqs

    def run(self, reqs: list[dict], timeout_s: float = 0.0) -> list[dict]:
        return self.ctx.serve(reqs, slots=self.slots, hbm_budget_bytes=self.budget,
                              in_order=self.in_order, timeout_s=timeout_s, priority_bytes=self.priority_bytes)


def report(reqs: list[dict], results: list[dict]) -> dict:
    """Latency (done - arrival) percentiles in ms, throughput, admission counts."""
    ok = [(q, r) for q, r in zip(reqs, results) if r["status"] == 0]
    lat = np.array([(r["done_s"] - q["arrival_s"]) * 1e3 for q, r in ok])
    wait = np.array([(r["admit_s"] - q["arrival_s"]) * 1e3 for q, r in ok])
    t_first = min(q["arrival_s"] for q in reqs) if reqs else 0.0
    t_last = max((r["done_s"] for _, r in ok), default=t_first)
    span = max(t_last - t_first, 1e-9)
    forms = {"sumcheck": sum(1 for q, _ in ok if q["form"] == zc.ZC_FORM_SUMCHECK),
             "ntt": sum(1 for q, _ in ok if q["form"] == zc.ZC_FORM_NTT)}
    return {
        "requests": len(reqs), "completed": len(ok),
        "failed": len(reqs) - len(ok),
        "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
        "mean_ms": float(lat.mean()) if len(lat) else None,
        "queue_wait_p50_ms": float(np.percentile(wait, 50)) if len(wait) else None,
        "proofs_per_s": len(ok) / span,
        "makespan_s": span,
        "admitted_on_arrival": int(np.sum(wait < 1.0)) if len(wait) else 0,
        "waited_for_memory": sum(1 for _, r in ok if r["waited_for_memory"]),
        "peak_slot": max((r["slot"] for _, r in ok), default=0) + 1,
        "forms": forms,
    }
