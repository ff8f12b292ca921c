"""Cost-model routing between the two ZeroCheck forms.

The paper's comparison (Sec. 4) is exactly this question: for a gate of
degree d over 2^n rows, is the SumCheck form or the NTT form cheaper on the
hardware at hand?  The answer is measured, not assumed: ``calibrate`` times
single proofs of each form on the GPU at a few sizes per (gate, d); a size
that was not measured is predicted from the nearest measured one of the
same (form, gate, d), scaled by the ratio of algorithmic work (``costs``).
``route`` picks the form with the smaller predicted time, among the forms
whose scratch fits the memory the caller still has.
"""
from __future__ import annotations

import json

from . import costs, witness, zc

FORMS = {zc.ZC_FORM_SUMCHECK: "sumcheck", zc.ZC_FORM_NTT: "ntt"}


class CostModel:
    def __init__(self, table: dict | None = None):
        # (form, gate, d, n) -> measured ms per proof
        self.table: dict[tuple[int, int, int, int], float] = dict(table or {})

    # -- persistence --------------------------------------------------------
    def to_json(self) -> str:
        return json.dumps([[*k, v] for k, v in sorted(self.table.items())])

    @classmethod
    def from_json(cls, text: str) -> "CostModel":
        return cls({(int(f), int(g), int(d), int(n)): float(ms) for f, g, d, n, ms in json.loads(text)})

    # -- prediction ---------------------------------------------------------
    def predict(self, form: int, gate: int, n: int, d: int) -> float:
        key = (form, gate, d, n)
        if key in self.table:
            return self.table[key]
        same = [k for k in self.table if k[:3] == (form, gate, d)]
        if not same:
            raise KeyError(f"no measurement for form {form}, gate {gate}, d {d}")
        ref = min(same, key=lambda k: (abs(k[3] - n), -k[3]))
        name = FORMS[form]
        scale = (costs.algorithmic_mulmods(name, n, d, gate)
                 / costs.algorithmic_mulmods(name, ref[3], d, gate))
        return self.table[ref] * scale

    def route(self, gate: int, n: int, d: int, fits=None) -> int:
        """The form with the smaller predicted time; fits(form) -> bool filters."""
        best, best_ms = None, None
        for form in (zc.ZC_FORM_SUMCHECK, zc.ZC_FORM_NTT):
            if fits is not None and not fits(form):
                continue
            try:
                ms = self.predict(form, gate, n, d)
            except KeyError:
                continue
            if best_ms is None or ms < best_ms:
                best, best_ms = form, ms
        if best is None:
            raise ValueError(f"no form can take gate {gate}, n {n}, d {d}")
        return best

    # -- measurement --------------------------------------------------------
    def calibrate(self, ctx: "zc.Context", gate_degrees, ns, reps: int = 3, seed: int = 900) -> None:
        """Time one proof of each form for every (gate, d) in gate_degrees and n in ns."""
        import torch
        stream = torch.cuda.Stream()
        for gate, d in gate_degrees:
            for n in ns:
                cols = witness.generate(gate, n, d, seed + n)
                dcols = [torch.from_numpy(c).cuda() for c in cols]
                for form in (zc.ZC_FORM_SUMCHECK, zc.ZC_FORM_NTT):
                    proof = torch.empty(zc.proof_size(gate, n, d, form), dtype=torch.uint8, device="cuda")
                    run = ((lambda: ctx.prove_sumcheck(gate, n, d, dcols, stream=stream, proof_out=proof))
                           if form == zc.ZC_FORM_SUMCHECK else
                           (lambda: ctx.prove_ntt(gate, n, d, dcols, stream=stream, proof_out=proof, want_q=False)))
                    run()
                    times = []
                    for _ in range(reps):
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        run()
                        b.record(stream)
                        b.synchronize()
                        times.append(a.elapsed_time(b))
                    self.table[(form, gate, d, n)] = sorted(times)[len(times) // 2]
                del dcols
