"""ZeroCheck prover benchmark (one JSON line on rank 0).

Workload: the Plonk-gate ZeroCheck at n = 22 (N = 2^22 rows, 8 columns,
1 GiB of columns), BLS12-381 scalar field, seeded synthetic witness (see
paper_2606_16146_gb300/witness.py).  One step = one SumCheck-form proof and
one NTT-form proof of the same witness, inputs resident in HBM, column
commitments precomputed (stage (1) of the prover workflow, untimed).  The
columns (1 GiB) exceed L2, so no flush is needed between steps.

Lines:
  value        device time per step (ms), CUDA events on the proving stream,
               max over ranks; with N GPUs every rank proves its own copy
               (replicas) and value = elapsed / (K * N).
  e2e          the same step through the C ABI with pinned host buffers:
               H2D of the columns, D2H of the proofs and the quotient.
  roofline     dominant kernel launch, integer-pipe bound: algorithmic
               modular multiplications / launch time against
               152 SMs x 64 IMAD/clk x 2.07 GHz / 272 IMAD per mulmod.
  cpu_baseline the CPU oracle on a bounded sample (n = 18), scaled to n = 22
               by the algorithmic-work ratio.
--impl reference times the CPU oracle instead (each step the n = 18 sample,
scaled), since the paper ships no implementation.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ZeroCheck prove ms (SumCheck vs NTT) by n, degree; served p50/p99 ms"
GATE, N_LOG, DEG = 1, 22, 3
SAMPLE_N = 18
SM_COUNT, IMAD_PER_CLK, SM_MAX_MHZ, IMAD_PER_MULMOD = 152, 64, 2070.0, 272
ALU_PEAK_MULMOD = SM_COUNT * IMAD_PER_CLK * SM_MAX_MHZ * 1e6 / IMAD_PER_MULMOD


def algorithmic_mulmods(form: str, n: int, d: int = 3, gate: int = 1) -> float:
    """Per-proof modular multiplications (the counts fixed for the roofline)."""
    N = 1 << n
    c = 8 if gate == 1 else d + 1
    g = 5 if gate == 1 else d - 1
    s = 1 << max(0, (d - 1).bit_length())
    M = s * N
    if form == "sumcheck":
        return (N - 1) * ((d + 1) * (g + 1) + 1 + c)
    return (c * (N / 2) * n + c * s * (N + (N / 2) * n) + M * (g + 1)
            + (M / 2) * math.log2(M) + M + c * N + (d - 1) * N)


def algorithmic_bytes(form: str, n: int, d: int = 3, gate: int = 1) -> float:
    N = 1 << n
    c = 8 if gate == 1 else d + 1
    s = 1 << max(0, (d - 1).bit_length())
    M = s * N
    if form == "sumcheck":
        return 128.0 * c * N
    return 32.0 * (2 * c * N + c * M + M + 2 * M + c * N + M)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows: list[list[str]] = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_sample(steps: int = 1) -> dict:
    """Time the CPU oracle on the n = SAMPLE_N witness; scale to n = N_LOG."""
    import oracle
    from paper_2606_16146_gb300 import witness
    cols = witness.generate(GATE, SAMPLE_N, DEG, 1000 + SAMPLE_N)
    roots = [oracle.root(c) for c in cols]
    ts, tn = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.prove_sumcheck(GATE, SAMPLE_N, DEG, cols, roots=roots)
        t1 = time.perf_counter()
        oracle.prove_ntt(GATE, SAMPLE_N, DEG, cols, roots=roots)
        t2 = time.perf_counter()
        ts.append(t1 - t0)
        tn.append(t2 - t1)
    ks = algorithmic_mulmods("sumcheck", N_LOG) / algorithmic_mulmods("sumcheck", SAMPLE_N)
    kn = algorithmic_mulmods("ntt", N_LOG) / algorithmic_mulmods("ntt", SAMPLE_N)
    sc_ms = float(np.median(ts)) * 1e3 * ks
    nt_ms = float(np.median(tn)) * 1e3 * kn
    return {"value": sc_ms + nt_ms, "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"one SumCheck and one NTT proof of the Plonk witness at n={SAMPLE_N}, "
                       f"scaled to n={N_LOG} by the algorithmic mulmod ratio "
                       f"(x{ks:.1f} SumCheck, x{kn:.1f} NTT)"),
            "sumcheck_ms": sc_ms, "ntt_ms": nt_ms, "raw_s": [float(np.median(ts)), float(np.median(tn))]}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("ZC_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def run_reference(args, world, rank):
    if rank != 0:
        return
    for _ in range(args.warmup):
        pass
    samples = [cpu_sample(1)["value"] for _ in range(args.steps)]
    base = cpu_sample(1)
    ms = float(np.median(samples))
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32x8 (255-bit field, exact)",
            "data": "synthetic", "config": workload_config(world),
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(world):
    return {"workload": f"Plonk-gate ZeroCheck, n={N_LOG} (N=2^{N_LOG}, 8 columns), both forms, "
                        "BLS12-381 Fr, seeded synthetic witness",
            "n": N_LOG, "d": DEG, "gate": "plonk", "forms": ["sumcheck", "ntt"], "lde": "4N coset, g=7",
            "parallelism": f"replicas x{world}", "l2": "inputs (1 GiB) larger than L2; no flush"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="override n (profiling smaller cases)")
    ap.add_argument("--form", default="both", choices=["both", "sumcheck", "ntt"],
                    help="restrict the step to one form (profiling); the bench line uses both")
    args = ap.parse_args()
    global N_LOG
    if args.n:
        N_LOG = args.n
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    from paper_2606_16146_gb300 import witness, zc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = zc.Context(local, max_n=24, max_d=8)
    cols = witness.generate(GATE, N_LOG, DEG, 1000 + N_LOG)
    dcols = [torch.from_numpy(c).to(dev) for c in cols]
    roots = ctx.roots(GATE, N_LOG, DEG, dcols)
    stream = torch.cuda.Stream(dev)
    N = 1 << N_LOG
    M = 4 * N
    ps_sc = zc.proof_size(GATE, N_LOG, DEG, zc.ZC_FORM_SUMCHECK)
    ps_nt = zc.proof_size(GATE, N_LOG, DEG, zc.ZC_FORM_NTT)
    p_sc = torch.zeros(ps_sc, dtype=torch.uint8, device=dev)
    p_nt = torch.zeros(ps_nt, dtype=torch.uint8, device=dev)
    q_dev = torch.zeros(M * 32, dtype=torch.uint8, device=dev)
    have_ntt = True

    run_sc = args.form in ("both", "sumcheck")
    if args.form == "sumcheck":
        have_ntt = False

    def step():
        nonlocal have_ntt
        st_sc = None
        if run_sc:
            ctx.prove_sumcheck(GATE, N_LOG, DEG, dcols, roots=roots, stream=stream, proof_out=p_sc)
            st_sc = ctx.stats()
        st_nt = None
        if have_ntt:
            try:
                ctx.prove_ntt(GATE, N_LOG, DEG, dcols, roots=roots, stream=stream, proof_out=p_nt, q_out=q_dev)
                st_nt = ctx.stats()
            except zc.ZCError as e:
                if e.status != 5:
                    raise
                have_ntt = False
        return st_sc, st_nt

    torch.cuda.synchronize()
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # per-form device times (separately, for the by-form breakdown)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    sc_ms, nt_ms, st_sc, st_nt = [], [], None, None
    for _ in range(3):
        with torch.cuda.stream(stream):
            e0.record(stream)
            if run_sc:
                ctx.prove_sumcheck(GATE, N_LOG, DEG, dcols, roots=roots, stream=stream, proof_out=p_sc)
            e1.record(stream)
        if run_sc:
            st_sc = ctx.stats()
        if have_ntt:
            ctx.prove_ntt(GATE, N_LOG, DEG, dcols, roots=roots, stream=stream, proof_out=p_nt, q_out=q_dev)
            e2.record(stream)
            st_nt = ctx.stats()
        stream.synchronize()
        sc_ms.append(e0.elapsed_time(e1))
        if have_ntt:
            nt_ms.append(e1.elapsed_time(e2))

    # ---- timed region
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    t0.record(stream)
    for _ in range(args.steps):
        a, b = step()
        launches += (int(a[9]) if a else 0) + (int(b[9]) if b else 0)
    t1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1)
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([elapsed], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    ms_per_step = elapsed / args.steps
    value = elapsed / (args.steps * world)

    # ---- end to end through the C ABI with pinned host buffers
    hcols = [torch.from_numpy(c).pin_memory() for c in cols]
    hq = torch.empty(M * 32, dtype=torch.uint8).pin_memory()
    e2e_ms = []
    for it in range(3):
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        ctx.prove_sumcheck(GATE, N_LOG, DEG, hcols, roots=roots, stream=stream)
        if have_ntt:
            ctx.prove_ntt(GATE, N_LOG, DEG, hcols, roots=roots, stream=stream, q_out=hq)
        stream.synchronize()
        e2e_ms.append((time.perf_counter() - t_a) * 1e3)
    h2d = 2 * 8 * N * 32 if have_ntt else 8 * N * 32
    d2h = ps_sc + ((ps_nt + M * 32) if have_ntt else 0)

    # ---- dominant kernel roofline (the longest single launch of the step)
    dom = st_nt if (st_nt and st_nt[6] > st_sc[6]) else st_sc
    dom_name = ("ntt slice-LDE pass" if dom is st_nt else "sumcheck round-1 evaluate kernel")
    dom_ms = dom[6]
    achieved = dom[7] / (dom_ms * 1e-3) if dom_ms > 0 else 0.0
    roof = {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": ALU_PEAK_MULMOD,
            "unit": "mulmod/s", "frac": achieved / ALU_PEAK_MULMOD, "traffic": None,
            "algorithmic_mulmods_per_launch": dom[7], "algorithmic_bytes_per_launch": dom[8],
            "hbm_gbs_at_algorithmic_bytes": dom[8] / (dom_ms * 1e-3) / 1e9 if dom_ms > 0 else None,
            "peak_note": "derived: 152 SMs x 64 IMAD/clk x 2070 MHz / 272 IMAD per mulmod"}
    by_form = {"sumcheck": {"ms": float(np.median(sc_ms)),
                            "roofline_ms": 1e3 * max(algorithmic_mulmods("sumcheck", N_LOG) / ALU_PEAK_MULMOD,
                                                      algorithmic_bytes("sumcheck", N_LOG) / 6674.2e9),
                            "phases_ms": [round(x, 4) for x in st_sc[:5]]}}
    by_form["sumcheck"]["roofline_frac"] = by_form["sumcheck"]["roofline_ms"] / by_form["sumcheck"]["ms"]
    if have_ntt:
        by_form["ntt"] = {"ms": float(np.median(nt_ms)),
                          "roofline_ms": 1e3 * max(algorithmic_mulmods("ntt", N_LOG) / ALU_PEAK_MULMOD,
                                                    algorithmic_bytes("ntt", N_LOG) / 6674.2e9),
                          "phases_ms": [round(x, 4) for x in st_nt[:6]]}
        by_form["ntt"]["roofline_frac"] = by_form["ntt"]["roofline_ms"] / by_form["ntt"]["ms"]
    else:
        by_form["ntt"] = {"status": "not built"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32x8 (255-bit field, exact)",
                "data": "synthetic", "config": workload_config(world),
                "e2e": {"value": float(np.median(e2e_ms)), "unit": "ms", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "roofline": roof, "clocks": clk, "by_form": by_form}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_sample(1)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
