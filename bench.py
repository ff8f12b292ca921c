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
               SMs x 64 IMAD/clk x max SM clock / 272 IMAD per mulmod, with
               the SM count and the maximum SM clock queried on the device.
  cpu_baseline the CPU oracle on the same n = 22 step (one SumCheck and one
               NTT proof, all host cores, measured once, no scaling), plus
               the SumCheck proof on one core.
--impl reference times the CPU oracle instead (the paper ships no
implementation): each step is the whole n = 22 step; the number of steps is
capped so that the run stays within a few minutes, and the line reports the
steps it ran.
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

from paper_2606_16146_gb300.costs import algorithmic_bytes, algorithmic_mulmods, blowup, ncols  # noqa: E402

METRIC = "ZeroCheck prove ms (SumCheck vs NTT) by n, degree; served p50/p99 ms"
GATE, N_LOG, DEG = 1, 22, 3
IMAD_PER_CLK, IMAD_PER_MULMOD = 64, 272
# GB300 figures, used only until the device has been queried (alu_peak)
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
ALU_PEAK_MULMOD = SM_COUNT * IMAD_PER_CLK * SM_MAX_MHZ * 1e6 / IMAD_PER_MULMOD
REF_BUDGET_S = 150.0   # reference arm: timed CPU work per run


def query_device(local: int) -> dict:
    """SM count (CUDA device properties) and maximum SM clock (nvidia-smi) of
    the GPU, and the integer-pipe roofline they give: SMs x 64 IMAD/clk x
    clock / 272 IMAD per modular multiplication."""
    import torch
    sms = int(torch.cuda.get_device_properties(local).multi_processor_count)
    mhz, src = None, "nvidia-smi clocks.max.sm"
    try:
        out = subprocess.run(["nvidia-smi", f"--id={local}", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=20).stdout.strip()
        mhz = float(out.splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        mhz, src = SM_MAX_MHZ, "fallback 2070 MHz (nvidia-smi unavailable)"
    return {"sm_count": sms, "sm_max_mhz": mhz, "clock_source": src,
            "alu_peak_mulmod_s": sms * IMAD_PER_CLK * mhz * 1e6 / IMAD_PER_MULMOD}


def set_alu_peak(local: int) -> dict:
    global SM_COUNT, SM_MAX_MHZ, ALU_PEAK_MULMOD
    info = query_device(local)
    SM_COUNT, SM_MAX_MHZ, ALU_PEAK_MULMOD = info["sm_count"], info["sm_max_mhz"], info["alu_peak_mulmod_s"]
    return info


def peak_note() -> str:
    return (f"queried: {SM_COUNT} SMs x {IMAD_PER_CLK} IMAD/clk x {SM_MAX_MHZ:.0f} MHz / "
            f"{IMAD_PER_MULMOD} IMAD per mulmod")


def _hbm_peak_bytes_s() -> float:
    """Measured HBM copy bandwidth of this GPU model (bytes/s), else the fallback 6.8 TB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]) * 1e9
    except (OSError, KeyError, ValueError):
        return 6.8e12


HBM_PEAK = _hbm_peak_bytes_s()

TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "ntt_pass_plonk_n22_traffic.md")


def recorded_traffic(path: str = TRAFFIC_RECORD):
    """DRAM bytes per launch of the dominant kernel from a committed ncu record,
    or None when the kernel sources changed since the counters were taken."""
    import hashlib
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "sources",
                                                              "source_sha256")):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
        h = hashlib.sha256()
        for rel in fields["sources"].split(","):
            with open(os.path.join(ROOT, rel.strip()), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != fields["source_sha256"]:
            return None
        return float(fields["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


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


def cpu_model() -> str:
    """The host CPU's model name (as /proc/cpuinfo or lscpu report it)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def _oracle_step(cols, roots):
    """One SumCheck and one NTT proof by the oracle: (sumcheck s, ntt s)."""
    import oracle
    t0 = time.perf_counter()
    oracle.prove_sumcheck(GATE, N_LOG, DEG, cols, roots=roots)
    t1 = time.perf_counter()
    oracle.prove_ntt(GATE, N_LOG, DEG, cols, roots=roots)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


_ONE_CORE_SCRIPT = """
import json, sys, time
sys.path.insert(0, sys.argv[1])
import oracle
from paper_2606_16146_gb300 import witness
g, n, d, seed = (int(x) for x in sys.argv[2:6])
cols = witness.generate(g, n, d, seed)
roots = [oracle.root(c) for c in cols]
t0 = time.perf_counter()
oracle.prove_sumcheck(g, n, d, cols, roots=roots)
print(json.dumps({"s": time.perf_counter() - t0, "threads": oracle.num_threads()}))
"""


def cpu_one_core_sumcheck() -> dict | None:
    """The oracle's SumCheck proof of the same witness on one core (a child
    process with OMP_NUM_THREADS=1)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", _ONE_CORE_SCRIPT, ROOT, str(GATE), str(N_LOG), str(DEG),
                              str(1000 + N_LOG)], capture_output=True, text=True, env=env, timeout=600,
                             check=True).stdout
        r = json.loads(out.strip().splitlines()[-1])
        return {"sumcheck_ms": r["s"] * 1e3, "cores": r["threads"]}
    except (OSError, ValueError, IndexError, subprocess.SubprocessError) as e:
        return {"error": str(e)[:200]}


def cpu_sample() -> dict:
    """The CPU oracle on the bench step itself (Plonk n = 22, one proof of each
    form, roots given), all host cores, measured once with no scaling; plus the
    SumCheck proof on one core."""
    import oracle
    from paper_2606_16146_gb300 import witness
    cols = witness.generate(GATE, N_LOG, DEG, 1000 + N_LOG)
    roots = [oracle.root(c) for c in cols]
    ts, tn = _oracle_step(cols, roots)
    del cols
    one = cpu_one_core_sumcheck()
    return {"value": (ts + tn) * 1e3, "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
            "cpu": cpu_model(),
            "sample": (f"the bench step itself: one SumCheck and one NTT proof of the Plonk witness at "
                       f"n={N_LOG} (seed {1000 + N_LOG}, roots given), measured once on all host cores, "
                       f"no scaling"),
            "sumcheck_ms": ts * 1e3, "ntt_ms": tn * 1e3, "one_core": one}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("ZC_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest value over all ranks (replicas: the slowest rank's time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_reference(args, world, rank):
    """The CPU oracle on the bench step (Plonk n = 22, one proof of each form):
    every step is the whole step, measured, with no scaling.  A step takes the
    oracle tens of seconds, so warm-up steps are skipped and the timed steps
    are capped at what fits REF_BUDGET_S (at least one); the line reports the
    steps it ran."""
    if rank != 0:
        return
    import oracle
    from paper_2606_16146_gb300 import witness
    cols = witness.generate(GATE, N_LOG, DEG, 1000 + N_LOG)
    roots = [oracle.root(c) for c in cols]
    per = []
    t_start = time.perf_counter()
    while len(per) < max(1, args.steps):
        ts, tn = _oracle_step(cols, roots)
        per.append((ts + tn) * 1e3)
        spent = time.perf_counter() - t_start
        if spent + spent / len(per) > REF_BUDGET_S:
            break
    ms = float(np.median(per))
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": len(per), "warmup": 0, "steps_requested": args.steps, "warmup_requested": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32x8 (255-bit field, exact)", "data": "synthetic", "config": workload_config(world),
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
                             "cpu": cpu_model(),
                             "sample": (f"each step the whole bench step: one SumCheck and one NTT proof of "
                                        f"the Plonk witness at n={N_LOG} by the CPU oracle, roots given; "
                                        f"{len(per)} steps (capped to ~{REF_BUDGET_S:.0f} s of CPU work), "
                                        f"no warm-up, no scaling")},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "step_ms": per}
    print(json.dumps(line), flush=True)


def workload_config(world):
    return {"workload": f"Plonk-gate ZeroCheck, n={N_LOG} (N=2^{N_LOG}, 8 columns), both forms, "
                        "BLS12-381 Fr, seeded synthetic witness",
            "n": N_LOG, "d": DEG, "gate": "plonk", "forms": ["sumcheck", "ntt"], "lde": "4N coset, g=7",
            "parallelism": f"replicas x{world}", "l2": "inputs (1 GiB) larger than L2; no flush"}


def _median_event_ms(fn, stream, reps):
    import torch
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts)), ts


def _base_line(args, world, value, unit, hib, config):
    return {"metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": hib, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32x8 (255-bit field, exact)", "data": "synthetic",
            "config": config}


def run_batched(args, world, rank, local):
    """64 mixed instances (n 10..20 log-uniform, Plonk d=3 / product d=8), seeds
    3000+i: one CUDA graph per batch against 64 sequential plain calls, for
    all-SumCheck, all-NTT and cost-model-routed form assignments."""
    import torch
    device_info = set_alu_peak(local)
    from paper_2606_16146_gb300 import tune, witness, workloads, zc
    from paper_2606_16146_gb300.router import CostModel
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = zc.Context(local, max_n=24, max_d=8)
    inst = workloads.batched_instances()
    cols = [witness.generate(s.gate, s.n, s.d, seed) for s, seed in inst]
    dcols = [[torch.from_numpy(c).to(dev) for c in cc] for cc in cols]
    stream = torch.cuda.Stream(dev)
    model = CostModel()
    model.calibrate(ctx, [(1, 3), (2, 8)], ns=[10, 12, 14, 16, 18, 20], reps=3)
    variants = {
        "sumcheck": [zc.ZC_FORM_SUMCHECK] * len(inst),
        "ntt": [zc.ZC_FORM_NTT] * len(inst),
        "routed": [model.route(s.gate, s.n, s.d) for s, _ in inst],
    }
    params = [(s.gate, s.n, s.d, 0) for s, _ in inst]
    out = {}
    K, W = args.steps, max(3, args.warmup)
    for name, forms in variants.items():
        seq_p = [torch.zeros(zc.proof_size(s.gate, s.n, s.d, f), dtype=torch.uint8, device=dev)
                 for (s, _), f in zip(inst, forms)]
        bat_p = [torch.zeros_like(x) for x in seq_p]

        def sequential():
            for (s, _), f, dc, pr in zip(inst, forms, dcols, seq_p):
                if f == zc.ZC_FORM_SUMCHECK:
                    ctx.prove_sumcheck(s.gate, s.n, s.d, dc, stream=stream, proof_out=pr)
                else:
                    ctx.prove_ntt(s.gate, s.n, s.d, dc, stream=stream, proof_out=pr, want_q=False)
        for _ in range(W):
            sequential()
        seq_ms, _ = _median_event_ms(sequential, stream, K)
        tuned = tune.tune_batch(ctx, forms, params, dcols, bat_p, None, reps=3)
        g = ctx.batch_graph(forms, params, dcols, bat_p, None)
        for _ in range(W):
            g.launch(stream)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        bat_ms, _ = _median_event_ms(lambda: g.launch(stream), stream, K)
        clk = clocks.stop()
        torch.cuda.synchronize()
        exact = all(a.cpu().numpy().tobytes() == b.cpu().numpy().tobytes() for a, b in zip(seq_p, bat_p))
        mm = sum(algorithmic_mulmods("sumcheck" if f == 1 else "ntt", s.n, s.d, s.gate)
                 for (s, _), f in zip(inst, forms))
        out[name] = {"sequential_ms": seq_ms, "batched_ms": bat_ms, "speedup": seq_ms / bat_ms,
                     "proofs_per_s": len(inst) / (bat_ms * 1e-3),
                     "sequential_proofs_per_s": len(inst) / (seq_ms * 1e-3),
                     "exact_vs_sequential": exact, "graph_kernels": g.kernels,
                     "forms": {"sumcheck": forms.count(1), "ntt": forms.count(2)},
                     "tuned": {"settings": tuned["best"], "trials": len(tuned["trials"]),
                               "untuned_ms": tuned["trials"][0][2]},
                     "alu_frac": mm / (bat_ms * 1e-3) / ALU_PEAK_MULMOD, "clocks": clk}
        last_graph = g
    best = out["routed"]
    # end to end: columns from pinned host memory, one graph launch, proofs back
    hcols = [[torch.from_numpy(c).pin_memory() for c in cc] for cc in cols]
    forms = variants["routed"]
    proofs = [torch.zeros(zc.proof_size(s.gate, s.n, s.d, f), dtype=torch.uint8, device=dev)
              for (s, _), f in zip(inst, forms)]
    g = ctx.batch_graph(forms, params, dcols, proofs, None)
    hp = [torch.empty(x.numel(), dtype=torch.uint8).pin_memory() for x in proofs]
    e2e = []
    for _ in range(3):
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        with torch.cuda.stream(stream):
            for dc, hc in zip(dcols, hcols):
                for d_, h_ in zip(dc, hc):
                    d_.copy_(h_, non_blocking=True)
            g.launch(stream)
            for d_, h_ in zip(proofs, hp):
                h_.copy_(d_, non_blocking=True)
        stream.synchronize()
        e2e.append((time.perf_counter() - t_a) * 1e3)
    h2d = sum(c.nbytes for cc in cols for c in cc)
    d2h = sum(x.numel() for x in proofs)
    mm = sum(algorithmic_mulmods("sumcheck" if f == 1 else "ntt", s.n, s.d, s.gate)
             for (s, _), f in zip(inst, forms))
    achieved = mm / (best["batched_ms"] * 1e-3)
    config = {"workload": "batched: 64 ZeroCheck instances, n log-uniform 10..20, Plonk d=3 / product "
                          "d=8 with equal probability, seeds 3000+i, one CUDA graph per batch; baseline "
                          "64 sequential plain calls on one stream",
              "instances": len(inst), "n_range": [10, 20], "degrees": [3, 8],
              "parallelism": f"replicas x{world}", "l2": "batch columns (~GBs) larger than L2; no flush"}
    line = _base_line(args, world, best["batched_ms"], "ms", False, config)
    line["ms_per_step"] = best["batched_ms"]
    line["proofs_per_s"] = best["proofs_per_s"]
    line["by_variant"] = out
    line["e2e"] = {"value": float(np.median(e2e)), "unit": "ms", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h}
    line["gpu_launches"] = best["graph_kernels"] * args.steps
    line["roofline"] = {"bound": "alu", "kernel": "whole batch graph (all instances)", "achieved": achieved,
                        "peak": ALU_PEAK_MULMOD, "unit": "mulmod/s", "frac": achieved / ALU_PEAK_MULMOD,
                        "traffic": None,
                        "peak_note": peak_note()}
    line["clocks"] = best["clocks"]
    line["cost_model_ms"] = [[*k, v] for k, v in sorted(model.table.items())]
    line["device"] = device_info
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_sample_batched(inst, cols, forms)
    if rank == 0:
        print(json.dumps(line), flush=True)
    del last_graph, g
    ctx.close()


def cpu_sample_batched(inst, cols, forms):
    """Oracle on the instances with n <= 14 of the batch, scaled to the whole batch by work."""
    import oracle
    t_s, mm_s, mm_all = 0.0, 0.0, 0.0
    for (s, _), cc, f in zip(inst, cols, forms):
        name = "sumcheck" if f == 1 else "ntt"
        w = algorithmic_mulmods(name, s.n, s.d, s.gate)
        mm_all += w
        if s.n > 14:
            continue
        t0 = time.perf_counter()
        if f == 1:
            oracle.prove_sumcheck(s.gate, s.n, s.d, cc)
        else:
            oracle.prove_ntt(s.gate, s.n, s.d, cc)
        t_s += time.perf_counter() - t0
        mm_s += w
    ms = t_s * 1e3 * mm_all / mm_s
    return {"value": ms, "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"the batch's instances with n <= 14 (routed forms), {t_s:.2f} s, scaled to "
                      f"all 64 by algorithmic mulmods (x{mm_all / mm_s:.1f})"}


# (gate, n, d[, NTT domain word]): Plonk n = 12, 20, 22 and the product gate
# at n = 22, then the other domains of Sec. 4's degree scaling: Plonk on the
# quotient-sized 2N and the step-radix 3N = 2N + N; the product gate d = 4 on
# 3N (against its default 4N) and d = 6 on 5N = 4N + N (against 8N).
SWEEP = [(1, 12, 3), (1, 20, 3), (1, 22, 3), (2, 22, 2), (2, 22, 4), (2, 22, 8), (2, 22, 16), (2, 22, 32),
         (1, 22, 3, 1), (1, 22, 3, 0x101), (2, 22, 4, 0x101), (2, 22, 6), (2, 22, 6, 0x102)]


def _time_shapes(local, shapes, K, W, seed_of, label_of):
    """One proof of each form at a time per (gate, n, d) shape, column roots
    given (untimed): median CUDA-event ms, roofline ms and fraction, phases."""
    import torch
    set_alu_peak(local)
    from paper_2606_16146_gb300 import witness, zc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = zc.Context(local, max_n=24, max_d=32)
    stream = torch.cuda.Stream(dev)
    rows = []
    clocks = ClockSampler(local)
    clocks.start()
    for shape in shapes:
        gate, n, d = shape[:3]
        lb = shape[3] if len(shape) > 3 else 0
        cols = witness.generate(gate, n, d, seed_of(gate, n, d))
        dcols = [torch.from_numpy(c).to(dev) for c in cols]
        del cols
        roots = ctx.roots(gate, n, d, dcols)
        row = {"gate": label_of(gate, d), "n": n, "d": d}
        if lb:
            row["ntt_log_blowup"] = lb
        for form, name in ((zc.ZC_FORM_SUMCHECK, "sumcheck"), (zc.ZC_FORM_NTT, "ntt")):
            proof = torch.zeros(zc.proof_size(gate, n, d, form), dtype=torch.uint8, device=dev)
            if form == zc.ZC_FORM_SUMCHECK:
                def fn():
                    ctx.prove_sumcheck(gate, n, d, dcols, roots=roots, stream=stream, proof_out=proof)
            else:
                def fn():
                    ctx.prove_ntt(gate, n, d, dcols, roots=roots, stream=stream, proof_out=proof,
                                  want_q=False, log_blowup=lb)
            for _ in range(W):
                fn()
            ms, _ = _median_event_ms(fn, stream, K)
            roof = 1e3 * max(algorithmic_mulmods(name, n, d, gate, lb) / ALU_PEAK_MULMOD,
                             algorithmic_bytes(name, n, d, gate, lb) / HBM_PEAK)
            row[name] = {"ms": ms, "roofline_ms": roof, "roofline_frac": roof / ms,
                         "phases_ms": [round(x, 4) for x in ctx.stats()[:6]]}
        rows.append(row)
        del dcols
        torch.cuda.empty_cache()
    clk = clocks.stop()
    ctx.close()
    return rows, clk


def run_sweep(args, world, rank, local):
    """Both forms, one proof at a time, over the plain and high-degree shapes:
    Plonk n = 12, 20, 22 and the product gate at n = 22 for d = 2..32."""
    K, W = max(1, args.steps), max(3, args.warmup)
    rows, clk = _time_shapes(local, SWEEP, K, W,
                             lambda g, n, d: 1000 + n if g == 1 else 2000 + 10 * d + n,
                             lambda g, d: "plonk" if g == 1 else "product")
    head = rows[2]
    config = {"workload": "sweep: one proof of each form at a time; Plonk n=12, 20, 22 and product gate "
                          "n=22, d in {2, 4, 8, 16, 32}; NTT domains 2N and 3N = 2N + N for Plonk n=22, "
                          "3N for d=4 and 5N = 4N + N against 8N for d=6; column roots given (untimed)",
              "parallelism": f"replicas x{world}", "l2": "n >= 20 inputs larger than L2; no flush"}
    line = _base_line(args, world, head["sumcheck"]["ms"] + head["ntt"]["ms"], "ms", False, config)
    line["value_is"] = "Plonk n=22: SumCheck ms + NTT ms"
    line["rows"] = rows
    line["clocks"] = clk
    line["e2e"] = None
    line["e2e_note"] = "device-resident columns; the plain workload line carries the host-buffer run"
    if rank == 0:
        print(json.dumps(line), flush=True)


# The paper's polynomials (Sec. 5, Table poly_examples) as sum gates: (name, m, d)
FAMILY = [("g1g2", 0, 2), ("g1g2+g3", 1, 2), ("g1g2+g3+g4", 2, 2), ("g1g2+g3+g4+g5", 3, 2),
          ("g1g2g3", 0, 3), ("g1g2g3g4", 0, 4)]
FAMILY_N = (18, 20, 22, 24)


def run_family(args, world, rank, local):
    """The paper's workload family through the sum gate, both forms, one proof
    at a time, at N = 2^18 .. 2^24 (the paper sweeps 2^17 .. 2^32)."""
    from paper_2606_16146_gb300 import witness
    K, W = max(1, args.steps), max(3, args.warmup)
    names = {(witness.gate_sum(m), d): name for name, m, d in FAMILY}
    shapes = [(witness.gate_sum(m), n, d) for n in FAMILY_N for _, m, d in FAMILY]
    # g1g2g3 again on the quotient-sized 2N domain (Sec. 4 sizes its transform at 2N)
    shapes += [(witness.gate_sum(0), n, 3, 1) for n in FAMILY_N]
    rows, clk = _time_shapes(local, shapes, K, W,
                             lambda g, n, d: 7000 + 100 * (g >> 8) + 10 * d + n,
                             lambda g, d: names[(g, d)])
    config = {"workload": "family: the paper's six polynomials (g1g2, g1g2+g3, g1g2+g3+g4, "
                          "g1g2+g3+g4+g5, g1g2g3, g1g2g3g4) as sum gates, one proof of each form at "
                          "a time, n in {18, 20, 22, 24}, plus g1g2g3 on the 2N domain; column roots "
                          "given (untimed)",
              "parallelism": f"replicas x{world}", "l2": "n >= 20 inputs larger than L2; no flush"}
    at22 = [r for r in rows if r["n"] == 22 and "ntt_log_blowup" not in r]
    line = _base_line(args, world, sum(r["sumcheck"]["ms"] + r["ntt"]["ms"] for r in at22), "ms",
                      False, config)
    line["value_is"] = "n=22: sum over the six polynomials of SumCheck ms + NTT ms"
    line["rows"] = rows
    line["clocks"] = clk
    line["e2e"] = None
    line["e2e_note"] = "device-resident columns; the plain workload line carries the host-buffer run"
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_pcs(args, world, rank, local):
    """The hash-based commitment around the ZeroCheck (stages (1) and (3) of
    the prover workflow): commit to the Plonk n = 22 witness, prove the
    SumCheck form with the commitment as every column root, recover the
    point from the proof, open there, verify on the host."""
    import torch
    from paper_2606_16146_gb300 import witness, zc
    torch.cuda.set_device(local)
    device_info = set_alu_peak(local)
    ctx = zc.Context(local, max_n=24, max_d=8)
    n, t = N_LOG, args.pcs_queries
    cols = witness.generate(GATE, n, DEG, 1000 + n)
    dcols = [torch.from_numpy(c).cuda() for c in cols]
    c = len(cols)
    stream = torch.cuda.Stream()
    K, W = max(1, args.steps), max(3, args.warmup)

    def timed(fn, reps):
        ts, out = [], None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(ts)), out

    for _ in range(W):
        ctx.pcs_commit(n, dcols, t, stream=stream).close()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    cms = []
    for _ in range(K):
        ms, com = timed(lambda: ctx.pcs_commit(n, dcols, t, stream=stream), 1)
        cms.append(ms)
        if len(cms) < K:
            com.close()
    commit_ms = float(np.median(cms))
    roots = [com.root] * c
    proof = torch.zeros(zc.proof_size(GATE, n, DEG, 1), dtype=torch.uint8, device="cuda")
    sc_ms, _ = timed(lambda: ctx.prove_sumcheck(GATE, n, DEG, dcols, roots=roots, stream=stream,
                                                proof_out=proof), K)
    pb = proof.cpu().numpy().tobytes()
    zc.sumcheck_point(GATE, n, DEG, 1, roots, pb)  # first call builds the host constants
    pt_ms, (alpha, vals, ok) = timed(lambda: zc.sumcheck_point(GATE, n, DEG, 1, roots, pb), K)
    open_ms, pr = timed(lambda: com.open(alpha, vals, stream=stream), K)
    clk = clocks.stop()
    t0 = time.perf_counter()
    accept = zc.pcs_verify(n, c, t, com.root, alpha, vals, pr)
    verify_ms = (time.perf_counter() - t0) * 1e3
    com.close()
    N = 1 << n
    config = {"workload": f"hash-based commitment around the ZeroCheck: Plonk n={n} (8 columns), rate-1/4 "
                          f"Reed-Solomon rows of 2^{min(n, 12)}, {t} queries; commit, SumCheck proof with "
                          "the commitment as every column root, point replay, opening, host verification",
              "n": n, "columns": c, "queries": t, "parallelism": f"replicas x{world}"}
    line = _base_line(args, world, commit_ms + sc_ms + open_ms, "ms", False, config)
    line["value_is"] = "commit + SumCheck proof + opening (device work, host-timed with synchronisation)"
    line["phases_ms"] = {"commit": commit_ms, "sumcheck": sc_ms, "point_replay_host": pt_ms, "open": open_ms,
                         "verify_host": verify_ms}
    line["sizes_bytes"] = {"columns": c * N * 32, "encoded": 4 * c * N * 32, "opening_proof": len(pr),
                           "sumcheck_proof": len(pb)}
    line["verified"] = bool(accept and ok)
    line["clocks"] = clk
    line["device"] = device_info
    line["e2e"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_served(args, world, rank, local):
    """Poisson request loop (n 12..24, d in {3, 8, 16}), admission by HBM
    footprint against a 180 GB pool, cost-model routing; against the same
    requests one at a time (one slot)."""
    import torch
    device_info = set_alu_peak(local)
    from paper_2606_16146_gb300 import serve, workloads, zc
    from paper_2606_16146_gb300.router import CostModel
    torch.cuda.set_device(local)
    ctx = zc.Context(local, max_n=24, max_d=16)
    model = CostModel()
    # measured over the whole served range of n (no extrapolation past n = 24)
    model.calibrate(ctx, [(1, 3), (2, 8), (2, 16)], ns=[12, 14, 16, 18, 20, 22, 24], reps=3)
    rates = [float(r) for r in args.rates.split(",")]
    lists = {r: workloads.served_requests(r, args.requests) for r in rates}
    budget = 180 * 10**9
    prio_bytes = 1 << 30   # requests with >= 1 GiB of scratch (the n >= 22 shapes) get the priority slot
    srv = serve.Server(ctx, model=model, slots=8, hbm_budget_bytes=budget, priority_bytes=prio_bytes)
    flat = serve.Server(ctx, model=model, slots=8, hbm_budget_bytes=budget)
    one = serve.Server(ctx, model=model, slots=1, hbm_budget_bytes=budget, in_order=True)
    t_pool = time.perf_counter()
    srv.load_pool([s for lst in lists.values() for _, s in lst])
    t_pool = time.perf_counter() - t_pool
    one.pool = srv.pool
    flat.pool = srv.pool
    # warm-up: every shape once through the loop (tables, lanes, pool allocation)
    warm = [(0.0, s) for s in sorted(srv.pool, key=lambda s: (s.n, s.d))]
    srv.run(srv.build(warm))
    one.run(one.build(warm))
    if args.served_ntt > 0:
        srv.run(srv.build(warm, [zc.ZC_FORM_NTT] * len(warm)))
    torch.cuda.synchronize()
    rows = {}
    clocks = ClockSampler(local)
    clocks.start()
    launches = 0
    for r, lst in lists.items():
        reqs = srv.build(lst)
        res = srv.run(reqs)
        launches += ctx.stats()[9]
        rep = serve.report(reqs, res)
        base_reqs = one.build(lst)
        base = serve.report(base_reqs, one.run(base_reqs))
        flat_reqs = flat.build(lst)
        flat_rep = serve.report(flat_reqs, flat.run(flat_reqs))
        exact = all(a["proof"].cpu().numpy().tobytes() == b["proof"].cpu().numpy().tobytes()
                    == c["proof"].cpu().numpy().tobytes() for a, b, c in zip(reqs, base_reqs, flat_reqs))
        rows[str(int(r))] = {"served": rep, "one_at_a_time": base, "served_no_priority_slot": flat_rep,
                             "exact_vs_one_at_a_time": exact}
    # the NTT form through the same loop: every request forced to NTT (the cost
    # model never picks it for this mix), served against one at a time
    ntt_rows = {}
    if args.served_ntt > 0:
        for r in [float(x) for x in args.served_ntt_rates.split(",")]:
            lst = workloads.served_requests(r, args.served_ntt)
            srv.load_pool([sh for _, sh in lst])
            forms = [zc.ZC_FORM_NTT] * len(lst)
            reqs = srv.build(lst, forms)
            rep = serve.report(reqs, srv.run(reqs))
            launches += ctx.stats()[9]
            base_reqs = one.build(lst, forms)
            base = serve.report(base_reqs, one.run(base_reqs))
            exact = all(a["proof"].cpu().numpy().tobytes() == b["proof"].cpu().numpy().tobytes()
                        for a, b in zip(reqs, base_reqs))
            ntt_rows[str(int(r))] = {"served": rep, "one_at_a_time": base, "exact_vs_one_at_a_time": exact}
    clk = clocks.stop()
    mid = rows[str(int(rates[len(rates) // 2]))]["served"]
    config = {"workload": "served: Poisson arrivals, n uniform 12..24, d in {3 (Plonk), 8, 16 (product)}, "
                          "witness pool per shape on the device, admission by scratch footprint against "
                          "a 180 GB pool, 8 slots (requests with >= 1 GiB of scratch one at a time on a "
                          "high-priority slot), cost-model routing calibrated at n = 12..24; baselines: "
                          "the same requests one at a time (1 slot) and on 8 equal slots",
              "rates_req_s": rates, "requests_per_rate": args.requests, "slots": 8, "priority_bytes": prio_bytes,
              "hbm_budget_bytes": budget, "parallelism": f"replicas x{world}",
              "l2": "pool witnesses (tens of GB) larger than L2; no flush"}
    line = _base_line(args, world, mid["p99_ms"], "ms", False, config)
    line["value_is"] = f"p99 latency at {int(rates[len(rates) // 2])} req/s"
    line["by_rate"] = rows
    if ntt_rows:
        line["ntt_forced_by_rate"] = ntt_rows
        line["ntt_forced_requests_per_rate"] = args.served_ntt
    line["gpu_launches"] = int(launches)
    line["clocks"] = clk
    line["pool_setup_s"] = t_pool
    line["device"] = device_info
    line["cost_model_ms"] = [[*k, v] for k, v in sorted(model.table.items())]
    line["e2e"] = None
    line["e2e_note"] = ("latencies are host-observed from arrival to completion; request columns come "
                        "from the device-resident witness pool, so there is no separate host-buffer run")
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="override n (profiling smaller cases)")
    ap.add_argument("--d", type=int, default=None,
                    help="override the degree (profiling; d != 3 or --gate 2 uses the product gate)")
    ap.add_argument("--gate", type=int, default=1, choices=[1, 2])
    ap.add_argument("--form", default="both", choices=["both", "sumcheck", "ntt"],
                    help="restrict the step to one form (profiling); the bench line uses both")
    ap.add_argument("--pcs-queries", type=int, default=189, help="pcs: queried positions of an opening")
    ap.add_argument("--workload", default="plain", choices=["plain", "batched", "served", "sweep", "family", "pcs"],
                    help="plain: one Plonk n=22 proof per form (the headline line); batched: 64 "
                         "mixed instances in one graph; served: Poisson request loop; sweep: "
                         "sizes and degrees; family: the paper's polynomials as sum gates; pcs: the "
                         "hash-based commitment around the ZeroCheck")
    ap.add_argument("--rates", default="50,100,200,500,1000,2000", help="served: arrival rates (req/s)")
    ap.add_argument("--requests", type=int, default=200, help="served: requests per rate")
    ap.add_argument("--served-ntt", type=int, default=0,
                    help="served: also run this many requests per rate with every request forced to the NTT form")
    ap.add_argument("--served-ntt-rates", default="5,20", help="served: arrival rates of the forced-NTT runs")
    args = ap.parse_args()
    global N_LOG, GATE, DEG
    if args.n:
        N_LOG = args.n
    if args.d:
        GATE, DEG = (1, 3) if args.d == 3 and args.gate != 2 else (2, args.d)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batched":
        run_batched(args, world, rank, local)
        return
    if args.workload == "served":
        run_served(args, world, rank, local)
        return
    if args.workload == "sweep":
        run_sweep(args, world, rank, local)
        return
    if args.workload == "family":
        run_family(args, world, rank, local)
        return
    if args.workload == "pcs":
        run_pcs(args, world, rank, local)
        return
    import torch
    from paper_2606_16146_gb300 import witness, zc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    device_info = set_alu_peak(local)
    ctx = zc.Context(local, max_n=24, max_d=8)
    cols = witness.generate(GATE, N_LOG, DEG, 1000 + N_LOG)
    dcols = [torch.from_numpy(c).to(dev) for c in cols]
    roots = ctx.roots(GATE, N_LOG, DEG, dcols)
    stream = torch.cuda.Stream(dev)
    N = 1 << N_LOG
    M = blowup(DEG) * N
    C = ncols(GATE, DEG)
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
        """One step on one stream (also finds out whether the NTT form is built)."""
        nonlocal have_ntt
        if run_sc:
            ctx.prove_sumcheck(GATE, N_LOG, DEG, dcols, roots=roots, stream=stream, proof_out=p_sc)
        if have_ntt:
            try:
                ctx.prove_ntt(GATE, N_LOG, DEG, dcols, roots=roots, stream=stream, proof_out=p_nt, q_out=q_dev)
            except zc.ZCError as e:
                if e.status != 5:
                    raise
                have_ntt = False

    torch.cuda.synchronize()
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # The timed step runs its two proofs on two streams (the SumCheck proof on a
    # context of its own), forked from and joined back into the proving stream
    # every step, so the SumCheck proof's latency-bound stretches overlap the
    # NTT passes.  No call inside the timed region waits on the device.
    two_streams = run_sc and have_ntt
    if two_streams:
        ctx_sc = zc.Context(local, max_n=24, max_d=8)
        stream_sc = torch.cuda.Stream(dev)
        p_sc2 = torch.zeros(ps_sc, dtype=torch.uint8, device=dev)

    def step2():
        fork = torch.cuda.Event()
        fork.record(stream)
        stream_sc.wait_event(fork)
        ctx_sc.prove_sumcheck(GATE, N_LOG, DEG, dcols, roots=roots, stream=stream_sc, proof_out=p_sc2)
        ctx.prove_ntt(GATE, N_LOG, DEG, dcols, roots=roots, stream=stream, proof_out=p_nt, q_out=q_dev)
        join = torch.cuda.Event()
        join.record(stream_sc)
        stream.wait_event(join)

    timed_step = step2 if two_streams else step
    if two_streams:
        for _ in range(max(3, args.warmup)):
            step2()
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
    launches_per_step = (int(st_sc[9]) if st_sc else 0) + (int(st_nt[9]) if st_nt else 0)

    # ---- timed region
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        timed_step()
    t1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1)
    elapsed = max_over_ranks(elapsed, world, dev)
    ms_per_step = elapsed / args.steps
    value = elapsed / (args.steps * world)
    launches = launches_per_step * args.steps
    step_how = ("the SumCheck and NTT proofs on two streams (two contexts), forked and joined every step"
                if two_streams else "the step's proofs one after the other on one stream")
    one_stream_ms = None
    if two_streams:
        # the same steps one after the other on one stream, for comparison
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        for _ in range(args.steps):
            step()
        u1.record(stream)
        stream.synchronize()
        one_stream_ms = u0.elapsed_time(u1) / args.steps
        if p_sc2.cpu().numpy().tobytes() != p_sc.cpu().numpy().tobytes():
            raise RuntimeError("the two contexts' SumCheck proofs differ")
        ctx_sc.close()

    # ---- end to end through the C ABI with pinned host buffers
    hcols = [torch.from_numpy(c).pin_memory() for c in cols]
    hq = torch.empty(M * 32, dtype=torch.uint8).pin_memory()
    e2e_ms, e2e_seq_ms = [], []
    for it in range(7):   # host-timed: the median of seven; one call after the other
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        ctx.prove_sumcheck(GATE, N_LOG, DEG, hcols, roots=roots, stream=stream)
        if have_ntt:
            ctx.prove_ntt(GATE, N_LOG, DEG, hcols, roots=roots, stream=stream, q_out=hq)
        stream.synchronize()
        e2e_seq_ms.append((time.perf_counter() - t_a) * 1e3)
    e2e_ms = e2e_seq_ms
    if have_ntt and run_sc:
        # The two calls of a step issued from two host threads on two contexts
        # (each context is serialised by its own lock; ctypes releases the
        # interpreter lock), so one proof's host copies overlap the other's
        # kernels.  Same calls, buffers and copies as above.
        import concurrent.futures as cf
        ctx2 = zc.Context(local, max_n=24, max_d=8)
        stream2 = torch.cuda.Stream()
        ctx2.prove_sumcheck(GATE, N_LOG, DEG, hcols, roots=roots, stream=stream2)  # warm the context
        e2e_ms = []
        with cf.ThreadPoolExecutor(2) as ex:
            for it in range(7):
                torch.cuda.synchronize()
                t_a = time.perf_counter()
                f_nt = ex.submit(ctx.prove_ntt, GATE, N_LOG, DEG, hcols, roots=roots, stream=stream, q_out=hq)
                f_sc = ex.submit(ctx2.prove_sumcheck, GATE, N_LOG, DEG, hcols, roots=roots, stream=stream2)
                f_nt.result()
                f_sc.result()
                e2e_ms.append((time.perf_counter() - t_a) * 1e3)
        ctx2.close()
    h2d = 2 * C * N * 32 if have_ntt else C * N * 32
    d2h = ps_sc + ((ps_nt + M * 32) if have_ntt else 0)

    # ---- dominant kernel roofline (the longest single launch of the step)
    dom = st_nt if (st_nt and (st_sc is None or st_nt[6] > st_sc[6])) else st_sc
    dom_name = ("ntt slice-LDE pass" if dom is st_nt else "sumcheck round-1 evaluate kernel")
    dom_ms = dom[6]
    achieved = dom[7] / (dom_ms * 1e-3) if dom_ms > 0 else 0.0
    traffic = recorded_traffic() if (dom is st_nt and N_LOG == 22 and GATE == 1) else None
    roof = {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": ALU_PEAK_MULMOD,
            "unit": "mulmod/s", "frac": achieved / ALU_PEAK_MULMOD, "traffic": traffic,
            "traffic_source": "profiles/ntt_pass_plonk_n22_traffic.md" if traffic else None,
            "algorithmic_mulmods_per_launch": dom[7], "algorithmic_bytes_per_launch": dom[8],
            "hbm_gbs_at_algorithmic_bytes": dom[8] / (dom_ms * 1e-3) / 1e9 if dom_ms > 0 else None,
            "peak_note": peak_note()}
    by_form = {"sumcheck": {"ms": float(np.median(sc_ms)) if run_sc else None,
                            "roofline_ms": 1e3 * max(algorithmic_mulmods("sumcheck", N_LOG, DEG, GATE) / ALU_PEAK_MULMOD,
                                                      algorithmic_bytes("sumcheck", N_LOG, DEG, GATE) / HBM_PEAK),
                            "phases_ms": [round(x, 4) for x in st_sc[:5]] if st_sc else None}}
    if run_sc:
        by_form["sumcheck"]["roofline_frac"] = by_form["sumcheck"]["roofline_ms"] / by_form["sumcheck"]["ms"]
    if have_ntt:
        by_form["ntt"] = {"ms": float(np.median(nt_ms)),
                          "roofline_ms": 1e3 * max(algorithmic_mulmods("ntt", N_LOG, DEG, GATE) / ALU_PEAK_MULMOD,
                                                    algorithmic_bytes("ntt", N_LOG, DEG, GATE) / HBM_PEAK),
                          "phases_ms": [round(x, 4) for x in st_nt[:6]]}
        by_form["ntt"]["roofline_frac"] = by_form["ntt"]["roofline_ms"] / by_form["ntt"]["ms"]
    else:
        by_form["ntt"] = {"status": "not run (--form sumcheck)" if args.form == "sumcheck" else "not built"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32x8 (255-bit field, exact)",
                "data": "synthetic", "config": workload_config(world),
                "e2e": {"value": float(np.median(e2e_ms)), "unit": "ms", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h,
                        "how": ("the step's two C-ABI calls from pinned host buffers, issued from two host "
                                "threads on two contexts" if e2e_ms is not e2e_seq_ms else
                                "the step's C-ABI calls from pinned host buffers, one after the other"),
                        "one_after_the_other_ms": float(np.median(e2e_seq_ms))},
                "gpu_launches": launches, "roofline": roof, "clocks": clk, "by_form": by_form,
                "step": {"how": step_how, "one_stream_ms_per_step": one_stream_ms},
                "device": device_info}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_sample()
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
