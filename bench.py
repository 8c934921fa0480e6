"""Benchmark: Newton cell-iterations per second of the fully implicit black-oil
step (CPR-FGMRES(30), tolerance 1e-8) on the 100x100x20 synthetic reservoir.

A step is one 10-day time step: the Newton loop (assembly, CPR-FGMRES solve,
update) until the CNV test passes.  value = cells x Newton iterations / s over
the K timed steps, device time from CUDA events on the library's stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp64|mixed] [--workload bo100|bo200|bo400]

Prints one JSON line.  Under torchrun every rank runs its own replica of the
workload (the single-grid path does not shard), the time is the max over
ranks and the value sums the ranks' work ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton cell-iters/s"
UNIT = "cell-iters/s"


def workload(name: str, **solver):
    from paper_1606_00548_gb300 import synth
    if name == "bo100":
        return synth.black_oil_100x100x20(**solver), "black-oil 100x100x20 (200k cells, 3x3 blocks), 10-day steps"
    if name == "bo100c":
        return synth.black_oil_400cube(n=100, **solver), "black-oil 100^3 (1M cells), 1-day steps"
    if name == "bo200":
        return synth.black_oil_400cube(n=200, **solver), "black-oil 200^3 (8M cells), 1-day steps"
    if name == "bo400":
        return synth.black_oil_400cube(n=400, **solver), "black-oil 400^3 (64M cells), 1-day steps"
    raise SystemExit(f"unknown workload {name}")


def solver_overrides(args):
    """Solver options on top of the workload's defaults (FGMRES, theta 1e-8)."""
    o = {}
    if getattr(args, "solver", "default") == "paper":
        # the paper's experiments (Sec. 4): BiCGSTAB (at most 100 iterations),
        # adaptive forcing term (Eq. 14, choice 2), CNV tolerance 1e-3
        o.update(krylov=1, lin_max_iter=100, forcing=2, newton_tol=1e-3)
    if args.amg_cycles is not None:
        o["amg_cycles"] = args.amg_cycles
    if getattr(args, "decouple", "qi") == "abf":
        o["decouple"] = 1
    if getattr(args, "cpr_stages", 2) == 3:
        o["cpr_stages"] = 3
    if getattr(args, "orth", "cgs2") == "selective":
        o["orth"] = 1
    return o


def solver_desc(sv: dict) -> str:
    dec = "ABF" if sv.get("decouple", 0) == 1 else "QI"
    stages = "FPF" if sv.get("cpr_stages", 2) == 3 else "two-stage"
    kry = "BiCGSTAB" if sv.get("krylov", 0) == 1 else \
        f"FGMRES({sv.get('gmres_m', 30)}, {'selective CGS' if sv.get('orth', 0) else 'CGS2'})"
    forcing = "theta 1e-8" if sv.get("forcing", 0) == 0 else f"forcing choice {sv['forcing']} of Eq. 14"
    return (f"CPR {stages} ({dec}, aggregation AMG {sv.get('amg_cycles', 1)}x V(1,1), red-black block ILU0) "
            f"{kry}, {forcing}, CNV {sv.get('newton_tol', 1e-10):g}")


def kernel_sha1(name: str) -> str:
    """SHA-1 of a kernel's source text in csrc/krylov.cu (template line to the
    closing brace), so recorded ncu counters are dropped once the kernel changes."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_1606_00548_gb300", "csrc", "krylov.cu")).read()
    i = src.index(f" {name}(")
    i = src.rindex("template", 0, i)
    j = src.index("\n}\n", i)
    return hashlib.sha1(src[i:j].encode()).hexdigest()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": len(self.rows)}
        if not self.rows:
            return out
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 3 + k and r[3 + k].lower().startswith("active"):
                    reasons.add(nm)
        out.update(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons))
        return out


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _all_reduce(v, op):
    import torch
    import torch.distributed as dist
    # NCCL reduces device tensors; the gloo group of the CPU tests reduces host ones
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch.distributed as dist
    return _all_reduce(v, dist.ReduceOp.MAX)


def sum_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch.distributed as dist
    return _all_reduce(v, dist.ReduceOp.SUM)


def job_throughput(ws, work, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time.  Returns (value, max seconds)."""
    t_max = max_over_ranks(ws, seconds)
    return sum_over_ranks(ws, float(work)) / t_max, t_max


def shard(items, ws, rank):
    """The share of independent units (ensemble members) of one rank: every
    ws-th item from `rank` on, so the ranks' shares partition the list."""
    return items[rank::ws]


def cpu_oracle_sample(case, newton_its=1):
    """The oracle as it stands, one thread: a bounded number of Newton iterations
    of the first time step of the workload.  Returns (cell-iters/s, seconds)."""
    import oracle
    o = oracle.Oracle(case)
    dt = case["dt"][0]
    N = case["nx"] * case["ny"] * case["nz"]
    t0 = time.perf_counter()
    its = 0
    for _ in range(newton_its):
        rc, info = o.newton_step(dt)
        its += info.newton_iterations
        if info.converged:
            break
    t = time.perf_counter() - t0
    return N * max(its, 1) / t, t


def run_reference(args):
    ws, rank = dist_info()
    if rank != 0:
        return 0
    case, desc = workload(args.workload, **solver_overrides(args))
    N = case["nx"] * case["ny"] * case["nz"]
    import oracle
    oracle.build()
    o = oracle.Oracle(case)
    dt = case["dt"][0]
    # warm-up and timed steps: one oracle Newton iteration each (a bounded sample)
    for _ in range(args.warmup):
        o.newton_step(dt)
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        rc, info = o.newton_step(dt)
        its += max(1, info.newton_iterations)
    t = time.perf_counter() - t0
    value = N * its / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "sample": "one oracle Newton iteration per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} Newton iterations of the first time step, 1 thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank = dist_info()
    if ws > 1:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    from paper_1606_00548_gb300 import build
    build.build()
    from paper_1606_00548_gb300.sim import Simulator

    case, desc = workload(args.workload, **solver_overrides(args))
    N = case["nx"] * case["ny"] * case["nz"]
    prec = 1 if args.precision == "mixed" else 0
    stream = torch.cuda.Stream()
    sim = Simulator(case, precision=prec, stream=stream.cuda_stream)
    dts = case["dt"]

    def dt_of(k):
        return dts[k % len(dts)]

    k = 0
    for _ in range(args.warmup):
        sim.step(dt_of(k)); k += 1
    torch.cuda.synchronize()
    st0 = sim.stats()
    sampler = ClockSampler(dev) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    newton = 0
    lin = 0
    cuts = 0
    for _ in range(args.steps):
        st, info = sim.step(dt_of(k)); k += 1
        newton += info.newton_iterations
        lin += info.linear_iterations
        cuts += info.cuts
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop() if sampler else None
    t_dev = e0.elapsed_time(e1) / 1e3
    st1 = sim.stats()
    value, t_max = job_throughput(ws, N * newton, t_dev)

    # end to end through the C ABI with host buffers: H2D state, step, D2H state
    p, sw, x3, ph = sim.get_state()
    p = np.ascontiguousarray(p); sw = np.ascontiguousarray(sw); x3 = np.ascontiguousarray(x3)
    e2e_newton = 0
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.set_state(p, sw, x3, ph)
        st, info = sim.step(dt_of(k)); k += 1
        e2e_newton += info.newton_iterations
        p, sw, x3, ph = sim.get_state()
    torch.cuda.synchronize()
    e2e_value, t_e2e = job_throughput(ws, N * e2e_newton, time.perf_counter() - t0)
    state_bytes = N * (3 * 8 + 1)

    # roofline of the block SpMV: y = J x, 7 b^2 + 2 b doubles per cell; device
    # time of back-to-back launches on the library's stream (CUDA events)
    b = sim.b
    sim.time_op(0, 3)
    t_spmv = sim.time_op(0, 50) / 1e6
    # breakdown at the current Newton system: preconditioner apply and one full solve
    sim.assemble(dt_of(k))
    sim.precond_setup()
    sim.time_op(1, 3)
    t_prec = sim.time_op(1, 20) / 1e6
    x = torch.randn(N * b, dtype=torch.float64, device="cuda")
    z = torch.empty_like(x)
    s0 = torch.cuda.Event(enable_timing=True); s1 = torch.cuda.Event(enable_timing=True)
    rhs = torch.randn(N * b, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()            # rhs is written on torch's stream, read on the library's
    with torch.cuda.stream(stream):
        s0.record(stream)
        _, li = sim.linear_solve(rhs, z)
        s1.record(stream)
    torch.cuda.synchronize()
    t_solve = s0.elapsed_time(s1) / 1e3
    breakdown = {"spmv_us": t_spmv * 1e6, "precond_apply_us": t_prec * 1e6,
                 "solve_ms": t_solve * 1e3, "solve_iterations": li.iterations,
                 "us_per_iteration": t_solve * 1e6 / max(1, li.iterations)}
    bytes_spmv = (7 * b * b + 2 * b) * 8 * N
    flops_spmv = 2 * 7 * b * b * N
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_peak = float(peaks["hbm_gbs"]); hbm_src = "measured"
    except Exception:
        hbm_peak = 6800.0; hbm_src = "fallback"
    from paper_1606_00548_gb300.sim import sim_probe_fma_rates
    fp64_fma, fp32_fma = sim_probe_fma_rates()
    fp64_nominal_tflops = 1.25      # GB300 FP64 (nominal, profiling recipe table; 2 FMA/clk/SM at 2.07 GHz)
    achieved_tflops = flops_spmv / t_spmv / 1e12
    traffic = None
    try:
        ctr = json.load(open(os.path.join(ROOT, "profiles", "roofline_counters.json")))[f"spmv_kernel<{b}, double>"]
        # counters count only for the kernel source they were taken on
        if ctr["workload_cells"] == N and ctr.get("kernel_sha1") == kernel_sha1("spmv_kernel"):
            traffic = ctr["dram_bytes_per_launch"]
    except Exception:
        traffic = None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        v, t = cpu_oracle_sample(case, 1)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one Newton iteration of the first {dts[0]:g}-day step ({t:.1f} s, 1 thread)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f64+f32",
            "data": "synthetic",
            "config": {"workload": desc, "precision": args.precision,
                       "solver": solver_desc(case["solver"]),
                       "newton_iterations": newton, "linear_iterations": lin, "cuts": cuts,
                       "l2": "working set (J 101 MB + Krylov basis 149 MB + ...) larger than L2"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes},
            "gpu_launches": int(st1.kernel_launches - st0.kernel_launches),
            "roofline": {"kernel": "spmv_kernel (block stencil SpMV y = J x, FP64)", "bound": "alu",
                         "achieved": achieved_tflops, "peak": fp64_nominal_tflops, "unit": "TFLOP/s",
                         "frac": achieved_tflops / fp64_nominal_tflops, "traffic": traffic,
                         "peak_source": "nominal FP64 rate of the profiling recipe",
                         "fp64_probe_tflops": 2 * fp64_fma / 1e12, "frac_of_probe": achieved_tflops / (2 * fp64_fma / 1e12),
                         "flops_per_cell": 2 * 7 * b * b, "bytes_per_cell": (7 * b * b + 2 * b) * 8,
                         "hbm_achieved_gbs": bytes_spmv / t_spmv / 1e9, "hbm_peak_gbs": hbm_peak,
                         "hbm_frac": bytes_spmv / t_spmv / 1e9 / hbm_peak, "hbm_peak_source": hbm_src,
                         "launch_us": t_spmv * 1e6},
            "clocks": clocks,
            "breakdown": breakdown,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_ensemble(args):
    """Batched ensemble: 64 oil-water realisations on uneven grids (nx, ny in
    32..128, nz in 8..32, sigma 0.5..2), 1-day steps, advanced together on one
    GPU (concurrent members, per-member CUDA graphs, autotuned launch shapes)
    versus one member at a time.  Under torchrun the members are partitioned
    across ranks (no collective on the data path)."""
    import torch
    ws, rank = dist_info()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    from paper_1606_00548_gb300 import build, synth
    build.build()
    from paper_1606_00548_gb300.sim import Batch, Simulator
    prec = 1 if args.precision == "mixed" else 0
    members = shard(synth.ensemble_members(64, nsteps=20, dt=1.0), ws, rank)
    sims = [Simulator(c, precision=prec) for c in members]
    cells = [c["nx"] * c["ny"] * c["nz"] for c in members]
    for sm in sims:
        sm.autotune(1.0)
    batch = Batch(sims)
    for _ in range(args.warmup):
        batch.step(1.0)
    barrier(ws); torch.cuda.synchronize()
    t0 = time.perf_counter()
    work = 0
    for _ in range(args.steps):
        sts, infos = batch.step(1.0)
        work += sum(n * inf.newton_iterations for n, inf in zip(cells, infos))
    torch.cuda.synchronize()
    value, t_batch = job_throughput(ws, work, time.perf_counter() - t0)
    # one member at a time (same handles, next steps)
    t0 = time.perf_counter()
    work_seq = 0
    for _ in range(args.steps):
        for n, sm in zip(cells, sims):
            st, inf = sm.step(1.0)
            work_seq += n * inf.newton_iterations
    torch.cuda.synchronize()
    value_seq, t_seq = job_throughput(ws, work_seq, time.perf_counter() - t0)
    if rank == 0:
        st0 = sims[0].stats()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_batch / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64" if prec == 0 else "f64+f32", "data": "synthetic",
            "config": {"workload": "ensemble of 64 oil-water realisations (8.6M cells in total), 1-day steps",
                       "members_on_rank0": len(members), "cells_on_rank0": sum(cells),
                       "timing": "host wall clock around fully synchronised batch steps",
                       "autotuned_blocks_member0": [st0.spmv_block, st0.amg_block]},
            "one_at_a_time": {"value": value_seq, "ms_per_step": 1e3 * t_seq / args.steps},
            "batched_over_sequential": value / value_seq,
        }
        print(json.dumps(line), flush=True)
    batch.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_learned(args):
    """Second metric: CPR-FGMRES time to 1e-8 relative residual on the 256x256x64
    black-oil system (sigma 2): FP64 CPR and FP32-preconditioned CPR (two-stage
    and CPR-FPF), and FP32 CPR + learned stage (network trained on the device on
    128x128x32 systems).  value = the learned form's time."""
    import torch
    from paper_1606_00548_gb300 import build, learned
    build.build()
    ev = learned.evaluate(train_steps=args.train_steps)
    r = ev["results"]
    best = min(r, key=lambda k: r[k]["seconds"])
    line = {
        "metric": "CPR-FGMRES time to 1e-8 rel. residual", "value": r["mixed_cpr_learned"]["seconds"], "unit": "s",
        "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32+bf16", "data": "synthetic",
        "config": {"workload": "black-oil 256x256x64 (4.2M cells), sigma 2, first Newton system; "
                               "network trained on 128x128x32 (sigma 1) pairs",
                   "train_seconds": ev["train_seconds"], "pairs_seconds": ev["pairs_seconds"],
                   "train_loss": ev["train_loss"][-3:]},
        "results": r, "fastest": best,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default="bo100", choices=["bo100", "bo100c", "bo200", "bo400", "learned", "ensemble"])
    ap.add_argument("--train-steps", type=int, default=300)
    ap.add_argument("--amg-cycles", type=int, default=None, help="V-cycles per CPR pressure stage")
    ap.add_argument("--solver", default="default", choices=["default", "paper"],
                    help="paper: BiCGSTAB, adaptive forcing (Eq. 14 choice 2), CNV 1e-3")
    ap.add_argument("--decouple", default="qi", choices=["qi", "abf"])
    ap.add_argument("--cpr-stages", type=int, default=2, choices=[2, 3])
    ap.add_argument("--orth", default="cgs2", choices=["cgs2", "selective"],
                    help="FGMRES Gram-Schmidt: two passes always, or the second only when needed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
