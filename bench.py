"""Benchmark: Newton cell-iterations per second of the fully implicit black-oil
Newton step (CPR-FGMRES(30), tolerance 1e-8) on the 400x400x400 synthetic
reservoir (64M cells, 3x3 blocks, 25 wells, 1-day steps).

A step is one Newton iteration of Algorithm 1 with its linear solve: assembly
and CNV test, CPR setup, CPR-FGMRES solve, update (a converged time step is
accepted and the next one started inside the step that follows it, so its
convergence test counts too).  value = cells x Newton iterations / device
time of the K timed steps (CUDA events on the library's stream, bracketing the
device work of each step); e2e = the same iterations over wall-clock time with
the iterate copied from pinned host memory before each step and back after it
through the C ABI (sim_set_iterate / sim_get_iterate).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp64|mixed] [--workload bo400|bo200|bo100c|bo100]

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


def kernel_sha1(*names: str) -> str:
    """SHA-1 of kernel sources in csrc/krylov.cu (each from its template line to
    the closing brace), so recorded ncu counters are dropped once they change."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_1606_00548_gb300", "csrc", "krylov.cu")).read()
    h = hashlib.sha1()
    for name in names:
        i = src.index(f" {name}(")
        i = src.rindex("template", 0, i) if name != "scale_body" else src.rindex("\n", 0, i) + 1
        j = src.index("\n}\n", i)
        h.update(src[i:j].encode())
    return h.hexdigest()


# the Gram-Schmidt kernels' bodies (one Arnoldi step: dots, second pass, update and norm, scale)
GS_SOURCES = ("dots_body", "orth_dots_body", "orth_norm_body", "scale_body")

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


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
def corner_cut(case, n):
    """The n x n x n corner (x, y, z from 0) of a case: its rock, initial state
    and the wells whose column lies inside, perforations clipped to the cut."""
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    cx, cy, cz = min(n, nx), min(n, ny), min(n, nz)

    def sub(a):
        return np.ascontiguousarray(np.asarray(a).reshape(nz, ny, nx)[:cz, :cy, :cx].reshape(-1))

    out = dict(case)
    out.update(nx=cx, ny=cy, nz=cz, name=f"{case['name']} corner {cx}x{cy}x{cz}")
    for k in ("kx", "ky", "kz", "poro"):
        out[k] = sub(case[k])
    out["init"] = {k: sub(v) for k, v in case["init"].items()}
    wells = []
    for w in case["wells"]:
        if w["i"] < cx and w["j"] < cy and w["k0"] < cz:
            w2 = dict(w); w2["k1"] = min(w["k1"], cz - 1); wells.append(w2)
    out["wells"] = wells
    return out


def oracle_iterations(case, warmup, count):
    """Time `count` oracle Newton iterations that perform a linear solve (after
    `warmup` untimed ones), advancing through the case's time steps: when the
    CNV test passes, the step is accepted (the iterate becomes the state) and
    the next starts.  Returns the seconds of the timed iterations."""
    import oracle
    oracle.build()
    o = oracle.Oracle(case)
    dts = case["dt"]
    k = 0
    times = []
    done = 0
    while done < warmup + count:
        t0 = time.perf_counter()
        rc, info = o.newton_step(dts[k % len(dts)])
        if rc != 0:
            raise RuntimeError("oracle Newton iteration failed")
        if info.converged:
            o.set_state(*o.get_state())          # accept: the next step starts from here
            k += 1
            rc, info = o.newton_step(dts[k % len(dts)])
            if rc != 0 or info.converged:
                raise RuntimeError("oracle: no Newton iteration after accepting a step")
        t = time.perf_counter() - t0
        if done >= warmup:
            times.append(t)
        done += 1
    return times


def _oracle_worker(args):
    case, warmup, count = args
    return oracle_iterations(case, warmup, count)


def oracle_on_cores(case, warmup, count, procs):
    """`procs` concurrent single-threaded oracle replicas (spawned processes);
    returns (aggregate cell-iters/s, per-replica seconds lists)."""
    import multiprocessing as mp
    N = case["nx"] * case["ny"] * case["nz"]
    if procs <= 1:
        ts = [oracle_iterations(case, warmup, count)]
    else:
        with mp.get_context("spawn").Pool(procs) as pool:
            ts = pool.map(_oracle_worker, [(case, warmup, count)] * procs)
    t_max = max(sum(t) for t in ts)
    return procs * N * count / t_max, ts


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample_case(args, case=None, desc=None):
    """The bounded sample of the workload the oracle runs: the n^3 corner of
    the same field (--oracle-cut, 48: 110k cells, a few seconds per Newton
    iteration; the full 64M-cell grid would take the oracle about 20 minutes
    per Newton iteration)."""
    if case is None:
        case, desc = workload(args.workload, **solver_overrides(args))
    N = case["nx"] * case["ny"] * case["nz"]
    if N <= 300_000:
        return case, desc, "the whole grid"
    cut = corner_cut(case, args.oracle_cut)
    return cut, desc, (f"the {cut['nx']}x{cut['ny']}x{cut['nz']} corner of the same field "
                       f"({cut['nx'] * cut['ny'] * cut['nz']} cells, {len(cut['wells'])} well(s) inside it)")


def run_reference(args):
    ws, rank = dist_info()
    if rank != 0:
        return 0
    case, desc, where = oracle_sample_case(args)
    cores = host_cores()
    value, ts = oracle_on_cores(case, args.warmup, args.steps, cores)
    t_max = max(sum(t) for t in ts)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc,
                   "sample": f"each step: one oracle Newton iteration with its linear solve on {where}; "
                             f"{cores} concurrent single-threaded replicas, one per host core"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} Newton iterations (after {args.warmup}) on {where}, "
                                   f"{cores} replicas"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------
class NewtonDriver:
    """Algorithm 1 driven one Newton iteration at a time through the C ABI:
    sim_newton_step; when it reports the CNV test met, sim_accept_step and the
    next time step's first iteration.  A time step taking more than newton_max
    iterations is an error here (the benchmark does not cut steps)."""

    def __init__(self, sim, dts):
        self.sim, self.dts, self.k, self.its_in_step = sim, dts, 0, 0

    def dt(self):
        return self.dts[self.k % len(self.dts)]

    def iteration(self):
        st, info = self.sim.newton_step(self.dt())
        phase = info.phase.as_dict()
        if info.converged:
            self.sim.accept_step(self.dt())
            self.k += 1
            self.its_in_step = 0
            st, info = self.sim.newton_step(self.dt())
            for key, v in info.phase.as_dict().items():
                phase[key] += v
        if st != 0 or info.converged:
            raise RuntimeError(f"Newton iteration failed (status {st})")
        self.its_in_step += 1
        if self.its_in_step > self.sim.opts.newton_max:
            raise RuntimeError("time step did not converge within newton_max iterations")
        return info, phase

    def finish_step(self):
        """Newton iterations until the current time step converges; accept it
        (the next call of iteration() starts the following step)."""
        while True:
            st, info = self.sim.newton_step(self.dt())
            if info.converged:
                self.sim.accept_step(self.dt())
                self.k += 1
                self.its_in_step = 0
                return
            self.its_in_step += 1
            if st != 0 or self.its_in_step > self.sim.opts.newton_max:
                raise RuntimeError(f"Newton iteration failed (status {st})")


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
    from paper_1606_00548_gb300.sim import Simulator, sim_probe_fma_rates, sim_probe_fp64_pipe

    case, desc = workload(args.workload, **solver_overrides(args))
    N = case["nx"] * case["ny"] * case["nz"]
    prec = 1 if args.precision == "mixed" else 0
    stream = torch.cuda.Stream()
    sim = Simulator(case, precision=prec, stream=stream.cuda_stream)
    b = sim.b
    drv = NewtonDriver(sim, case["dt"])
    for _ in range(args.warmup):
        drv.iteration()
    torch.cuda.synchronize()

    # pinned host copies of the iterate (the step's input and output on the host)
    x_h = torch.empty(N * b, dtype=torch.float64, pin_memory=True)
    ph_h = torch.empty(N, dtype=torch.int8, pin_memory=True)
    xp = x_h.numpy(); php = ph_h.numpy()
    sim.L.sim_get_iterate(sim.h, xp.ctypes.data_as(sim_dp()), php.ctypes.data_as(sim_i8p()))

    st0 = sim.stats()
    sampler = ClockSampler(dev) if rank == 0 else None
    if sampler:
        sampler.start()
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    lin = 0
    phases = {}
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        check(sim, sim.L.sim_set_iterate(sim.h, xp.ctypes.data_as(sim_dp()), php.ctypes.data_as(sim_i8p())))
        events[k][0].record(stream)
        info, ph = drv.iteration()
        events[k][1].record(stream)
        check(sim, sim.L.sim_get_iterate(sim.h, xp.ctypes.data_as(sim_dp()), php.ctypes.data_as(sim_i8p())))
        lin += info.linear_iterations
        for key, v in ph.items():
            phases[key] = phases.get(key, 0.0) + v
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t0
    barrier(ws)
    clocks = sampler.stop() if sampler else None
    st1 = sim.stats()
    report = sim.run_report()   # the timed handle's run so far (warm-up included), before the kernel studies
    t_dev = sum(e0.elapsed_time(e1) for e0, e1 in events) / 1e3
    newton = args.steps
    value, t_max = job_throughput(ws, N * newton, t_dev)
    e2e_value, _ = job_throughput(ws, N * newton, t_wall)
    iterate_bytes = N * (b * 8 + 1)

    # kernel-level device times (CUDA events on the library's stream, each
    # launch preceded by a 256 MB write that evicts its operands from L2)
    sim.time_op(0, 3)
    t_spmv = sim.time_op(0, 10) / 1e6
    sim.precond_setup()
    sim.time_op(1, 2)
    t_prec = sim.time_op(1, 5) / 1e6
    nv = min(16, sim.opts.gmres_m)
    sim.time_op(2, 2)
    t_orth = sim.time_op(2, 5) / 1e6
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_peak = float(peaks["hbm_gbs"]); hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        hbm_peak = 6800.0; hbm_src = "fallback of the profiling recipe"
    fp64_fma, fp32_fma = sim_probe_fma_rates()
    fp64_tflops = 2 * fp64_fma / 1e12
    # FP64 peak of this run: the pipe's unit count (2 FMA per clock per SM) x the SMs x the
    # median SM clock sampled during the timed region.  The FMA-loop probe, timed against
    # its own clock (clock64 against %globaltimer), runs at full clock but below that
    # per-clock rate, under what the SpMV reaches: it does not measure the pipe's peak.
    _, probe_mhz, fma_per_clk = sim_probe_fp64_pipe()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    run_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    fp64_peak = 2 * 2 * sms * run_mhz * 1e6 / 1e12
    fp64_peak_src = (f"FP64 pipe unit count: 2 FMA/clk/SM x {sms} SMs x {run_mhz:.0f} MHz (median SM clock of the "
                     f"timed region); the FMA-loop probe reaches {fma_per_clk:.3f} FMA/clk/SM at its own "
                     f"{probe_mhz:.0f} MHz ({fp64_tflops:.3f} TFLOP/s): full clock, below the pipe's rate; "
                     "the FP64 SpMV of this run reaches ")
    n = N * b
    bytes_spmv = (7 * b * b + 2 * b) * 8 * N
    flops_spmv = 2 * 7 * b * b * N
    bytes_orth = (3 * nv + 7) * n * 8
    kernels = {
        "spmv_kernel": {"what": "block stencil SpMV y = J x, FP64", "launch_us": t_spmv * 1e6,
                        "bytes": bytes_spmv, "hbm_gbs": bytes_spmv / t_spmv / 1e9,
                        "hbm_frac": bytes_spmv / t_spmv / 1e9 / hbm_peak,
                        "fp64_tflops": flops_spmv / t_spmv / 1e12,
                        "fp64_frac": flops_spmv / t_spmv / 1e12 / fp64_tflops},
        "gram_schmidt_step": {"what": f"dots_kernel<{nv}> + orth_dots_kernel<{nv}> + orth_norm_kernel<{nv}> + "
                                      "scale_kernel: one CGS2 Arnoldi step against 16 basis vectors",
                              "launch_us": t_orth * 1e6, "bytes": bytes_orth,
                              "hbm_gbs": bytes_orth / t_orth / 1e9, "hbm_frac": bytes_orth / t_orth / 1e9 / hbm_peak},
        "cpr_apply": {"what": "one CPR application (restriction, V-cycle, stage F)", "launch_us": t_prec * 1e6},
    }
    # one CGS2 Arnoldi step at NV basis vectors: dots NV + 1 FMAs per element,
    # second pass (update and dots) 2 NV, update and norm NV + 1, scale 1
    flops_orth = 2 * (4 * nv + 3) * n
    kernels["gram_schmidt_step"].update(fp64_tflops=flops_orth / t_orth / 1e12,
                                        fp64_frac=flops_orth / t_orth / 1e12 / fp64_peak)
    kernels["spmv_kernel"]["fp64_frac"] = flops_spmv / t_spmv / 1e12 / fp64_peak
    dom = kernels["gram_schmidt_step"]
    traffic = None
    try:
        ctr = json.load(open(os.path.join(ROOT, "profiles", "roofline_counters.json")))[f"gram_schmidt_step<{b}>"]
        # counters count only for the kernel sources they were taken on
        if ctr.get("kernel_sha1") == kernel_sha1(*GS_SOURCES) and ctr.get("nv") == nv:
            traffic = ctr["dram_bytes_per_element"] * n
    except Exception:
        traffic = None

    # time to the 1e-8 relative residual per Newton system (CPR set-up and
    # CPR-FGMRES solve, the phases of the timed iterations)
    def per_system(ph, its):
        return {"setup_s": ph.get("setup_us", 0.0) / 1e6 / its, "solve_s": ph.get("solve_us", 0.0) / 1e6 / its,
                "to_tolerance_s": (ph.get("setup_us", 0.0) + ph.get("solve_us", 0.0)) / 1e6 / its}
    forms = None
    if prec == 0 and args.mixed_steps > 0:
        # FP64 and FP32-preconditioner forms from the same accepted state: the
        # current time step is finished, its state saved, and each form runs
        # mixed_steps Newton iterations from there (the same Newton systems up to
        # the 1e-8 solves' differences); the FP32 form gets a second handle after
        # the first is freed (both do not fit in HBM)
        def timed_form(simx, drx, K):
            evx = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            lin_x, ph_x = 0, {}
            torch.cuda.synchronize()
            for q in range(K):
                evx[q][0].record(stream)
                info, ph = drx.iteration()
                evx[q][1].record(stream)
                lin_x += info.linear_iterations
                for key, v in ph.items():
                    ph_x[key] = ph_x.get(key, 0.0) + v
            torch.cuda.synchronize()
            t_x = sum(a_.elapsed_time(b_) for a_, b_ in evx) / 1e3
            return dict(value=N * K / t_x, linear_iterations_per_newton=lin_x / K, newton_iterations=K,
                        **per_system(ph_x, K))
        drv.finish_step()
        saved = sim.get_state()
        step_index = drv.k
        forms = {"start": f"time step {step_index + 1} from its accepted state", "fp64": timed_form(sim, drv, args.mixed_steps)}
        sim.close()
        torch.cuda.synchronize()
        simm = Simulator(case, precision=1, stream=stream.cuda_stream)
        simm.set_state(*saved)
        drm = NewtonDriver(simm, case["dt"])
        drm.k = step_index
        forms["mixed"] = timed_form(simm, drm, args.mixed_steps)
        forms["mixed_over_fp64_time_to_tolerance"] = forms["mixed"]["to_tolerance_s"] / forms["fp64"]["to_tolerance_s"]
        simm.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        ocase, _, where = oracle_sample_case(args, case, desc)
        v1, t1 = oracle_on_cores(ocase, 0, 1, 1)
        cores = host_cores()
        vall, tall = oracle_on_cores(ocase, 0, 1, cores)
        cpu = {"value": vall, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one Newton iteration with its linear solve on {where}, {cores} concurrent "
                         f"single-threaded replicas ({max(sum(t) for t in tall):.1f} s)",
               "single_thread": {"value": v1, "seconds": sum(t1[0])}}

    if rank == 0:
        J_bytes = 7 * b * b * 8 * N
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f64+f32",
            "data": "synthetic",
            "config": {"workload": desc, "cells": N, "precision": args.precision,
                       "solver": solver_desc(case["solver"]),
                       "step": "one Newton iteration (assembly, CNV test, CPR setup, CPR-FGMRES solve, update)",
                       "newton_iterations": newton, "linear_iterations": lin, "time_steps_accepted": drv.k,
                       "l2": f"inputs larger than L2: the Jacobian alone is {J_bytes / 1e9:.1f} GB "
                             f"and the Krylov basis {(sim.opts.gmres_m + 1) * n * 8 / 1e9:.1f} GB (L2 129 MB)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": iterate_bytes,
                    "d2h_bytes_per_step": iterate_bytes},
            "gpu_launches": int(st1.kernel_launches - st0.kernel_launches),
            "roofline": {"kernel": dom["what"], "bound": "alu", "achieved": dom["fp64_tflops"],
                         "peak": fp64_peak, "unit": "TFLOP/s", "frac": dom["fp64_frac"],
                         "traffic": traffic,
                         "peak_source": fp64_peak_src + f"{kernels['spmv_kernel']['fp64_tflops']:.3f}",
                         "flops_per_launch": flops_orth, "launch_us": dom["launch_us"],
                         "hbm_achieved_gbs": dom["hbm_gbs"], "hbm_peak_gbs": hbm_peak, "hbm_frac": dom["hbm_frac"],
                         "hbm_peak_source": hbm_src, "bytes_per_launch": dom["bytes"],
                         "share_of_kernel_time": "37% (profiles/launch_list_black_oil_400cube.md)"},
            "kernels": kernels,
            "fp64_probe_tflops": fp64_tflops,
            "fp64_pipe": {"fma_per_clk_per_sm": fma_per_clk, "probe_sm_mhz": probe_mhz, "run_sm_mhz": run_mhz,
                          "peak_tflops": fp64_peak},
            "phases_per_newton": {k: v / newton for k, v in phases.items()},
            "forms": forms,
            "run_report": {"counters": report["counters"], "phases": report["phases"],
                           "note": "sim_run_report of the timed handle: warm-up and timed Newton iterations"},
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def sim_dp():
    import ctypes
    return ctypes.POINTER(ctypes.c_double)


def sim_i8p():
    import ctypes
    return ctypes.POINTER(ctypes.c_int8)


def check(sim, st):
    from paper_1606_00548_gb300.sim import _check
    _check(sim.h, st)


def run_ensemble(args):
    """Batched ensemble: 64 oil-water realisations on uneven grids (nx, ny in
    32..128, nz in 8..32, sigma 0.5..2), 1-day steps, advanced together on one
    GPU.  Three runtimes on the same members, each timed over its own K steps
    (after W warm-up steps, members advancing in time throughout): lockstep
    (one batched FGMRES per Newton round, every Krylov operation one launch
    over all members; the value), concurrent (each member's sim_step on its
    own stream) and one member at a time.  Under torchrun the members are
    partitioned across ranks (no collective on the data path)."""
    import torch
    ws, rank = dist_info()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    from paper_1606_00548_gb300 import build, synth
    build.build()
    from paper_1606_00548_gb300.sim import SIM_BATCH_CONCURRENT, SIM_BATCH_LOCKSTEP, Batch, Simulator
    prec = 1 if args.precision == "mixed" else 0
    members = shard(synth.ensemble_members(64, nsteps=20, dt=1.0), ws, rank)
    sims = [Simulator(c, precision=prec) for c in members]
    cells = [c["nx"] * c["ny"] * c["nz"] for c in members]
    batch = Batch(sims)
    assert batch.mode() == SIM_BATCH_LOCKSTEP

    def timed(mode):
        """K batch steps in the given mode: (cell-iters/s over ranks, seconds, work)"""
        batch.L.sim_batch_set_mode(batch.h, mode)
        barrier(ws); torch.cuda.synchronize()
        t0 = time.perf_counter()
        work = 0
        for _ in range(args.steps):
            sts, infos = batch.step(1.0)
            if any(st != 0 for st in sts):
                raise RuntimeError(f"ensemble step failed: {sts} {batch.last_error()}")
            work += sum(n * inf.newton_iterations for n, inf in zip(cells, infos))
        torch.cuda.synchronize()
        v, t = job_throughput(ws, work, time.perf_counter() - t0)
        return v, t, work

    for _ in range(args.warmup):
        batch.step(1.0)
    s0 = batch.stats()
    ph0 = batch.phase_seconds()
    launches0 = sum(sm.stats().kernel_launches for sm in sims)
    value, t_lock, _ = timed(SIM_BATCH_LOCKSTEP)
    s1 = batch.stats()
    ph1 = batch.phase_seconds()
    launches_lock = sum(sm.stats().kernel_launches for sm in sims) - launches0 + (s1["launches"] - s0["launches"])
    batch.L.sim_batch_set_mode(batch.h, SIM_BATCH_CONCURRENT)
    l1 = sum(sm.stats().kernel_launches for sm in sims)
    v_conc, t_conc, _ = timed(SIM_BATCH_CONCURRENT)
    launches_conc = sum(sm.stats().kernel_launches for sm in sims) - l1
    batch.L.sim_batch_set_mode(batch.h, SIM_BATCH_LOCKSTEP)
    # one member at a time (same handles, next steps)
    barrier(ws); torch.cuda.synchronize()
    t0 = time.perf_counter()
    work_seq = 0
    for _ in range(args.steps):
        for n, sm in zip(cells, sims):
            st, inf = sm.step(1.0)
            work_seq += n * inf.newton_iterations
    torch.cuda.synchronize()
    value_seq, t_seq = job_throughput(ws, work_seq, time.perf_counter() - t0)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_lock / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64" if prec == 0 else "f64+f32", "data": "synthetic",
            "config": {"workload": "ensemble of 64 oil-water realisations (8.6M cells in total), 1-day steps",
                       "members_on_rank0": len(members), "cells_on_rank0": sum(cells),
                       "runtime": "lockstep: one batched FGMRES per Newton round (one launch per Krylov "
                                  "operation over all members, restart cycle as one CUDA graph)",
                       "timing": "host wall clock around fully synchronised batch steps",
                       "lockstep_rounds": s1["rounds"] - s0["rounds"], "member_solves": s1["solves"] - s0["solves"],
                       "lockstep_host_seconds": {k: ph1[k] - ph0[k] for k in ph1}},
            "gpu_launches": int(launches_lock),
            "concurrent": {"value": v_conc, "ms_per_step": 1e3 * t_conc / args.steps, "gpu_launches": int(launches_conc)},
            "one_at_a_time": {"value": value_seq, "ms_per_step": 1e3 * t_seq / args.steps},
            "lockstep_over_concurrent": value / v_conc,
            "lockstep_over_one_at_a_time": value / value_seq,
        }
        print(json.dumps(line), flush=True)
    batch.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def conv_roofline(nx=256, ny=256, nz=64, reps=10):
    """The learned stage's kernels on the evaluation grid, each launch after an
    L2 eviction: forward convolution of a 16 -> 16 layer (tcgen05), its weight
    gradient (mma.sync, with the fold) and data gradient (tcgen05).  Algorithmic
    work per cell: 2 x 27 x 16 x 16 FLOP; bytes: the input and output
    activations, 32 B each (the weight gradient reads two 32-B activations and
    writes 27 x 16 x 16 FP32 partials per CTA, counted)."""
    import torch
    from paper_1606_00548_gb300.sim import Net
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    hbm, bf16 = float(peaks["hbm_gbs"]), float(peaks["bf16_tflops"])
    N = nx * ny * nz
    net = Net(nx, ny, nz, seed=0)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(N * 4, dtype=torch.float32, device="cuda", generator=g)
    t = torch.randn(N, dtype=torch.float32, device="cuda", generator=g)
    y = torch.empty(N, dtype=torch.float32, device="cuda")
    net.forward(x, y)
    net.loss_grad(x, t)
    flop = 2.0 * 27 * 16 * 16 * N
    out = {}
    for which, name, nbytes in ((0, "conv_tc_kernel forward 16->16", 64.0 * N),
                                (1, "wgrad_tc_kernel + fold", 64.0 * N),
                                (2, "conv_tc_kernel data gradient 16->16", 96.0 * N)):
        net.time_conv(which, 3)
        us = net.time_conv(which, reps)
        out[name] = {"us": us, "tflops": flop / us / 1e6, "tensor_frac_bf16": flop / us / 1e6 / bf16,
                     "hbm_gbs": nbytes / us / 1e3, "hbm_frac": nbytes / us / 1e3 / hbm}
    net.close()
    fwd = out["conv_tc_kernel forward 16->16"]
    roof = {"kernel": "conv_tc_kernel (forward, 16 -> 16 channels, 256x256x64)", "bound": "hbm",
            "achieved": fwd["hbm_gbs"], "peak": hbm, "unit": "GB/s", "frac": fwd["hbm_frac"], "traffic": None,
            "note": "arithmetic intensity 216 FLOP/B is below the measured BF16/HBM balance "
                    f"{bf16 * 1e3 / hbm:.0f} FLOP/B, so HBM bounds it; the tensor-core fraction is "
                    f"{fwd['tensor_frac_bf16']:.3f} of the measured {bf16:.0f} TFLOP/s BF16 "
                    "(profiles/conv_kernels_learned_256x256x64.md)"}
    return {"roofline": roof, "kernels": out}


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
    # the plain forms again with two V-cycles per pressure stage (the network is
    # trained on what one cycle leaves, so the learned form stays at one)
    from paper_1606_00548_gb300 import synth
    ecase = synth.black_oil_256x256x64_sigma2()
    r2 = {name: learned.time_solve(ecase, prec, repeats=3, amg_cycles=2, **extra)
          for name, prec, extra in (("fp64_cpr", 0, {}), ("fp64_cpr_fpf", 0, {"cpr_stages": 3}),
                                    ("mixed_cpr", 1, {}), ("mixed_cpr_fpf", 1, {"cpr_stages": 3}))}
    conv = conv_roofline()
    line = {
        "metric": "CPR-FGMRES time to 1e-8 rel. residual", "value": r["mixed_cpr_learned"]["seconds"], "unit": "s",
        "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32+bf16", "data": "synthetic",
        "config": {"workload": "black-oil 256x256x64 (4.2M cells), sigma 2, first Newton system; "
                               "network trained on 128x128x32 (sigma 1) pairs",
                   "train_seconds": ev["train_seconds"], "pairs_seconds": ev["pairs_seconds"],
                   "train_loss": ev["train_loss"][-3:]},
        "results": r, "fastest": best, "results_two_vcycles": r2,
        "roofline": conv["roofline"], "conv_kernels": conv["kernels"],
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
    ap.add_argument("--workload", default="bo400", choices=["bo100", "bo100c", "bo200", "bo400", "learned", "ensemble"])
    ap.add_argument("--oracle-cut", type=int, default=48, help="edge of the corner cut the oracle runs on")
    ap.add_argument("--mixed-steps", type=int, default=3,
                    help="Newton iterations of the FP32-preconditioner form timed after the FP64 ones (0: none)")
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
        if args.workload in ("learned", "ensemble"):
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm covers the single-grid workloads"}))
            return 0
        return run_reference(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
