"""Training and evaluation of the learned pressure stage (driver only: every
arithmetic step runs in the CUDA library; this module sequences the calls).

Training data are the simulator's own pressure systems: after each Newton
iteration's CPR-FGMRES solve, the first Krylov vectors of its last restart
cycle give pairs (pressure residual left by the stage-P V-cycle -> the error
it corresponds to, A_p^-1 r', from eight V-cycles of iterative refinement),
each normalised by its RMS, plus standardised log-transmissibility features
(include/sim.h, sim_learned_pairs).  The stage thus learns what the V-cycle
misses, and is applied to exactly that residual inside the preconditioner.  The network is trained on the
GPU by the library's own forward / backward kernels and Adam, then used as an
extra CPR stage on a larger, more heterogeneous grid, where the solve's time
to the FP64 tolerance is compared with plain FP64 CPR and FP32-preconditioned
CPR at the same tolerance.
"""
from __future__ import annotations

import time

import numpy as np

from . import synth
from .sim import Net, Simulator


def collect_pairs(case, newton_iterations=4, k=16, precision=1):
    """Pairs from the first Newton iterations of `case` (torch tensors on cuda)."""
    import torch
    sim = Simulator(case, precision=precision)
    N = sim.N
    xs, ys = [], []
    dt = case["dt"][0]
    for _ in range(newton_iterations):
        st, info = sim.newton_step(dt)
        if info.converged:
            break
        kk = min(k, sim.learned_available())
        if kk < 1:
            continue
        x = torch.empty((kk, N, 4), dtype=torch.float32, device="cuda")
        y = torch.empty((kk, N), dtype=torch.float32, device="cuda")
        sim.learned_pairs(kk, x, y)
        xs.append(x); ys.append(y)
    sim.close()
    return torch.cat(xs), torch.cat(ys)


def train(net, X, Y, steps=300, lr=1e-3, seed=0):
    """Adam on the pairs in a seeded random order; returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    order = rng.integers(0, X.shape[0], size=steps)
    hist = []
    for s, j in enumerate(order):
        want = (s % 25 == 0) or s == steps - 1
        loss = net.train_step(X[j].contiguous(), Y[j].contiguous(), lr, want_loss=want)
        if want:
            hist.append((s, loss))
    torch.cuda.synchronize()
    return hist


def time_solve(case, precision, net=None, repeats=1, **solver):
    """Time of the first Newton system's CPR-FGMRES solve to the tolerance
    (setup included), and its iterations; solver overrides the case's options."""
    import torch
    sim = Simulator(case, precision=precision, **solver)
    if net is not None:
        sim.set_learned_stage(net, True)
    dt = case["dt"][0]
    sim.assemble(dt)
    R = torch.tensor(sim.residual(), dtype=torch.float64, device="cuda")
    b = -R
    x = torch.empty_like(b)
    best = None
    for _ in range(max(1, repeats)):
        sim.assemble(dt)                     # invalidates the preconditioner: setup is timed too
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = sim.linear_solve(b, x)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        if best is None or t < best[0]:
            best = (t, info.iterations, info.converged, info.r_norm / max(info.b_norm, 1e-300))
    out = dict(seconds=best[0], iterations=best[1], converged=bool(best[2]), rel_residual=best[3],
               fallbacks=int(sim.learned_fallbacks()))
    sim.close()
    return out


def evaluate(train_case=None, eval_case=None, train_steps=300, lr=1e-3, pairs_newton=4, pairs_k=16, seed=0):
    """Train on train_case, then compare solves on eval_case: FP64 CPR
    (two-stage and CPR-FPF), FP32-preconditioned CPR (both), FP32 CPR + the
    learned stage (all to the same FP64 tolerance)."""
    train_case = train_case or synth.black_oil_128x128x32()
    eval_case = eval_case or synth.black_oil_256x256x64_sigma2()
    t0 = time.perf_counter()
    X, Y = collect_pairs(train_case, pairs_newton, pairs_k)
    t_pairs = time.perf_counter() - t0
    net_t = Net(train_case["nx"], train_case["ny"], train_case["nz"], seed=seed)
    t0 = time.perf_counter()
    hist = train(net_t, X, Y, train_steps, lr, seed)
    t_train = time.perf_counter() - t0
    params = net_t.get_params()
    net_t.close()
    del X, Y
    net_e = Net(eval_case["nx"], eval_case["ny"], eval_case["nz"], seed=seed)
    net_e.set_params(params)
    res = {
        "fp64_cpr": time_solve(eval_case, 0),
        "fp64_cpr_fpf": time_solve(eval_case, 0, cpr_stages=3),
        "mixed_cpr": time_solve(eval_case, 1),
        "mixed_cpr_fpf": time_solve(eval_case, 1, cpr_stages=3),
        "mixed_cpr_learned": time_solve(eval_case, 1, net=net_e),
    }
    net_e.close()
    return dict(train_loss=hist, pairs_seconds=t_pairs, train_seconds=t_train, results=res)
