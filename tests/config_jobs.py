"""Oracle runs of the full-size configurations, for the per-configuration
parity tests (tests/test_gpu_configs.py).  Each job is a plain function of
picklable arguments so that it runs in a spawned worker process while the GPU
side of the tests runs in the main process; it returns the oracle's states
and counts after every time step (or Newton step).  Inputs come from
paper_1606_00548_gb300.synth only."""
from __future__ import annotations

import numpy as np


def corner_cut(case, n):
    """The n x n x n corner of a case (rock, initial state and the wells whose
    column lies inside, perforations clipped to the cut)."""
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    cx, cy, cz = min(n, nx), min(n, ny), min(n, nz)

    def sub(a):
        return np.ascontiguousarray(np.asarray(a).reshape(nz, ny, nx)[:cz, :cy, :cx].reshape(-1))

    out = dict(case)
    out.update(nx=cx, ny=cy, nz=cz, name=f"{case['name']} corner {cx}x{cy}x{cz}")
    for k in ("kx", "ky", "kz", "poro"):
        out[k] = sub(case[k])
    out["init"] = {k: sub(v) for k, v in case["init"].items()}
    out["wells"] = [dict(w, k1=min(w["k1"], cz - 1)) for w in case["wells"]
                    if w["i"] < cx and w["j"] < cy and w["k0"] < cz]
    return out


def case_of(name):
    from paper_1606_00548_gb300 import synth
    if name == "black_oil_100x100x20":
        return synth.black_oil_100x100x20()
    if name == "black_oil_400cube_corner100":
        return corner_cut(synth.black_oil_400cube(n=400), 100)
    if name == "learned_eval_256x256x64":
        return synth.black_oil_256x256x64_sigma2()
    raise KeyError(name)


def run_steps(name, nsteps, **solver):
    """The oracle through nsteps time steps of a case: per step the state and
    the step's counts."""
    import oracle
    case = case_of(name)
    o = oracle.Oracle(case, **solver)
    out = []
    for k in range(nsteps):
        rc, info = o.step(case["dt"][k])
        p, sw, x3, ph = o.get_state()
        out.append(dict(rc=rc, p=p, sw=sw, x3=x3, ph=ph, newton=info.newton_iterations,
                        linear=info.linear_iterations, cuts=info.cuts, substeps=info.substeps))
    return out


def run_newton(name, **solver):
    """One oracle Newton step of a case from its initial state."""
    import oracle
    case = case_of(name)
    o = oracle.Oracle(case, **solver)
    rc, info = o.newton_step(case["dt"][0])
    x, ph = o.get_iterate()
    return dict(rc=rc, x=x, ph=ph, linear=info.linear_iterations)


def run_members(scale, nsteps, first, count):
    """Oracle time steps of ensemble members first..first+count-1."""
    import oracle
    from paper_1606_00548_gb300 import synth
    members = synth.ensemble_members(64, nsteps=nsteps, dt=1.0, scale=scale)[first:first + count]
    out = []
    for case in members:
        o = oracle.Oracle(case)
        rows = []
        for k in range(nsteps):
            rc, info = o.step(case["dt"][k])
            p, sw, _, _ = o.get_state()
            rows.append(dict(rc=rc, p=p, sw=sw, newton=info.newton_iterations, linear=info.linear_iterations,
                             cuts=info.cuts, substeps=info.substeps))
        out.append(rows)
    return out
