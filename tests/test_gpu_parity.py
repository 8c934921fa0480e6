"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Element-by-element on the same seeded inputs: residual and Jacobian
assembly, block SpMV, quasi-IMPES weights and pressure block, AMG
aggregates and Galerkin operators (integer results bit-exact), CPR
application, FGMRES solutions and iteration counts, Newton updates and
whole time steps (pressure <= 1e-6 relative, saturations <= 1e-6 absolute,
Newton counts within 1).  Sizes span several thread blocks with ragged
tails; edge cases: one cell, one-dimensional grids, no wells.
"""
import numpy as np
import pytest

from paper_1606_00548_gb300 import synth
from helpers import random_state
from gpu_util import gpu_J_from_ora, ora_J_from_gpu, rel_err, to_cm, to_il

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_00548_gb300 import build
    build.build()
    return torch


def pair(case, **kw):
    import oracle
    from paper_1606_00548_gb300.sim import Simulator
    prec = kw.pop("precision", 0)
    return Simulator(case, precision=prec, **kw), oracle.Oracle(case, **kw)


CASES = {
    "ow_ragged": lambda: synth.oil_water_case(nx=37, ny=23, nz=7, sigma=1.0, seed=41),
    "bo_ragged": lambda: synth.black_oil_case(nx=29, ny=31, nz=6, seed=42),
    "ow_1d": lambda: synth.oil_water_case(nx=300, ny=1, nz=1, dy=1.0, dz=1.0, sigma=0.5, seed=43,
                                          wells=[synth.well(0, 0, 0, 0, 1, 230.0), synth.well(299, 0, 0, 0, 0, 170.0)]),
    "bo_column": lambda: synth.black_oil_case(nx=1, ny=1, nz=40, seed=44,
                                              wells=[synth.well(0, 0, 0, 9, 0, 180.0)]),
    "bo_no_wells": lambda: synth.black_oil_case(nx=9, ny=8, nz=5, seed=45, wells=[]),
    "ow_one_cell": lambda: synth.oil_water_case(nx=1, ny=1, nz=1, wells=[synth.well(0, 0, 0, 0, 0, 150.0)]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_assembly_matches_oracle(torch_cuda, name):
    case = CASES[name]()
    g, o = pair(case)
    N, b = g.N, g.b
    dt = 10.0 if case["model"] == 3 else 1.0
    x, ph = random_state(case, 3, N, b)
    o.set_iterate(x, ph); o.assemble(dt)
    g.set_iterate(to_cm(x, N, b), ph); g.assemble(dt)
    Ro, Jo = o.residual(), o.jacobian()
    Rg, Jg = to_il(g.residual(), N, b), ora_J_from_gpu(g.jacobian(), N, b)
    scale_R = np.abs(Ro).max()
    assert np.abs(Rg - Ro).max() <= 1e-11 * scale_R + 1e-300
    for d in range(7):
        sc = np.abs(Jo[:, 0]).max()
        assert np.abs(Jg[:, d] - Jo[:, d]).max() <= 1e-11 * sc, d
    assert abs(g.cnv(dt) - o.cnv(dt)) <= 1e-9 * max(o.cnv(dt), 1e-30)
    assert np.allclose(g.well_rates(), o.well_rates(), rtol=1e-11, atol=1e-9 * max(1.0, np.abs(o.well_rates()).max()))


@pytest.mark.parametrize("name", ["ow_ragged", "bo_ragged", "bo_column"])
def test_spmv_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    case = CASES[name]()
    g, o = pair(case)
    N, b = g.N, g.b
    dt = 10.0
    x, ph = random_state(case, 4, N, b)
    o.set_iterate(x, ph); o.assemble(dt)
    g.set_iterate(to_cm(x, N, b), ph); g.assemble(dt)
    v = np.random.default_rng(1).standard_normal(N * b)
    yo = o.spmv(v)
    xd = torch.tensor(to_cm(v, N, b), device="cuda", dtype=torch.float64)
    yd = torch.empty_like(xd)
    g.spmv(xd, yd)
    assert rel_err(to_il(yd.cpu().numpy(), N, b), yo) <= 1e-12


def _loaded_pair(case, dt, seed, **kw):
    """Both sides with the oracle's Jacobian, so integer AMG results must agree exactly.
    seed None: the Jacobian of the initial state (a physical, solvable system)."""
    g, o = pair(case, **kw)
    N, b = g.N, g.b
    if seed is not None:
        x, ph = random_state(case, seed, N, b)
        o.set_iterate(x, ph)
        g.set_iterate(to_cm(x, N, b), ph)
    o.assemble(dt); g.assemble(dt)
    g.set_jacobian(gpu_J_from_ora(o.jacobian(), N, b))
    o.precond_setup(); g.precond_setup()
    return g, o


@pytest.mark.parametrize("name", ["ow_ragged", "bo_ragged"])
@pytest.mark.parametrize("decouple", [0, 1])
def test_qi_and_amg_hierarchy_bitexact(torch_cuda, name, decouple):
    """Decoupling weights (first row of L: quasi-IMPES or ABF), the pressure
    block and the whole AMG hierarchy agree bit for bit."""
    case = CASES[name]()
    dt = 10.0 if case["model"] == 3 else 1.0
    g, o = _loaded_pair(case, dt, 5, amg_coarse_max=32, decouple=decouple)
    N, b = g.N, g.b
    wg, apg = g.qi()
    wo, apo = o.qi()
    assert np.array_equal(to_il(wg, N, b), wo)
    assert np.array_equal(apg.reshape(7, N).T, apo)
    lo, lg = o.amg_levels(), g.amg_levels()
    assert [L["n"] for L in lo] == [L["n"] for L in lg]
    assert len(lo) >= 3
    for l in range(len(lo) - 1):
        assert np.array_equal(lo[l]["agg"], lg[l]["agg"]), l
    for l in range(1, len(lo)):
        L = lo[l]
        n = L["n"]
        G = lg[l]
        for i in range(n):
            cols = L["col"][L["rowptr"][i]:L["rowptr"][i + 1]]
            vals = L["val"][L["rowptr"][i]:L["rowptr"][i + 1]]
            gc = G["col"][:, i]; gv = G["val"][:, i]
            k = len(cols)
            assert np.array_equal(gc[:k], cols) and (gc[k:] == -1).all()
            assert np.array_equal(gv[:k], vals)


@pytest.mark.parametrize("name", ["ow_ragged", "bo_ragged"])
@pytest.mark.parametrize("stage2,cycles,decouple,stages", [(0, 1, 0, 2), (1, 1, 0, 2), (1, 3, 0, 2), (1, 1, 1, 2),
                                                           (0, 1, 1, 2), (1, 1, 0, 3), (0, 1, 0, 3), (1, 2, 1, 3)])
def test_cpr_apply_matches_oracle(torch_cuda, name, stage2, cycles, decouple, stages):
    torch = torch_cuda
    case = CASES[name]()
    dt = 10.0 if case["model"] == 3 else 1.0
    g, o = _loaded_pair(case, dt, 6, stage2=stage2, amg_cycles=cycles, decouple=decouple, cpr_stages=stages)
    N, b = g.N, g.b
    r = np.random.default_rng(2).standard_normal(N * b)
    zo = o.precond_apply(r)
    rd = torch.tensor(to_cm(r, N, b), device="cuda", dtype=torch.float64)
    zd = torch.empty_like(rd)
    g.precond_apply(rd, zd)
    assert rel_err(to_il(zd.cpu().numpy(), N, b), zo) <= 1e-9


@pytest.mark.parametrize("name,cycles,decouple,stages,orth", [
    ("ow_ragged", 1, 0, 2, 0), ("bo_ragged", 1, 0, 2, 0), ("ow_1d", 1, 0, 2, 0), ("bo_column", 1, 0, 2, 0),
    ("bo_ragged", 2, 0, 2, 0), ("bo_ragged", 1, 1, 2, 0), ("bo_ragged", 1, 0, 3, 0), ("ow_ragged", 1, 1, 3, 0),
    ("bo_column", 1, 1, 3, 0), ("bo_ragged", 1, 0, 2, 1), ("ow_ragged", 1, 0, 2, 1)])
def test_linear_solve_matches_oracle(torch_cuda, name, cycles, decouple, stages, orth):
    torch = torch_cuda
    case = CASES[name]()
    dt = 10.0 if case["model"] == 3 else 1.0
    g, o = _loaded_pair(case, dt, None, amg_cycles=cycles, decouple=decouple, cpr_stages=stages, orth=orth)
    N, b = g.N, g.b
    rhs = np.random.default_rng(3).standard_normal(N * b)
    xo, io = o.linear_solve(rhs)
    bd = torch.tensor(to_cm(rhs, N, b), device="cuda", dtype=torch.float64)
    xd = torch.empty_like(bd)
    st, ig = g.linear_solve(bd, xd)
    assert ig.converged and io.converged
    assert abs(ig.iterations - io.iterations) <= 1
    # both meet ||b - J x|| <= 1e-8 ||b||: solutions agree to the conditioning of J
    assert ig.r_norm <= 1e-8 * ig.b_norm
    assert rel_err(to_il(xd.cpu().numpy(), N, b), xo) <= 1e-5


@pytest.mark.parametrize("name", ["ow_ragged", "bo_ragged", "bo_no_wells"])
def test_newton_step_matches_oracle(torch_cuda, name):
    case = CASES[name]()
    dt = 10.0 if case["model"] == 3 else 1.0
    g, o = pair(case)
    N, b = g.N, g.b
    sg, ig = g.newton_step(dt)
    so, io = o.newton_step(dt)
    xg, phg = g.get_iterate()
    xo, pho = o.get_iterate()
    xo = to_cm(xo, N, b)
    assert np.array_equal(phg, pho)
    assert rel_err(xg[:N], xo[:N]) <= 1e-6
    assert np.abs(xg[N:] - xo[N:]).max() <= 1e-6 * max(1.0, np.abs(xo[N:]).max())
    assert abs(ig.linear_iterations - io.linear_iterations) <= 1
    # the info's final linear residual: the true ||b - J dx|| / ||b|| the solve stopped at
    assert ig.linear_failures == 0 and 0.0 < ig.lin_residual <= 1e-8 * (1 + 1e-9), ig.lin_residual


def _run_steps(case, nsteps, precision=0):
    g, o = pair(case, precision=precision)
    rows = []
    for k in range(nsteps):
        dt = case["dt"][k]
        sg, ig = g.step(dt)
        so, io = o.step(dt)
        pg, swg, x3g, phg = g.get_state()
        po, swo, x3o, pho = o.get_state()
        rows.append(dict(dp=rel_err(pg, po), dsw=np.abs(swg - swo).max(),
                         dsg=np.abs(np.where(pho == 1, x3g - x3o, 0)).max(),
                         ph=int((phg != pho).sum()), ng=ig.newton_iterations, no=io.newton_iterations,
                         lg=ig.linear_iterations, lo=io.linear_iterations, cg=ig.cuts, co=io.cuts))
    return g, o, rows


@pytest.mark.parametrize("which", ["quarter_five_spot", "black_oil_small"])
def test_time_steps_match_oracle(torch_cuda, which):
    if which == "quarter_five_spot":
        case = synth.quarter_five_spot_20x20x5()
        nsteps = 10
    else:
        case = synth.black_oil_case(nx=24, ny=24, nz=6, nsteps=4, dt=10.0, seed=46)
        nsteps = 4
    g, o, rows = _run_steps(case, nsteps)
    for k, r in enumerate(rows):
        assert r["dp"] <= 1e-6 and r["dsw"] <= 1e-6 and r["dsg"] <= 1e-6 and r["ph"] == 0, (k, r)
        assert abs(r["ng"] - r["no"]) <= 1 and r["cg"] == r["co"], (k, r)
        # linear iterations within 1 per linear solve of the step
        assert abs(r["lg"] - r["lo"]) <= max(r["ng"], r["no"]), (k, r)
    mg, mo = g.component_mass(), o.component_mass()
    assert rel_err(mg, mo) <= 1e-9
    assert rel_err(g.cumulative_well_mass(), o.cumulative_well_mass()) <= 1e-6


@pytest.mark.parametrize("decouple,stages", [(0, 2), (1, 3)])
def test_mixed_precision_reaches_the_same_solution(torch_cuda, decouple, stages):
    case = synth.black_oil_case(nx=24, ny=24, nz=6, nsteps=3, dt=10.0, seed=47)
    case["solver"].update(decouple=decouple, cpr_stages=stages)
    g, o, rows = _run_steps(case, 3, precision=1)
    for k, r in enumerate(rows):
        assert r["dp"] <= 1e-6 and r["dsw"] <= 1e-6 and r["dsg"] <= 1e-6, (k, r)


def test_full_size_black_oil_100x100x20(torch_cuda):
    """The 200k-cell workload at full size: assembly element-wise, one linear
    solve and one Newton update against the oracle (pressure and bubble-point
    pressure 1e-6 relative, saturations 1e-6, linear iterations within 1)."""
    torch = torch_cuda
    case = synth.black_oil_100x100x20()
    g, o = pair(case)
    N, b = g.N, g.b
    dt = case["dt"][0]
    o.assemble(dt); g.assemble(dt)
    Ro, Jo = o.residual(), o.jacobian()
    assert np.abs(to_il(g.residual(), N, b) - Ro).max() <= 1e-11 * np.abs(Ro).max()
    Jg = ora_J_from_gpu(g.jacobian(), N, b)
    assert np.abs(Jg - Jo).max() <= 1e-11 * np.abs(Jo).max()
    sg, ig = g.newton_step(dt)
    so, io = o.newton_step(dt)
    xg, phg = g.get_iterate()
    xo, pho = o.get_iterate()
    xo = to_cm(xo, N, b)
    assert (phg != pho).sum() <= 0
    assert rel_err(xg[:N], xo[:N]) <= 1e-6
    assert np.abs(xg[N:2 * N] - xo[N:2 * N]).max() <= 1e-6          # Sw
    sat = pho == 1                                                    # x3: Sg where saturated, pb (bar) elsewhere
    assert np.abs(np.where(sat, xg[2 * N:] - xo[2 * N:], 0.0)).max() <= 1e-6
    assert rel_err(np.where(sat, 0.0, xg[2 * N:]), np.where(sat, 0.0, xo[2 * N:])) <= 1e-6
    assert abs(ig.linear_iterations - io.linear_iterations) <= 1


def test_graph_replay_matches_direct_launches(torch_cuda):
    """The restart cycle replayed as a CUDA graph gives the same iterates as
    launching its kernels one by one (identical arithmetic, same order)."""
    case = synth.black_oil_case(nx=24, ny=24, nz=6, nsteps=2, dt=10.0, seed=48)
    from paper_1606_00548_gb300.sim import Simulator
    a = Simulator(case, graphs=1)
    b = Simulator(case, graphs=0)
    for dt in case["dt"]:
        sa, ia = a.step(dt)
        sb, ib = b.step(dt)
        assert ia.newton_iterations == ib.newton_iterations and ia.linear_iterations == ib.linear_iterations
    pa = a.get_state(); pb = b.get_state()
    for u, v in zip(pa, pb):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("name,precond,decouple,stages", [("ow_ragged", 2, 0, 2), ("bo_ragged", 2, 0, 2),
                                                          ("bo_ragged", 2, 1, 3), ("bo_column", 2, 0, 2),
                                                          ("ow_1d", 1, 0, 2)])
def test_bicgstab_matches_oracle(torch_cuda, name, precond, decouple, stages):
    """BiCGSTAB (the paper's solver): iteration count within 2 of the oracle's
    (the recurrence amplifies rounding differences), both at the tolerance."""
    torch = torch_cuda
    case = CASES[name]()
    dt = 10.0 if case["model"] == 3 else 1.0
    g, o = _loaded_pair(case, dt, None, krylov=1, lin_max_iter=400, precond=precond, decouple=decouple,
                        cpr_stages=stages)
    N, b = g.N, g.b
    rhs = np.random.default_rng(8).standard_normal(N * b)
    xo, io = o.linear_solve(rhs)
    bd = torch.tensor(to_cm(rhs, N, b), device="cuda", dtype=torch.float64)
    xd = torch.empty_like(bd)
    st, ig = g.linear_solve(bd, xd)
    assert ig.converged and io.converged
    assert abs(ig.iterations - io.iterations) <= 2, (ig.iterations, io.iterations)
    assert ig.r_norm <= 1e-8 * ig.b_norm
    assert rel_err(to_il(xd.cpu().numpy(), N, b), xo) <= 1e-5


def test_bicgstab_iteration_limit_and_graph_replay(torch_cuda):
    """A solve stopped by the iteration limit returns the same iterate as the
    oracle's after the same number of iterations (no convergence reached)."""
    torch = torch_cuda
    case = CASES["bo_ragged"]()
    for graphs in (0, 1):
        g, o = _loaded_pair(case, 10.0, None, krylov=1, lin_max_iter=3, lin_tol=1e-14, graphs=graphs)
        N, b = g.N, g.b
        rhs = np.random.default_rng(9).standard_normal(N * b)
        xo, io = o.linear_solve(rhs)
        bd = torch.tensor(to_cm(rhs, N, b), device="cuda", dtype=torch.float64)
        xd = torch.empty_like(bd)
        st, ig = g.linear_solve(bd, xd)
        assert not ig.converged and ig.iterations == io.iterations == 3
        assert rel_err(to_il(xd.cpu().numpy(), N, b), xo) <= 1e-8


@pytest.mark.parametrize("forcing,krylov,precision", [(2, 1, 0), (1, 0, 0), (3, 1, 1)])
def test_forcing_terms_match_oracle(torch_cuda, forcing, krylov, precision):
    """Inexact Newton with the adaptive forcing terms of Eq. 14: the same
    number of Newton iterations (within 1) and the same converged state."""
    case = synth.black_oil_case(nx=24, ny=24, nz=6, nsteps=2, dt=1.0, seed=48)
    case["solver"].update(forcing=forcing, krylov=krylov)
    g, o, rows = _run_steps(case, 2, precision=precision)
    for k, r in enumerate(rows):
        assert r["dp"] <= 1e-6 and r["dsw"] <= 1e-6 and r["dsg"] <= 1e-6, (k, r)
        assert abs(r["ng"] - r["no"]) <= 1, (k, r)


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_coarse_cycle_matches_per_level_kernels(torch_cuda, precision):
    """The one-launch cluster kernel for the coarse AMG levels computes what
    the per-level kernels compute (same row operations, same order)."""
    torch = torch_cuda
    from paper_1606_00548_gb300.sim import Simulator
    case = CASES["bo_ragged"]()
    out = []
    for fused in (0, 1):
        g = Simulator(case, precision=precision, amg_coarse_max=32, fused_coarse=fused)
        N, b = g.N, g.b
        g.assemble(10.0)
        g.precond_setup()
        assert len(g.amg_levels()) >= 4
        r = np.random.default_rng(11).standard_normal(N * b)
        rd = torch.tensor(r, device="cuda", dtype=torch.float64)
        zd = torch.empty_like(rd)
        g.precond_apply(rd, zd)
        out.append(zd.cpu().numpy())
    tol = 1e-13 if precision == 0 else 1e-6
    assert rel_err(out[1], out[0]) <= tol


def test_time_op_leaves_state_and_reports_time(torch_cuda):
    """The measurement entry point times both operations without touching the
    simulator's state (a later solve gives the same answer as before)."""
    torch = torch_cuda
    case = CASES["bo_ragged"]()
    g, o = _loaded_pair(case, 10.0, None)
    N, b = g.N, g.b
    rhs = torch.tensor(np.random.default_rng(12).standard_normal(N * b), device="cuda", dtype=torch.float64)
    x1 = torch.empty_like(rhs); x2 = torch.empty_like(rhs)
    st, i1 = g.linear_solve(rhs, x1)
    t_spmv, t_prec = g.time_op(0, 5), g.time_op(1, 5)
    assert 0.0 < t_spmv < 1e5 and 0.0 < t_prec < 1e5
    st, i2 = g.linear_solve(rhs, x2)
    assert i1.iterations == i2.iterations and torch.equal(x1, x2)


@pytest.mark.parametrize("which", ["quarter_five_spot", "black_oil_small"])
def test_step_reports_its_mass_balance_error(torch_cuda, which):
    """sim_step_info.mb_error: |M_c(end) - M_c(start) - dt q_c| / sum_c M_c, the
    conservation of Eq. (3) over the step.  With CNV at 1e-10 it stays near
    that level, and for a step without cuts it equals what the component
    masses and the cumulative well masses of the API give."""
    from paper_1606_00548_gb300.sim import Simulator
    if which == "quarter_five_spot":
        case = synth.quarter_five_spot_20x20x5(nsteps=3)
    else:
        case = synth.black_oil_case(nx=24, ny=24, nz=6, nsteps=3, dt=10.0, seed=46)
    g = Simulator(case)
    m0, c0 = np.array(g.component_mass()), np.array(g.cumulative_well_mass())
    worst = 0.0
    for dt in case["dt"]:
        st, info = g.step(dt)
        assert st == 0
        m1, c1 = np.array(g.component_mass()), np.array(g.cumulative_well_mass())
        assert 0.0 < info.mb_error <= 1e-9, info.mb_error
        if info.substeps == 1:
            ref = np.abs((m1 - m0) - (c1 - c0))[:g.b].max() / m1[:g.b].sum()
            assert abs(info.mb_error - ref) <= 1e-6 * ref + 1e-15, (info.mb_error, ref)
        worst = max(worst, info.mb_error)
        m0, c0 = m1, c1
    assert g.run_report()["counters"]["max_mass_balance_error"] == pytest.approx(worst, rel=1e-3)
