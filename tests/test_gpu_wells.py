"""Parity of the rate-controlled wells (Sec. 2.3, Eq. 8-9, Eq. 16) on the GPU
with the oracle: border blocks of the assembly, the Schur operator S, the
preconditioner built from S on the 7-point pattern (AMG hierarchy
bit-exact), linear solves and whole time steps with BHP unknowns."""
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


def rate_case(model=3, nx=21, ny=17, nz=5, seed=101):
    """Two rate-controlled wells (water-rate injector, oil-rate producer) and
    two BHP producers on a ragged grid."""
    wells = [synth.well(2, 3, 0, nz - 1, synth.WATER_INJECTOR, 230.0, ctrl=1, rate=4.0e4),
             synth.well(nx - 3, ny - 2, 0, nz - 1, synth.PRODUCER, 185.0, ctrl=2, rate=-2.5e4),
             synth.well(nx - 2, 1, 1, nz - 2, synth.PRODUCER, 180.0),
             synth.well(1, ny - 2, 0, 0, synth.PRODUCER, 182.0)]
    if model == 3:
        return synth.black_oil_case(nx=nx, ny=ny, nz=nz, seed=seed, wells=wells)
    return synth.oil_water_case(nx=nx, ny=ny, nz=nz, sigma=1.0, seed=seed, wells=wells)


def pair(case, **kw):
    import oracle
    from paper_1606_00548_gb300.sim import Simulator
    prec = kw.pop("precision", 0)
    return Simulator(case, precision=prec, **kw), oracle.Oracle(case, **kw)


BHP0 = np.array([226.0, 188.0, 180.0, 182.0])


@pytest.mark.parametrize("model", [3, 2])
def test_well_assembly_matches_oracle(torch_cuda, model):
    case = rate_case(model)
    g, o = pair(case)
    N, b = g.N, g.b
    dt = 10.0 if model == 3 else 1.0
    x, ph = random_state(case, 3, N, b)
    o.set_iterate(x, ph); o.set_well_bhp(BHP0); o.assemble(dt)
    g.set_iterate(to_cm(x, N, b), ph); g.set_well_bhp(BHP0); g.assemble(dt)
    Ro, Jo = o.residual(), o.jacobian()
    Rg, Jg = to_il(g.residual(), N, b), ora_J_from_gpu(g.jacobian(), N, b)
    assert np.abs(Rg - Ro).max() <= 1e-11 * np.abs(Ro).max()
    assert np.abs(Jg[:, 0] - Jo[:, 0]).max() <= 1e-11 * np.abs(Jo[:, 0]).max()
    so, sg = o.well_system(), g.well_system()
    for a, c in zip(so, sg):
        assert np.abs(c - a).max() <= 1e-11 * max(np.abs(a).max(), 1.0)
    qo, qg = o.well_component_rates(), g.well_component_rates()
    assert np.abs(qg - qo).max() <= 1e-11 * np.abs(qo).max()
    assert np.array_equal(g.well_bhp(), BHP0)


def _loaded(case, dt, **kw):
    """Both sides on the oracle's Jacobian and border blocks."""
    g, o = pair(case, **kw)
    N, b = g.N, g.b
    o.set_well_bhp(BHP0); g.set_well_bhp(BHP0)
    o.assemble(dt); g.assemble(dt)
    g.set_jacobian(gpu_J_from_ora(o.jacobian(), N, b))
    g.set_well_system(*o.well_system())
    o.precond_setup(); g.precond_setup()
    return g, o


@pytest.mark.parametrize("decouple", [0, 1])
def test_schur_operator_and_hierarchy_bitexact(torch_cuda, decouple):
    torch = torch_cuda
    case = rate_case()
    g, o = _loaded(case, 10.0, amg_coarse_max=32, decouple=decouple)
    N, b = g.N, g.b
    v = np.random.default_rng(1).standard_normal(N * b)
    yo = o.spmv(v)
    xd = torch.tensor(to_cm(v, N, b), device="cuda", dtype=torch.float64)
    yd = torch.empty_like(xd)
    g.spmv(xd, yd)
    assert rel_err(to_il(yd.cpu().numpy(), N, b), yo) <= 1e-12
    wg, apg = g.qi()
    wo, apo = o.qi()
    assert np.array_equal(to_il(wg, N, b), wo)
    assert np.array_equal(apg.reshape(7, N).T, apo)
    lo, lg = o.amg_levels(), g.amg_levels()
    assert [L["n"] for L in lo] == [L["n"] for L in lg]
    for l in range(len(lo) - 1):
        assert np.array_equal(lo[l]["agg"], lg[l]["agg"]), l


@pytest.mark.parametrize("stages,stage2", [(2, 1), (3, 0)])
def test_cpr_apply_and_solve_with_rate_wells(torch_cuda, stages, stage2):
    torch = torch_cuda
    case = rate_case()
    g, o = _loaded(case, 10.0, cpr_stages=stages, stage2=stage2)
    N, b = g.N, g.b
    r = np.random.default_rng(2).standard_normal(N * b)
    zo = o.precond_apply(r)
    rd = torch.tensor(to_cm(r, N, b), device="cuda", dtype=torch.float64)
    zd = torch.empty_like(rd)
    g.precond_apply(rd, zd)
    assert rel_err(to_il(zd.cpu().numpy(), N, b), zo) <= 1e-9
    xo, io = o.linear_solve(r)
    xd = torch.empty_like(rd)
    st, ig = g.linear_solve(rd, xd)
    assert ig.converged and io.converged and abs(ig.iterations - io.iterations) <= 1
    assert rel_err(to_il(xd.cpu().numpy(), N, b), xo) <= 1e-5


@pytest.mark.parametrize("model,krylov,precision", [(3, 0, 0), (2, 0, 0), (3, 1, 0), (3, 0, 1)])
def test_time_steps_with_rate_wells(torch_cuda, model, krylov, precision):
    case = rate_case(model)
    case["solver"].update(krylov=krylov)
    g, o = pair(case, precision=precision)
    dts = [1.0, 2.0, 5.0] if model == 3 else [0.5, 1.0, 1.0]
    for k, dt in enumerate(dts):
        sg, ig = g.step(dt)
        so, io = o.step(dt)
        assert ig.ok and io.ok, k
        pg, swg, x3g, phg = g.get_state()
        po, swo, x3o, pho = o.get_state()
        assert rel_err(pg, po) <= 1e-6 and np.abs(swg - swo).max() <= 1e-6, k
        assert np.abs(g.well_bhp() - o.well_bhp()).max() <= 1e-6 * 250.0, k
        assert abs(ig.newton_iterations - io.newton_iterations) <= 1, k
    # the rate targets are met at the end of each step
    q = g.well_component_rates()
    assert q[0, 0] == pytest.approx(4.0e4, rel=1e-8)
    assert q[1, 1] == pytest.approx(-2.5e4, rel=1e-8)
    mg, cg = g.component_mass(), g.cumulative_well_mass()
    mo, co = o.component_mass(), o.cumulative_well_mass()
    assert np.abs(np.asarray(mg) - mo).max() <= 1e-8 * np.abs(mo).max()
