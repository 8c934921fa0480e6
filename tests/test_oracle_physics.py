"""Pins of the oracle's full Newton time step against physics with known answers.

* Buckley-Leverett: incompressible 1-D waterflood of the two-phase model
  (Eq. 5) with Corey curves (Sec. 4.1); the saturation profile converges to
  the Welge/BL solution (constants in golden/buckley_leverett.json) as the
  grid is refined at fixed Courant number.
* single-phase incompressible flow between two BHP wells (Eq. 6-7): the
  steady pressure is linear across interior cells and every face carries the
  well rate T * lambda * dp (Eq. 11).
* cumulative mass balance of each component after every time step (the
  conservation form of Eq. 3 with Eq. 10 time stepping).
* the quarter five-spot on a square homogeneous grid stays symmetric about
  its diagonal.
"""
import json
import os

import numpy as np
import pytest

from paper_1606_00548_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "buckley_leverett.json")))


def _fprime(S, swc, sor, mu_o, mu_w):
    se = (S - swc) / (1 - swc - sor)
    a = mu_w / mu_o
    D = se ** 2 + a * (1 - se) ** 2
    return 2 * a * se * (1 - se) / D ** 2 / (1 - swc - sor)


def _bl_profile(xd, pvi):
    g = GOLD
    Sf = g["front_saturation"]
    out = np.full(xd.shape, g["swc"])
    for k, x in enumerate(xd):
        if x <= pvi * _fprime(Sf, g["swc"], g["sor"], g["mu_o"], g["mu_w"]):
            lo, hi = Sf, 1 - g["sor"]
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                if pvi * _fprime(mid, g["swc"], g["sor"], g["mu_o"], g["mu_w"]) > x:
                    lo = mid
                else:
                    hi = mid
            out[k] = 0.5 * (lo + hi)
    return out


def test_golden_constants_are_the_welge_solution():
    g = GOLD
    M = g["mu_o"] / g["mu_w"]
    Sf = g["swc"] + (1 - g["swc"] - g["sor"]) / np.sqrt(1 + M)
    assert Sf == pytest.approx(g["front_saturation"], abs=1e-6)
    v = _fprime(Sf, g["swc"], g["sor"], g["mu_o"], g["mu_w"])
    assert v == pytest.approx(g["front_speed_per_pv"], abs=1e-6)
    assert 1 / v == pytest.approx(g["breakthrough_pvi"], abs=1e-6)


def _bl_case(N, L=100.0):
    fl = synth.oil_water_fluid(c=0.0)
    return synth.oil_water_case(
        nx=N, ny=1, nz=1, dx=L / N, dy=1.0, dz=1.0, k=1000.0, poro=0.2, fluid=fl,
        wells=[synth.well(0, 0, 0, 0, synth.WATER_INJECTOR, 220.0),
               synth.well(N - 1, 0, 0, 0, synth.PRODUCER, 200.0)])


def test_buckley_leverett_converges_under_refinement(oracle_lib):
    import oracle
    errs = []
    for N in (25, 50, 100, 200):
        o = oracle.Oracle(_bl_case(N))
        pv = 100.0 * 0.2
        pvi = 0.0
        while pvi < 0.3:
            rc, info = o.step(10.0 / N)       # fixed Courant number
            assert rc == 0
            pvi = o.cumulative_well_mass()[0] / 1000.0 / pv
        _, sw, _, _ = o.get_state()
        xd = (np.arange(N) + 0.5) / N
        errs.append(np.abs(sw - _bl_profile(xd, pvi)).mean())
    for a, b in zip(errs, errs[1:]):
        assert b < 0.8 * a
    assert errs[-1] < 0.02


def test_single_phase_linear_pressure(oracle_lib):
    import oracle
    N = 20
    fl = synth.oil_water_fluid(c=0.0)
    case = synth.oil_water_case(
        nx=N, ny=1, nz=1, dx=5.0, dy=2.0, dz=1.0, k=250.0, poro=0.25, fluid=fl,
        wells=[synth.well(0, 0, 0, 0, synth.PRODUCER, 260.0),      # backflow: injects the cell's oil
               synth.well(N - 1, 0, 0, 0, synth.PRODUCER, 140.0)])
    o = oracle.Oracle(case, lin_tol=1e-12)
    rc, _ = o.step(1.0)
    assert rc == 0
    p, sw, _, _ = o.get_state()
    dp = np.diff(p)
    assert np.abs(dp - dp.mean()).max() <= 1e-10 * abs(dp.mean())
    assert np.allclose(sw, 0.1, atol=1e-14)          # only oil flows
    # face flux = T * rho_o / mu_o * dp equals the injected oil rate
    T = (86400.0 * 9.869233e-16 * 1e5 / 1e-3) * 250.0 * 2.0 * 1.0 / 5.0
    face_rate = T * 800.0 / 2.0 * (-dp.mean())
    # steady state: the oil entering at one well leaves at the other
    q = o.well_rates()
    assert abs(q[1]) <= 1e-8 * face_rate
    assert face_rate > 0


@pytest.mark.parametrize("which", ["ow", "bo"])
def test_cumulative_mass_balance(oracle_lib, which):
    import oracle
    if which == "ow":
        case = synth.quarter_five_spot_20x20x5(nsteps=4)
    else:
        case = synth.black_oil_case(nx=12, ny=12, nz=4, nsteps=4, dt=5.0)
    o = oracle.Oracle(case)
    m0 = o.component_mass()
    for dt in case["dt"]:
        rc, info = o.step(dt)
        assert rc == 0
        m = o.component_mass()
        cum = o.cumulative_well_mass()
        total = m0.sum()
        for c in range(o.b):
            assert abs(m[c] - m0[c] - cum[c]) <= 1e-10 * total


def test_quarter_five_spot_diagonal_symmetry(oracle_lib):
    import oracle
    case = synth.quarter_five_spot_20x20x5(nsteps=2)
    o = oracle.Oracle(case)
    for dt in case["dt"]:
        assert o.step(dt)[0] == 0
    p, sw, _, _ = o.get_state()
    P = p.reshape(5, 20, 20); S = sw.reshape(5, 20, 20)
    assert np.abs(P - P.transpose(0, 2, 1)).max() <= 1e-9 * np.abs(P).max()
    assert np.abs(S - S.transpose(0, 2, 1)).max() <= 1e-8
