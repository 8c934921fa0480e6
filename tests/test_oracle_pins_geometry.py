"""Pins of three parts of the oracle's discretisation against physics with a
known answer: gravity in the phase potential (Eq. 4, read with depth positive
down), the harmonic two-point transmissibility between cells of different
permeability (Eq. 11) and the Peaceman well index of the well model (Sec. 2.3,
Eq. 6).  Each case is chosen so that a plausible mistake fails it: a flipped
gravity sign or a missing bar conversion sets a column at rest flowing; an
arithmetic instead of a harmonic mean changes the pressure drop across every
layer interface; a wrong equivalent radius, a missing 2 pi or a dropped skin
moves the wellbore pressure off the radial-flow solution.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1606_00548_gb300 import synth

G = 9.80665
DARCY_C = 86400.0 * 9.869233e-16 * 1e5 / 1e-3   # m3 cP / (day mD m bar)
GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# gravity: a closed column initialised in hydrostatic equilibrium stays at rest
# ---------------------------------------------------------------------------
def _hydrostatic_column(p_top, depth, rho_of_p):
    """Pressures of a column in discrete hydrostatic equilibrium: between two
    neighbouring cell centres p_{k+1} - p_k = rho_face g dz / 1e5 with the face
    density the mean of the two cells' densities (fixed point per cell)."""
    p = [p_top]
    for k in range(1, len(depth)):
        dzk = depth[k] - depth[k - 1]
        q = p[-1] + rho_of_p(p[-1]) * G * dzk / 1e5
        for _ in range(60):
            q = p[-1] + 0.5 * (rho_of_p(p[-1]) + rho_of_p(q)) * G * dzk / 1e5
        p.append(q)
    return np.array(p)


def _column_case(model, nz):
    if model == "ow":
        fl = synth.oil_water_fluid(c=1e-5)
        case = synth.oil_water_case(nx=1, ny=1, nz=nz, dx=10.0, dy=10.0, dz=2.0, k=100.0, poro=0.2,
                                    fluid=fl, wells=[])
        # oil only is mobile at S_w = S_wc; its density law is the input's rho_ref exp(c (p - p_ref))
        rho = lambda p: fl["rho_o_ref"] * math.exp(fl["c_o"] * (p - 200.0))
    else:
        case = synth.black_oil_case(nx=1, ny=1, nz=nz, sigma=0.0, wells=[], nsteps=3, dt=10.0)
        fl = case["fluid"]
        pb = 200.0
        rs = np.interp(pb, fl["pvt_p"], fl["pvt_rs"])
        bo_sat = np.interp(pb, fl["pvt_p"], fl["pvt_bo"])
        # undersaturated oil: surface oil plus the gas dissolved at pb, in the volume Bo(p, pb)
        rho = lambda p: (fl["rho_os"] + fl["rho_gs"] * rs) / (bo_sat * (1.0 - fl["bo_c_us"] * (p - pb)))
    depth = case["top_depth"] + (np.arange(nz) + 0.5) * case["dz"]
    return case, depth, rho


@pytest.mark.parametrize("model", ["ow", "bo"])
def test_hydrostatic_column_stays_at_rest(oracle_lib, model):
    import oracle
    nz = 20
    case, depth, rho = _column_case(model, nz)
    p_eq = _hydrostatic_column(250.0, depth, rho)
    init = case["init"]
    o = oracle.Oracle(case)
    # the same column at uniform pressure: gravity alone drives the oil down
    o.set_state(np.full(nz, 250.0), init["sw"], init["x3"], init["phase"])
    o.assemble(1.0)
    r_flow = np.abs(o.residual()).max()
    assert r_flow > 1.0
    o.set_state(p_eq, init["sw"], init["x3"], init["phase"])
    o.assemble(1.0)
    assert np.abs(o.residual()).max() <= 1e-10 * r_flow
    for _ in range(3):
        rc, info = o.step(10.0)
        assert rc == 0
    p, sw, x3, ph = o.get_state()
    assert np.abs(p - p_eq).max() <= 1e-10 * p_eq.max()
    assert np.abs(sw - init["sw"]).max() <= 1e-12


# ---------------------------------------------------------------------------
# harmonic transmissibility: steady single-phase flow through layers in series
# ---------------------------------------------------------------------------
LAYERS = [50.0, 400.0, 20.0, 150.0]      # mD, five cells each


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_series_layers_follow_the_resistance_law(oracle_lib, axis):
    """Incompressible oil flows along one axis through four layers of different
    permeability between two BHP wells.  In steady state every face carries the
    same rate q, so the potential drop over a face inside layer a is
    q h / (C k_a A lambda), and over the face between layers a and b the two
    half-cell resistances add: q (h / 2) (1 / k_a + 1 / k_b) / (C A lambda)."""
    import oracle
    n = 5 * len(LAYERS)
    dims = [1, 1, 1]
    dims[axis] = n
    nx, ny, nz = dims
    h = [10.0, 8.0, 2.0]
    kcell = np.repeat(LAYERS, 5)
    fl = synth.oil_water_fluid(c=0.0)
    first = [0, 0, 0]; last = [0, 0, 0]; last[axis] = n - 1
    wells = [synth.well(first[0], first[1], first[2], first[2], synth.PRODUCER, 260.0),   # backflow: injects oil
             synth.well(last[0], last[1], last[2], last[2], synth.PRODUCER, 140.0)]
    case = synth.oil_water_case(nx=nx, ny=ny, nz=nz, dx=h[0], dy=h[1], dz=h[2], k=100.0, poro=0.2,
                                fluid=fl, wells=wells)
    for name in ("kx", "ky", "kz"):
        case[name] = kcell.copy()
    o = oracle.Oracle(case, lin_tol=1e-13)
    rc, _ = o.step(1.0)
    assert rc == 0
    p = o.get_state()[0]
    rho, mu = fl["rho_o_ref"], fl["mu_o"]
    depth = case["top_depth"] + (np.arange(nz) + 0.5) * h[2]
    z = np.repeat(depth, nx * ny) if axis != 2 else depth
    dphi = np.diff(p) - rho * G * np.diff(z) / 1e5          # potential drop between neighbours (Eq. 4)
    area = h[0] * h[1] * h[2] / h[axis]
    q_vol = -o.well_component_rates()[1][1] / rho            # m3/day leaving through the low-BHP well
    assert q_vol > 0
    unit = q_vol * h[axis] * mu / (DARCY_C * area)           # q h / (C A lambda) per mD^-1
    expect = []
    for f in range(n - 1):
        ka, kb = kcell[f], kcell[f + 1]
        expect.append(-unit / ka if ka == kb else -unit * 0.5 * (1.0 / ka + 1.0 / kb))
    expect = np.array(expect)
    assert np.abs(dphi - expect).max() <= 1e-9 * np.abs(expect).max()
    # the total drop between the well cells is the sum of the series resistances
    assert abs(dphi.sum() - expect.sum()) <= 1e-9 * abs(expect.sum())


# ---------------------------------------------------------------------------
# Peaceman well index
# ---------------------------------------------------------------------------
def _well_index_from_rate(kx, ky, dx, dy, dz, rw, skin):
    """Well index of a one-cell reservoir read off the oracle's well rate:
    q_oil = WI (rho_o k_ro / mu_o) (p_h - p) with oil only mobile (S_w = S_wc,
    k_ro = 1) and the perforation at the cell centre (no head term)."""
    import oracle
    fl = synth.oil_water_fluid(c=0.0)
    case = synth.oil_water_case(nx=1, ny=1, nz=1, dx=dx, dy=dy, dz=dz, k=100.0, poro=0.2, fluid=fl,
                                wells=[synth.well(0, 0, 0, 0, synth.PRODUCER, 150.0, rw=rw, skin=skin)])
    case["kx"] = np.array([kx]); case["ky"] = np.array([ky]); case["kz"] = np.array([0.1 * kx])
    o = oracle.Oracle(case)
    o.set_state(np.array([200.0]), np.array([fl["swc"]]), np.zeros(1), np.ones(1, np.int8))
    o.assemble(1.0)
    q_oil = o.well_component_rates()[0][1]
    return q_oil / (fl["rho_o_ref"] / fl["mu_o"] * (150.0 - 200.0))


def test_peaceman_index_of_an_anisotropic_cell(oracle_lib):
    g = json.load(open(os.path.join(GOLD, "peaceman_anisotropic.json")))
    c = g["cell"]
    wi = _well_index_from_rate(c["kx_mD"], c["ky_mD"], c["dx_m"], c["dy_m"], c["dz_m"], c["r_w_m"], c["skin"])
    assert wi == pytest.approx(g["well_index"], rel=1e-10)
    # the same cell turned by 90 degrees (kx <-> ky with dx <-> dy) has the same index
    wi_t = _well_index_from_rate(c["ky_mD"], c["kx_mD"], c["dy_m"], c["dx_m"], c["dz_m"], c["r_w_m"], c["skin"])
    assert wi_t == pytest.approx(g["well_index"], rel=1e-10)


@pytest.mark.parametrize("skin", [0.0, 2.0])
def test_peaceman_index_reproduces_radial_flow(oracle_lib, skin):
    """Peaceman's defining property: with the well index, the wellbore pressure
    is tied to the grid pressures by steady radial flow,
    p(r) - p_h = q mu / (2 pi C k h) (ln(r / r_w) + s), for cells a few blocks
    from the well (here the centre well of a 41 x 41 grid whose corner wells
    feed it; the lattice and far-field corrections are below 0.3 % at 3-6
    blocks).  An equivalent radius of 0.28 dx instead of 0.198 dx, for one,
    is off by 6 %."""
    import oracle
    n = 41
    fl = synth.oil_water_fluid(c=0.0)
    ws = [synth.well(20, 20, 0, 0, synth.PRODUCER, 100.0, skin=skin)]
    ws += [synth.well(i, j, 0, 0, synth.PRODUCER, 300.0) for i, j in ((0, 0), (n - 1, 0), (0, n - 1), (n - 1, n - 1))]
    k, h, dx, rw = 100.0, 2.0, 10.0, 0.1
    case = synth.oil_water_case(nx=n, ny=n, nz=1, dx=dx, dy=dx, dz=h, k=k, poro=0.2, fluid=fl, wells=ws)
    o = oracle.Oracle(case, lin_tol=1e-12)
    rc, _ = o.step(1.0)
    assert rc == 0
    P = o.get_state()[0].reshape(n, n)
    q_vol = -o.well_component_rates()[0][1] / fl["rho_o_ref"]
    A = q_vol * fl["mu_o"] / (2.0 * math.pi * DARCY_C * k * h)
    for r in (3, 4, 6):
        radial = A * (math.log(r * dx / rw) + skin)
        for pr in (P[20, 20 + r], P[20 + r, 20], P[20, 20 - r], P[20 - r, 20]):
            assert abs((pr - 100.0) / radial - 1.0) <= 5e-3
