"""Pins of the oracle's fluid and rock properties against closed forms.

Relative permeability: Corey curves (Sec. 4.1) and Stone II (Sec. 2.1), which
must reduce to the two-phase oil curves when one of the other phases is
absent.  PVT: tabulated properties (Sec. 2.1 allows analytic formulas or
tables) reproduce the table at its nodes and are linear between them.
Derivatives carried by the oracle's dual numbers are checked against central
differences of the values.
"""
import numpy as np
import pytest

from paper_1606_00548_gb300 import synth

KRW, KRO, KRG, RHO_W, RHO_O, RHO_G, MOB_WW, MOB_OO, MOB_OG, MOB_GG, BO, RS, MUO = range(13)
ACC_W, ACC_O, ACC_G, LAMT = 13, 14, 15, 16


@pytest.fixture(scope="module")
def ow(oracle_lib):
    return synth.oil_water_case(nx=2, ny=1, nz=1)


@pytest.fixture(scope="module")
def bo(oracle_lib):
    return synth.black_oil_case(nx=2, ny=2, nz=1)


def probe(case, what, p, sw, x3=0.0, ph=1):
    import oracle
    return oracle.props_probe(case, what, p, sw, x3, ph)


def test_corey_oil_water(ow):
    for sw in (0.05, 0.1, 0.3, 0.5, 0.77, 0.9, 0.95):
        se = min(1.0, max(0.0, (sw - 0.1) / 0.8))
        assert probe(ow, KRW, 200.0, sw)[0] == pytest.approx(se ** 2, abs=1e-15)
        assert probe(ow, KRO, 200.0, sw)[0] == pytest.approx((1 - se) ** 2, abs=1e-15)


def test_oil_water_density_exponential(ow):
    for p in (100.0, 200.0, 317.0):
        assert probe(ow, RHO_W, p, 0.5)[0] == pytest.approx(1000.0 * np.exp(1e-5 * (p - 200.0)), rel=1e-14)
        assert probe(ow, RHO_O, p, 0.5)[0] == pytest.approx(800.0 * np.exp(1e-5 * (p - 200.0)), rel=1e-14)


def test_stone2_reduces_to_two_phase_curves(bo):
    # Sg = 0 (gas absent): kro = krow(Sw)
    for sw in (0.1, 0.2, 0.45, 0.7, 0.85):
        krow = ((1 - 0.1 - sw) / 0.8) ** 2
        assert probe(bo, KRO, 200.0, sw, 0.0, 1)[0] == pytest.approx(krow, abs=1e-14)
    # Sw = Swc (water immobile): kro = krog(Sg)
    for sg in (0.0, 0.03, 0.2, 0.5, 0.75):
        krog = max(0.0, (1 - 0.1 - 0.1 - sg) / 0.8) ** 2
        assert probe(bo, KRO, 200.0, 0.1, sg, 1)[0] == pytest.approx(krog, abs=1e-14)


def test_gas_relperm_corey(bo):
    for sg in (0.0, 0.04, 0.05, 0.1, 0.4, 0.9):
        se = min(1.0, max(0.0, (sg - 0.05) / (1 - 0.1 - 0.1 - 0.05)))
        assert probe(bo, KRG, 200.0, 0.2, sg, 1)[0] == pytest.approx(se ** 2, abs=1e-15)


def test_pvt_table_nodes_and_linearity(bo):
    fl = bo["fluid"]
    for k, p in enumerate(fl["pvt_p"]):
        assert probe(bo, BO, p, 0.2, 0.1, 1)[0] == pytest.approx(fl["pvt_bo"][k], rel=1e-14)
        assert probe(bo, RS, p, 0.2, 0.1, 1)[0] == pytest.approx(fl["pvt_rs"][k], rel=1e-14)
        assert probe(bo, MUO, p, 0.2, 0.1, 1)[0] == pytest.approx(fl["pvt_muo"][k], rel=1e-14)
        assert probe(bo, RHO_G, p, 0.2, 0.1, 1)[0] == pytest.approx(0.9 / fl["pvt_bg"][k], rel=1e-14)
    # midway between nodes the table is the mean of the neighbours
    bg_mid = 0.5 * (fl["pvt_bg"][2] + fl["pvt_bg"][3])
    assert probe(bo, RHO_G, 175.0, 0.2, 0.1, 1)[0] == pytest.approx(0.9 / bg_mid, rel=1e-14)


def test_undersaturated_oil(bo):
    # undersaturated: Rs frozen at Rs(pb), Bo and mu_o follow the linear undersaturated laws
    pb, p = 150.0, 230.0
    bo_sat = 1.0 + 0.0015 * pb
    mu_sat = 1.5 - 0.0025 * (pb - 50.0)
    assert probe(bo, RS, p, 0.2, pb, 0)[0] == pytest.approx(0.5 * pb, rel=1e-14)
    assert probe(bo, BO, p, 0.2, pb, 0)[0] == pytest.approx(bo_sat * (1 - 1e-4 * (p - pb)), rel=1e-14)
    assert probe(bo, MUO, p, 0.2, pb, 0)[0] == pytest.approx(mu_sat * (1 + 5e-4 * (p - pb)), rel=1e-14)
    # at p = pb the undersaturated and saturated branches meet
    for what in (BO, RS, MUO):
        assert probe(bo, what, pb, 0.2, pb, 0)[0] == pytest.approx(probe(bo, what, pb, 0.2, 0.0, 1)[0], rel=1e-14)


def test_component_content_adds_up(bo):
    # saturated cell: oil + gas content per pore volume from Bo, Rs, Bg by hand
    p, sw, sg = 180.0, 0.3, 0.2
    bo_ = 1.0 + 0.0015 * p
    rs = 0.5 * p
    bg = 1.2 / 150.0 + (1.2 / 200.0 - 1.2 / 150.0) * (p - 150.0) / 50.0
    so = 1 - sw - sg
    phi = 1.0 + 5e-5 * (p - 200.0)   # porosity factor for unit pore volume and unit bulk volume
    assert probe(bo, ACC_O, p, sw, sg, 1)[0] == pytest.approx(phi * 800.0 * so / bo_, rel=1e-13)
    assert probe(bo, ACC_G, p, sw, sg, 1)[0] == pytest.approx(phi * 0.9 * (rs * so / bo_ + sg / bg), rel=1e-13)
    assert probe(bo, ACC_W, p, sw, sg, 1)[0] == pytest.approx(phi * 1000.0 * sw * (1 + 4e-5 * (p - 200.0)), rel=1e-13)


@pytest.mark.parametrize("what", [KRO, RHO_O, MOB_OO, MOB_OG, MOB_GG, ACC_O, ACC_G, ACC_W, LAMT])
@pytest.mark.parametrize("state", [(215.0, 0.31, 0.17, 1), (240.0, 0.42, 170.0, 0)])
def test_property_derivatives_central_difference(bo, what, state):
    p, sw, x3, ph = state
    v, g = probe(bo, what, p, sw, x3, ph)
    x = np.array([p, sw, x3])
    for k in range(3):
        h = 1e-6 * max(1.0, abs(x[k]))
        xp = x.copy(); xp[k] += h
        xm = x.copy(); xm[k] -= h
        fd = (probe(bo, what, *xp, ph)[0] - probe(bo, what, *xm, ph)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-9 * max(1.0, abs(v)))
