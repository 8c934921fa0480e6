"""Pin: the oracle's analytic Jacobian equals central finite differences of its
residual (Eq. 10-11 discretisation of Eq. 3/5 with the well terms of Eq. 6).

States are random and physical, away from the kinks of the upwind switch and
the relative-permeability clipping; both black-oil phase states are present.
"""
import numpy as np
import pytest

from paper_1606_00548_gb300 import synth
from helpers import dense_from_blocks, random_state


def fd_max_rel_error(case, dt, seed):
    import oracle
    o = oracle.Oracle(case)
    N, b = o.N, o.b
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    x, ph = random_state(case, seed, N, b)
    o.set_iterate(x, ph); o.assemble(dt)
    A = dense_from_blocks(o.jacobian(), nx, ny, nz)
    worst = 0.0
    for k in range(N * b):
        h = 1e-6 * max(1.0, abs(x[k]))
        xp = x.copy(); xp[k] += h
        o.set_iterate(xp, ph); o.assemble(dt); rp = o.residual()
        xm = x.copy(); xm[k] -= h
        o.set_iterate(xm, ph); o.assemble(dt); rm = o.residual()
        col = (rp - rm) / (2 * h)
        scale = np.abs(col).max() + np.abs(A[:, k]).max() + 1e-300
        worst = max(worst, np.abs(A[:, k] - col).max() / scale)
    return worst


@pytest.mark.parametrize("seed", [0, 1])
def test_jacobian_fd_oil_water(oracle_lib, seed):
    case = synth.oil_water_case(nx=4, ny=3, nz=3, sigma=1.0, seed=7 + seed)
    assert fd_max_rel_error(case, 1.0, seed) < 1e-5


@pytest.mark.parametrize("seed", [0, 1])
def test_jacobian_fd_black_oil(oracle_lib, seed):
    case = synth.black_oil_case(nx=4, ny=3, nz=3, seed=11 + seed)
    assert fd_max_rel_error(case, 10.0, seed) < 1e-5


def test_fluxes_conserve_mass(oracle_lib):
    """Inter-cell fluxes cancel in the sum of residuals: sum_i R_i dt equals the
    change of component mass minus the well rates times dt (exactly, up to rounding)."""
    import oracle
    case = synth.black_oil_case(nx=5, ny=4, nz=3, seed=3)
    o = oracle.Oracle(case)
    N, b = o.N, o.b
    m0 = o.component_mass()
    x, ph = random_state(case, 5, N, b)
    o.set_iterate(x, ph)
    dt = 10.0
    o.assemble(dt)
    R = o.residual().reshape(N, b).sum(0)
    m1 = o.component_mass()
    q = o.well_rates()
    for c in range(3):
        expect = (m1[c] - m0[c]) / dt - q[c]
        assert R[c] == pytest.approx(expect, rel=1e-9, abs=1e-9 * abs(m1[c]) / dt)
