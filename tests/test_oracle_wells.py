"""Pins of the oracle's well controls (Sec. 2.3, Eq. 6-9) and their place in
the Newton system (Eq. 16).

* the bordered Jacobian [[A, A_pw], [A_wp, A_ww]] of cells + well BHP
  unknowns equals central finite differences of (R, R_w), both well types,
  both controls, both black-oil phase states;
* the oracle's reduced operator S (wells eliminated) solves the bordered
  system: its Krylov solution equals LAPACK's on the full bordered matrix,
  and S x equals the bordered product with the well unknowns eliminated;
* control equivalence: a well under rate control with the target set to the
  rate it had under BHP control ends the step at that BHP and at the same
  cell state (both controls describe one physical solution);
* the converged rate matches the target; the mass balance still closes.
"""
import numpy as np
import pytest

from paper_1606_00548_gb300 import synth
from helpers import dense_from_blocks, random_state


def _case(ctrl_prod=2, ctrl_inj=1, rate_prod=-2.0e4, rate_inj=3.0e4, model=3, seed=71):
    nz = 3
    wells = [synth.well(0, 0, 0, nz - 1, synth.WATER_INJECTOR, 240.0, ctrl=ctrl_inj, rate=rate_inj),
             synth.well(3, 2, 0, nz - 1, synth.PRODUCER, 180.0, ctrl=ctrl_prod, rate=rate_prod),
             synth.well(1, 2, 1, 1, synth.PRODUCER, 190.0)]
    if model == 3:
        return synth.black_oil_case(nx=4, ny=3, nz=nz, seed=seed, wells=wells)
    return synth.oil_water_case(nx=4, ny=3, nz=nz, sigma=1.0, seed=seed, wells=wells)


def _bordered(o, case):
    N, b = o.N, o.b
    A = dense_from_blocks(o.jacobian(), case["nx"], case["ny"], case["nz"])
    Rw, Apw, Awp, Aww = o.well_system()
    nw = len(case["wells"])
    M = np.zeros((N * b + nw, N * b + nw))
    M[:N * b, :N * b] = A
    q = 0
    for w, wl in enumerate(case["wells"]):
        for k in range(wl["k0"], wl["k1"] + 1):
            i = wl["i"] + case["nx"] * (wl["j"] + case["ny"] * k)
            M[i * b:(i + 1) * b, N * b + w] += Apw[q]
            M[N * b + w, i * b:(i + 1) * b] += Awp[q]
            q += 1
    M[N * b:, N * b:] = np.diag(Aww)
    return M, np.concatenate([o.residual(), Rw])


@pytest.mark.parametrize("model,seed", [(3, 0), (3, 1), (2, 2)])
def test_bordered_jacobian_fd(oracle_lib, model, seed):
    import oracle
    case = _case(model=model, seed=71 + seed)
    o = oracle.Oracle(case)
    N, b = o.N, o.b
    x, ph = random_state(case, seed, N, b)
    bhp0 = np.array([235.0, 185.0, 190.0])
    dt = 10.0 if model == 3 else 1.0
    o.set_iterate(x, ph); o.set_well_bhp(bhp0); o.assemble(dt)
    M, _ = _bordered(o, case)
    nw = 3
    worst = 0.0
    for k in range(N * b + nw):
        cols = []
        for sgn in (1, -1):
            xx, pp = x.copy(), bhp0.copy()
            if k < N * b:
                h = 1e-6 * max(1.0, abs(x[k])); xx[k] += sgn * h
            else:
                h = 1e-6 * bhp0[k - N * b]; pp[k - N * b] += sgn * h
            o.set_iterate(xx, ph); o.set_well_bhp(pp); o.assemble(dt)
            Rw = o.well_system()[0]
            cols.append(np.concatenate([o.residual(), Rw]))
        col = (cols[0] - cols[1]) / (2 * h)
        scale = np.abs(col).max() + np.abs(M[:, k]).max() + 1e-300
        worst = max(worst, np.abs(M[:, k] - col).max() / scale)
    assert worst < 1e-5


def test_reduced_operator_solves_the_bordered_system(oracle_lib):
    import oracle
    case = _case()
    o = oracle.Oracle(case, lin_tol=1e-12)
    N, b = o.N, o.b
    x, ph = random_state(case, 3, N, b)
    o.set_iterate(x, ph); o.set_well_bhp([235.0, 185.0, 190.0]); o.assemble(10.0)
    M, _ = _bordered(o, case)
    nb = N * b
    rhs = np.random.default_rng(4).standard_normal(nb)
    full = np.linalg.solve(M, np.concatenate([rhs, np.zeros(3)]))
    xs, info = o.linear_solve(rhs)
    assert info.converged
    assert np.abs(xs - full[:nb]).max() <= 1e-8 * np.abs(full[:nb]).max()
    # S v: the bordered product with the well unknowns chosen to zero the well rows
    v = np.random.default_rng(5).standard_normal(nb)
    u = -np.linalg.solve(M[nb:, nb:], M[nb:, :nb] @ v)
    ref = M[:nb, :nb] @ v + M[:nb, nb:] @ u
    assert np.abs(o.spmv(v) - ref).max() <= 1e-12 * np.abs(ref).max()


def _run_step(case, dt, **kw):
    import oracle
    o = oracle.Oracle(case, **kw)
    rc, info = o.step(dt)
    assert rc == 0 and info.ok
    return o


@pytest.mark.parametrize("model", [3, 2])
def test_rate_control_reproduces_bhp_control(oracle_lib, model):
    """Producer (oil rate) and injector (water rate) under rate control with
    the rates they had under BHP control: same BHPs, same state."""
    dt = 1.0
    base = _case(ctrl_prod=0, ctrl_inj=0, model=model, seed=81)
    base["wells"] = base["wells"][:2]                     # one injector, one producer
    ob = _run_step(base, dt)
    qw = ob.well_component_rates()
    qinj, qprod = qw[0, 0], qw[1, 1]                      # injector's water, producer's oil
    assert qinj > 0 and qprod < 0
    rated = _case(ctrl_prod=2, ctrl_inj=1, rate_prod=qprod, rate_inj=qinj, model=model, seed=81)
    rated["wells"] = rated["wells"][:2]
    # initial guesses away from the answer, the injector's above the
    # reservoir pressure (a rate-controlled injector is meant to inject)
    rated["wells"][0]["bhp"] = 262.0
    rated["wells"][1]["bhp"] = 195.0
    orr = _run_step(rated, dt)
    bhp = orr.well_bhp()
    assert abs(bhp[0] - 240.0) <= 1e-8 * 240.0 and abs(bhp[1] - 180.0) <= 1e-8 * 180.0
    pb, swb, x3b, phb = ob.get_state()
    pr, swr, x3r, phr = orr.get_state()
    assert np.abs(pb - pr).max() <= 1e-6 * np.abs(pb).max()
    assert np.abs(swb - swr).max() <= 1e-7
    assert np.array_equal(phb, phr)
    # the targets are met
    qr = orr.well_component_rates()
    assert qr[0, 0] == pytest.approx(qinj, rel=1e-9) and qr[1, 1] == pytest.approx(qprod, rel=1e-9)
    assert np.abs(qr - qw).max() <= 1e-6 * np.abs(qw).max()


def test_rate_wells_conserve_mass(oracle_lib):
    import oracle
    case = _case(seed=91)
    o = oracle.Oracle(case)
    m0 = o.component_mass()
    for dt in (1.0, 2.0):
        rc, info = o.step(dt)
        assert rc == 0
    m1 = o.component_mass()
    cum = o.cumulative_well_mass()
    for c in range(3):
        assert abs((m1[c] - m0[c]) - cum[c]) <= 1e-9 * abs(m0[c])
