"""Pins of the oracle's BiCGSTAB solver and inexact-Newton forcing terms
(Algorithm 1, Eq. 14; the paper's experiments use BiCGSTAB, Sec. 4).

* the first k iterates of unpreconditioned and block-Jacobi-preconditioned
  BiCGSTAB equal scipy's BiCGSTAB iterates (the same recurrence, written
  independently), before any convergence test can intervene;
* with an exact preconditioner (one cell: CPR is J^-1) BiCGSTAB stops after
  one iteration with x = J^-1 b;
* BiCGSTAB + CPR (any decoupling / stage count) solves to the LAPACK
  solution;
* the forcing terms satisfy the defining inequality of Algorithm 1's inexact solve (Eq. 13),
  theta_0 = theta_max, safeguards lin_tol <= theta <= theta_max, and at the
  first adaptive iteration choice 2 <= choice 1 (triangle inequality:
  | ||b|| - ||r|| | <= ||b - r||) on identical histories.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_1606_00548_gb300 import synth
from helpers import dense_from_blocks, random_state


def _assembled(case, dt, seed=0, **solver):
    import oracle
    o = oracle.Oracle(case, **solver)
    if seed is not None:
        x, ph = random_state(case, seed, o.N, o.b)
        o.set_iterate(x, ph)
    o.assemble(dt)
    return o


CASES = [("ow", synth.oil_water_case(nx=4, ny=3, nz=3, sigma=1.0, seed=61), 1.0),
         ("bo", synth.black_oil_case(nx=3, ny=4, nz=2, seed=62), 10.0)]


def _scipy_iterate(A, b, k, M=None):
    x, _ = spla.bicgstab(A, b, x0=np.zeros_like(b), rtol=1e-300, atol=0.0, maxiter=k, M=M)
    return x


@pytest.mark.parametrize("name,case,dt", CASES)
@pytest.mark.parametrize("precond", [0, 1])
def test_iterates_equal_scipy_bicgstab(oracle_lib, name, case, dt, precond):
    # rounding differences grow geometrically with k on these ill-conditioned
    # systems (cond up to 1.5e7); three iterations exercise alpha, omega and beta
    for k in (1, 2, 3):
        o = _assembled(case, dt, krylov=1, precond=precond, lin_tol=1e-300, lin_max_iter=k)
        J = o.jacobian()
        A = dense_from_blocks(J, case["nx"], case["ny"], case["nz"])
        b = -o.residual()
        x, info = o.linear_solve(b)
        assert info.iterations == k and not info.converged and info.restarts == 0
        M = None
        if precond == 1:
            Dinv = np.linalg.inv(J[:, 0])
            N, nb = J.shape[0], J.shape[2]
            M = spla.LinearOperator(A.shape, matvec=lambda v: np.einsum("irc,ic->ir", Dinv, v.reshape(N, nb)).ravel())
        xs = _scipy_iterate(A, b, k, M)
        assert np.abs(x - xs).max() <= 1e-11 * np.abs(xs).max(), k


def test_exact_preconditioner_converges_in_one_iteration(oracle_lib):
    case = synth.black_oil_case(nx=1, ny=1, nz=1, seed=63, wells=[synth.well(0, 0, 0, 0, 0, 180.0)])
    o = _assembled(case, 10.0, krylov=1, lin_tol=1e-12)
    J = o.jacobian()
    b = -o.residual()
    x, info = o.linear_solve(b)
    assert info.converged and info.iterations == 1
    xe = np.linalg.solve(J[0, 0], b)
    assert np.abs(x - xe).max() <= 1e-12 * np.abs(xe).max()


@pytest.mark.parametrize("name,case,dt", CASES)
@pytest.mark.parametrize("decouple,stages,stage2", [(0, 2, 1), (1, 2, 1), (0, 3, 0), (1, 3, 1)])
def test_bicgstab_cpr_matches_dense_solve(oracle_lib, name, case, dt, decouple, stages, stage2):
    o = _assembled(case, dt, krylov=1, lin_tol=1e-12, decouple=decouple, cpr_stages=stages, stage2=stage2)
    A = dense_from_blocks(o.jacobian(), case["nx"], case["ny"], case["nz"])
    b = -o.residual()
    x, info = o.linear_solve(b)
    assert info.converged and info.r_norm <= 1e-12 * info.b_norm
    xe = np.linalg.solve(A, b)
    assert np.abs(x - xe).max() <= 1e-8 * np.abs(xe).max()


def _newton(case, dt, **solver):
    import oracle
    o = oracle.Oracle(case, **solver)
    rc, info = o.newton_solve(dt)
    return o, rc, info


@pytest.mark.parametrize("forcing", [1, 2, 3])
@pytest.mark.parametrize("krylov", [0, 1])
def test_forcing_terms(oracle_lib, forcing, krylov):
    case = synth.black_oil_case(nx=8, ny=7, nz=3, seed=64)
    o, rc, info = _newton(case, 1.0, forcing=forcing, krylov=krylov)
    assert rc == 0 and info.converged
    th, bn, rn = o.forcing_history()
    assert len(th) == info.newton_iterations >= 2
    assert th[0] == 0.5                                   # theta_max on the first iteration
    assert (th >= 1e-8).all() and (th <= 0.5).all()
    assert (rn <= th * bn * (1 + 1e-12)).all()           # ||b - A dx|| <= theta ||b|| (Eq. 13)
    # adaptive: looser than the fixed 1e-8 somewhere, and fewer linear iterations overall
    o2, rc2, info2 = _newton(case, 1.0, forcing=0, krylov=krylov)
    assert rc2 == 0 and info.linear_iterations < info2.linear_iterations
    # both end at CNV <= 1e-10: the same solution
    (x1, ph1), (x2, ph2) = o.get_iterate(), o2.get_iterate()
    x1, x2 = x1.reshape(o.N, o.b), x2.reshape(o.N, o.b)
    assert np.array_equal(ph1, ph2)
    assert np.abs(x1[:, 0] - x2[:, 0]).max() <= 1e-6 * np.abs(x2[:, 0]).max()
    assert np.abs(x1[:, 1] - x2[:, 1]).max() <= 1e-6


def test_choice2_not_above_choice1(oracle_lib):
    case = synth.black_oil_case(nx=8, ny=7, nz=3, seed=64)
    o1, _, _ = _newton(case, 1.0, forcing=1)
    o2, _, _ = _newton(case, 1.0, forcing=2)
    t1, b1, r1 = o1.forcing_history()
    t2, b2, r2 = o2.forcing_history()
    # identical first iteration (theta_max), hence identical b^1, r^0
    assert t1[0] == t2[0] and b1[0] == b2[0] and b1[1] == b2[1] and r1[0] == r2[0]
    assert t2[1] <= t1[1]
