"""Pins of the oracle's linear solver (Sec. 2.4.2) against mathematics.

* the CPR-preconditioned FGMRES solution equals a dense LAPACK solve;
* every preconditioner choice gives the same solution (preconditioning
  changes the path, not the answer);
* unrestarted GMRES on n <= m unknowns terminates within n iterations;
* the pairwise matching equals the sequential greedy matching on the same
  total order of edges (the handshake fixed point), brute force on small
  graphs;
* each coarse AMG operator is the Galerkin product P^T A P, and every
  member of an aggregate is coupled to another member;
* quasi-IMPES decoupling removes the saturation columns of the pressure
  row of every diagonal block;
* red-black block ILU(0): (D + L) D^-1 (D + U) reproduces the decoupled
  matrix on its 7-point block pattern (the defining property of ILU(0));
* ABF decoupling (Sec. 3.2): the scaled diagonal block D_ii^-1 J_ii is the
  identity, so the pressure row of every decoupled diagonal block is e_0;
* CPR-FPF: the three-stage operator is the composition
  z = x0 + M_2 (r - J x0), x0 = stage F of L r, where M_2 is the two-stage
  operator on the same hierarchy (every stage is linear in its input);
* stage P with m V-cycles works on the residual the previous cycles leave:
  the applications' successive differences shrink geometrically.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1606_00548_gb300 import synth
from helpers import dense_from_blocks, neighbour, random_state


def tiny_cases():
    return [("ow", synth.oil_water_case(nx=4, ny=4, nz=3, sigma=1.0, seed=21), 1.0),
            ("bo", synth.black_oil_case(nx=4, ny=4, nz=3, seed=22), 10.0)]


def assembled(case, dt, seed=0, **solver):
    import oracle
    o = oracle.Oracle(case, **solver)
    x, ph = random_state(case, seed, o.N, o.b)
    o.set_iterate(x, ph)
    o.assemble(dt)
    return o


@pytest.mark.parametrize("name,case,dt", tiny_cases())
@pytest.mark.parametrize("orth", [0, 1])
def test_fgmres_cpr_matches_dense_solve(oracle_lib, name, case, dt, orth):
    """CGS2 and the selective second Gram-Schmidt pass both solve to LAPACK's answer."""
    o = assembled(case, dt, lin_tol=1e-12, orth=orth)
    A = dense_from_blocks(o.jacobian(), case["nx"], case["ny"], case["nz"])
    b = -o.residual()
    x, info = o.linear_solve(b)
    assert info.converged
    xe = np.linalg.solve(A, b)
    assert np.abs(x - xe).max() <= 1e-9 * np.abs(xe).max()


@pytest.mark.parametrize("name,case,dt", [
    ("ow", synth.oil_water_case(nx=3, ny=3, nz=3, sigma=1.0, seed=23), 1.0),
    ("bo", synth.black_oil_case(nx=3, ny=3, nz=2, seed=24), 10.0)])
def test_preconditioners_give_same_solution(oracle_lib, name, case, dt):
    sols, its = [], []
    for pc, st, dec, stg in [(0, 0, 0, 2), (1, 0, 0, 2), (2, 0, 0, 2), (2, 1, 0, 2), (2, 1, 1, 2), (2, 1, 0, 3),
                             (2, 0, 1, 3), (2, 2, 0, 2), (2, 2, 1, 3)]:
        # m >= n: unrestarted, so even the unpreconditioned solve terminates
        o = assembled(case, dt, lin_tol=1e-11, precond=pc, stage2=st, decouple=dec, cpr_stages=stg, gmres_m=60,
                      gmres_max_restarts=3)
        x, info = o.linear_solve(-o.residual())
        assert info.converged
        sols.append(x); its.append(info.iterations)
    for x in sols[1:]:
        assert np.abs(x - sols[0]).max() <= 1e-8 * np.abs(sols[0]).max()
    # CPR needs far fewer iterations than no preconditioning
    assert its[3] < its[0]


def test_unrestarted_gmres_terminates_in_n_steps(oracle_lib):
    case = synth.oil_water_case(nx=3, ny=2, nz=2, sigma=1.0, seed=5)
    o = assembled(case, 1.0, precond=0, lin_tol=1e-13, gmres_m=30, gmres_max_restarts=0)
    n = o.N * o.b
    assert n <= 30
    x, info = o.linear_solve(-o.residual())
    assert info.iterations <= n
    A = dense_from_blocks(o.jacobian(), 3, 2, 2)
    xe = np.linalg.solve(A, -o.residual())
    assert np.abs(x - xe).max() <= 1e-7 * np.abs(xe).max()


def test_dense_lu_matches_lapack(oracle_lib):
    import oracle
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 40)); b = rng.standard_normal(40)
    rc, x = oracle.dense_lu_solve(A, b)
    assert rc == 0
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-11, atol=1e-11)


def _edge_hash(a, b):
    lo, hi = min(a, b), max(a, b)
    m = (1 << 64) - 1
    z = (((hi << 32) | lo) + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def _band(a):
    return int(np.float64(a).view(np.uint64) >> np.uint64(52)) & 0x7FF


def greedy_matching(n, edges):
    """Sequential greedy: take edges by decreasing (band, hash), skip used nodes."""
    order = sorted(edges, key=lambda e: (_band(e[2]), _edge_hash(e[0], e[1])), reverse=True)
    partner = [-1] * n
    for i, j, _ in order:
        if partner[i] < 0 and partner[j] < 0:
            partner[i] = j; partner[j] = i
    return partner


@pytest.mark.parametrize("seed", range(6))
def test_matching_equals_greedy_fixed_point(oracle_lib, seed):
    import oracle
    rng = np.random.default_rng(seed)
    n = 40
    # symmetric M-matrix on a random graph: chain + random chords, couplings over many octaves
    edges = {}
    for i in range(n - 1):
        edges[(i, i + 1)] = 10 ** rng.uniform(-1, 2)
    for _ in range(30):
        i, j = sorted(rng.choice(n, 2, replace=False))
        edges[(int(i), int(j))] = 10 ** rng.uniform(-1, 2)
    if seed % 2 == 0:        # many exact ties: hash decides
        for k in edges:
            edges[k] = 1.0
    A = np.zeros((n, n))
    for (i, j), w in edges.items():
        A[i, j] = A[j, i] = -w
    A[np.arange(n), np.arange(n)] = -A.sum(1) + 1.0
    M = sp.csr_matrix(A); M.sort_indices()
    partner, rounds = oracle.match_pass(M.indptr, M.indices, M.data, theta=0.0, rounds=1000)
    expect = greedy_matching(n, [(i, j, w) for (i, j), w in edges.items()])
    assert list(partner) == expect
    # valid matching along existing edges
    for i, p in enumerate(partner):
        if p >= 0:
            assert partner[p] == i and A[i, p] < 0


def test_matching_1d_laplacian_pairs(oracle_lib):
    import oracle
    n = 64
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    partner, _ = oracle.match_pass(A.indptr, A.indices, A.data, theta=0.25, rounds=1000)
    # maximal matching on a path: no two adjacent singletons
    for i in range(n - 1):
        assert not (partner[i] < 0 and partner[i + 1] < 0)
    assert (partner >= 0).mean() > 0.6


@pytest.mark.parametrize("name,case,dt", [
    ("ow", synth.oil_water_case(nx=12, ny=10, nz=4, sigma=1.0, seed=31), 1.0),
    ("bo", synth.black_oil_case(nx=14, ny=12, nz=4, seed=32), 10.0)])
def test_amg_galerkin_and_qi(oracle_lib, name, case, dt):
    o = assembled(case, dt, amg_coarse_max=16)
    o.precond_setup()
    levels = o.amg_levels()
    assert len(levels) >= 3
    for l in range(len(levels) - 1):
        L, Cl = levels[l], levels[l + 1]
        A = sp.csr_matrix((L["val"], L["col"], L["rowptr"]), shape=(L["n"], L["n"]))
        P = sp.csr_matrix((np.ones(L["n"]), (np.arange(L["n"]), L["agg"])), shape=(L["n"], Cl["n"]))
        Ac = (P.T @ A @ P).toarray()
        Cm = sp.csr_matrix((Cl["val"], Cl["col"], Cl["rowptr"]), shape=(Cl["n"], Cl["n"])).toarray()
        assert np.abs(Ac - Cm).max() <= 1e-12 * np.abs(Ac).max()
        sizes = np.bincount(L["agg"], minlength=Cl["n"])
        assert sizes.min() >= 1
        # every member of a multi-node aggregate couples (negatively) to another member
        Ad = A.toarray()
        for I in np.nonzero(sizes > 1)[0]:
            mem = np.nonzero(L["agg"] == I)[0]
            sub = Ad[np.ix_(mem, mem)] - np.diag(np.diag(Ad[np.ix_(mem, mem)]))
            assert ((sub < 0).any(axis=1)).all()
    # quasi-IMPES: pressure row of each decoupled diagonal block has no saturation columns
    J = o.jacobian()
    w, ap = o.qi()
    w = w.reshape(o.N, o.b)
    D = J[:, 0]
    row = np.einsum("ir,irc->ic", w, D)
    assert np.abs(row[:, 1:]).max() <= 1e-10 * np.abs(D).max()
    assert np.allclose(ap[:, 0], row[:, 0], rtol=1e-14)


@pytest.mark.parametrize("name,case,dt", tiny_cases())
def test_red_black_ilu0_reproduces_pattern(oracle_lib, name, case, dt):
    o = assembled(case, dt, stage2=1)
    o.precond_setup()
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    N, b = o.N, o.b
    J = o.jacobian()
    w, _ = o.qi(); w = w.reshape(N, b)
    # decoupled blocks: pressure row replaced by the weighted row combination
    Ah = J.copy()
    Ah[:, :, 0, :] = np.einsum("ir,idrc->idc", w, J)
    dinv = o.ilu_dinv()
    color = np.array([(i % nx + (i // nx) % ny + i // (nx * ny)) & 1 for i in range(N)])
    D = np.zeros((N * b, N * b)); Lm = np.zeros_like(D); Um = np.zeros_like(D); Di = np.zeros_like(D)
    pattern = np.zeros((N, N), bool)
    for i in range(N):
        sl = slice(i * b, (i + 1) * b)
        D[sl, sl] = np.linalg.inv(dinv[i]); Di[sl, sl] = dinv[i]
        for d in range(7):
            j = neighbour(nx, ny, nz, i, d)
            if j < 0:
                continue
            pattern[i, j] = True
            if d == 0:
                continue
            if color[i] == 1 and color[j] == 0:
                Lm[sl, j * b:(j + 1) * b] = Ah[i, d]
            if color[i] == 0 and color[j] == 1:
                Um[sl, j * b:(j + 1) * b] = Ah[i, d]
    M = (D + Lm) @ Di @ (D + Um)
    Ad = dense_from_blocks(Ah, nx, ny, nz)
    mask = np.kron(pattern, np.ones((b, b), bool))
    assert np.abs((M - Ad)[mask]).max() <= 1e-10 * np.abs(Ad).max()


@pytest.mark.parametrize("name,case,dt", tiny_cases())
def test_abf_scaled_diagonal_is_identity(oracle_lib, name, case, dt):
    o = assembled(case, dt, decouple=1)
    o.precond_setup()
    J = o.jacobian()
    w, ap = o.qi()
    w = w.reshape(o.N, o.b)
    # first row of D_ii^-1 times D_ii is e_0 (the inverse computed by cofactors)
    row = np.einsum("ir,irc->ic", w, J[:, 0])
    e0 = np.zeros(o.b); e0[0] = 1.0
    assert np.abs(row - e0).max() <= 1e-12
    assert np.abs(ap[:, 0] - 1.0).max() <= 1e-12
    # and the row is the first row of the true inverse
    assert np.allclose(w, np.linalg.inv(J[:, 0])[:, 0, :], rtol=1e-12, atol=0)


@pytest.mark.parametrize("name,case,dt", tiny_cases())
@pytest.mark.parametrize("decouple", [0, 1])
def test_fpf_is_the_composition_of_its_stages(oracle_lib, name, case, dt, decouple):
    """Block-Jacobi stage F: x0 = (L J_ii)^-1 L r = J_ii^-1 r, for either L."""
    o2 = assembled(case, dt, decouple=decouple, cpr_stages=2, stage2=0)
    o3 = assembled(case, dt, decouple=decouple, cpr_stages=3, stage2=0)
    N, b = o2.N, o2.b
    J = o2.jacobian()
    A = dense_from_blocks(J, case["nx"], case["ny"], case["nz"])
    r = np.random.default_rng(7).standard_normal(N * b)
    x0 = np.linalg.solve(J[:, 0], r.reshape(N, b)[:, :, None])[:, :, 0].reshape(-1)
    z3 = o3.precond_apply(r)
    zc = x0 + o2.precond_apply(r - A @ x0)
    assert np.abs(z3 - zc).max() <= 1e-10 * np.abs(zc).max()
    # and it differs from the two-stage operator (the first stage does something)
    assert np.abs(z3 - o2.precond_apply(r)).max() > 1e-6 * np.abs(zc).max()


@pytest.mark.parametrize("name,case,dt", tiny_cases())
def test_natural_ilu0_reproduces_pattern(oracle_lib, name, case, dt):
    """Natural-order block ILU(0) (the ordering study of the second stage):
    (D + L) D^-1 (D + U) equals the decoupled matrix on the 7-point pattern,
    with L / U the blocks of the lower (-x, -y, -z) / upper neighbours, and
    its application solves with that product."""
    o = assembled(case, dt, stage2=2)
    o.precond_setup()
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    N, b = o.N, o.b
    J = o.jacobian()
    w, _ = o.qi(); w = w.reshape(N, b)
    Ah = J.copy()
    Ah[:, :, 0, :] = np.einsum("ir,idrc->idc", w, J)
    dinv = o.ilu_dinv()
    D = np.zeros((N * b, N * b)); Lm = np.zeros_like(D); Um = np.zeros_like(D); Di = np.zeros_like(D)
    pattern = np.zeros((N, N), bool)
    for i in range(N):
        sl = slice(i * b, (i + 1) * b)
        D[sl, sl] = np.linalg.inv(dinv[i]); Di[sl, sl] = dinv[i]
        for d in range(7):
            j = neighbour(nx, ny, nz, i, d)
            if j < 0:
                continue
            pattern[i, j] = True
            if d in (1, 3, 5):
                Lm[sl, j * b:(j + 1) * b] = Ah[i, d]
            elif d in (2, 4, 6):
                Um[sl, j * b:(j + 1) * b] = Ah[i, d]
    M = (D + Lm) @ Di @ (D + Um)
    Ad = dense_from_blocks(Ah, nx, ny, nz)
    mask = np.kron(pattern, np.ones((b, b), bool))
    assert np.abs((M - Ad)[mask]).max() <= 1e-10 * np.abs(Ad).max()
    # the factors are lower / upper in the natural order
    assert not np.tril(Um).any() and not np.triu(Lm).any()


@pytest.mark.parametrize("name,case,dt", [
    ("ow", synth.oil_water_case(nx=10, ny=8, nz=4, sigma=1.0, seed=23), 1.0),
    ("bo", synth.black_oil_case(nx=10, ny=8, nz=4, seed=24), 10.0)])
def test_stage_p_cycles_work_on_the_residual_they_leave(oracle_lib, name, case, dt):
    """Stage P with m V-cycles: e_{m+1} = e_m + V(f - A_p e_m).  The CPR
    application is affine in e, so the differences z_{m+1} - z_m = K E^m V f
    (E = I - V A_p) shrink geometrically at the V-cycle's contraction rate
    toward the application with the exact pressure solve.  A later cycle on the
    original f would give equal differences, a sign error in the residual
    growing ones.  Initial state of a physical system; hierarchy of 3 levels."""
    import oracle
    r = np.random.default_rng(9).standard_normal(case["nx"] * case["ny"] * case["nz"] * (2 if case["model"] == 2 else 3))
    zs = []
    for m in range(1, 8):
        o = oracle.Oracle(case, amg_cycles=m, amg_coarse_max=16)
        o.assemble(dt)
        zs.append(o.precond_apply(r))
        if m == 1:
            assert len(o.amg_levels()) >= 3
    d = np.array([np.linalg.norm(zs[k + 1] - zs[k]) for k in range(len(zs) - 1)])
    assert d[0] > 1e-6 * np.linalg.norm(zs[0])          # the second cycle does something
    ratios = d[1:] / d[:-1]
    assert np.all(ratios > 0.2) and np.all(ratios < 0.85), ratios
