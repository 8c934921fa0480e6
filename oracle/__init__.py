"""ctypes binding to the CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline / reference leg.  The product path (the CUDA
library and its binding) never imports this package.

The oracle keeps its own layouts: vectors interleaved per cell (x[i*b + c]),
Jacobian blocks J[i, d, r, c] with d = centre, -x, +x, -y, +y, -z, +z.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so results do not depend on the host ISA)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class OraInput(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("top_depth", C.c_double),
        ("model", C.c_int32),
        ("kx", _dp), ("ky", _dp), ("kz", _dp), ("poro", _dp),
        ("c_rock", C.c_double), ("p_ref", C.c_double),
        ("rho_w_ref", C.c_double), ("rho_o_ref", C.c_double), ("c_w", C.c_double), ("c_o", C.c_double),
        ("mu_w", C.c_double), ("mu_o", C.c_double),
        ("rho_ws", C.c_double), ("rho_os", C.c_double), ("rho_gs", C.c_double), ("bw_c", C.c_double),
        ("bw_pref", C.c_double), ("bo_c_us", C.c_double), ("muo_c_us", C.c_double),
        ("npvt", C.c_int32),
        ("pvt_p", _dp), ("pvt_bo", _dp), ("pvt_rs", _dp), ("pvt_muo", _dp), ("pvt_bg", _dp), ("pvt_mug", _dp),
        ("swc", C.c_double), ("sor", C.c_double), ("sgc", C.c_double), ("sorg", C.c_double),
        ("nw", C.c_double), ("now", C.c_double), ("ng", C.c_double), ("nog", C.c_double),
        ("nwells", C.c_int32),
        ("w_i", _ip), ("w_j", _ip), ("w_k0", _ip), ("w_k1", _ip), ("w_type", _ip),
        ("w_bhp", _dp), ("w_rw", _dp), ("w_skin", _dp),
        ("cnv_rho", C.c_double * 3),
        ("newton_tol", C.c_double), ("newton_max", C.c_int32),
        ("lin_tol", C.c_double), ("gmres_m", C.c_int32), ("gmres_max_restarts", C.c_int32),
        ("precond", C.c_int32), ("stage2", C.c_int32),
        ("amg_theta", C.c_double), ("amg_rounds", C.c_int32), ("amg_coarse_max", C.c_int32),
        ("amg_max_levels", C.c_int32),
        ("chop_ds", C.c_double), ("chop_dp", C.c_double), ("max_cuts", C.c_int32),
        ("amg_cycles", C.c_int32), ("decouple", C.c_int32), ("cpr_stages", C.c_int32),
        ("krylov", C.c_int32), ("lin_max_iter", C.c_int32), ("forcing", C.c_int32),
        ("ew_gamma", C.c_double), ("ew_beta", C.c_double), ("theta_max", C.c_double),
        ("w_ctrl", C.POINTER(C.c_int32)), ("w_rate", C.POINTER(C.c_double)),
        ("orth", C.c_int32),
    ]


class LinInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("b_norm", C.c_double), ("r_norm", C.c_double)]


class NewtonInfo(C.Structure):
    _fields_ = [("newton_iterations", C.c_int32), ("linear_iterations", C.c_int32),
                ("converged", C.c_int32), ("linear_failures", C.c_int32), ("cnv", C.c_double)]


class StepInfo(C.Structure):
    _fields_ = [("cuts", C.c_int32), ("newton_iterations", C.c_int32), ("linear_iterations", C.c_int32),
                ("substeps", C.c_int32), ("ok", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        vp = C.c_void_p
        L.ora_create.restype = vp
        L.ora_create.argtypes = [C.POINTER(OraInput)]
        for name in ["ora_destroy", "ora_block_size"]:
            getattr(L, name).argtypes = [vp]
        L.ora_block_size.restype = C.c_int
        L.ora_destroy.restype = None
        L.ora_set_state.argtypes = [vp, _dp, _dp, _dp, C.c_void_p]
        L.ora_get_state.argtypes = [vp, _dp, _dp, _dp, C.c_void_p]
        L.ora_set_iterate.argtypes = [vp, _dp, C.c_void_p]
        L.ora_get_iterate.argtypes = [vp, _dp, C.c_void_p]
        L.ora_assemble.argtypes = [vp, C.c_double]
        L.ora_get_residual.argtypes = [vp, _dp]
        L.ora_get_jacobian.argtypes = [vp, _dp]
        L.ora_set_jacobian.argtypes = [vp, _dp]
        L.ora_cnv.argtypes = [vp, C.c_double]; L.ora_cnv.restype = C.c_double
        L.ora_spmv.argtypes = [vp, _dp, _dp]
        L.ora_precond_setup.argtypes = [vp]
        L.ora_precond_apply.argtypes = [vp, _dp, _dp]
        L.ora_linear_solve.argtypes = [vp, _dp, _dp, C.POINTER(LinInfo)]
        L.ora_newton_step.argtypes = [vp, C.c_double, C.POINTER(NewtonInfo)]
        L.ora_newton_solve.argtypes = [vp, C.c_double, C.POINTER(NewtonInfo)]
        L.ora_step.argtypes = [vp, C.c_double, C.POINTER(StepInfo)]
        L.ora_forcing_history.argtypes = [vp, _dp, _dp, _dp, C.c_int]
        L.ora_get_well_bhp.argtypes = [vp, _dp]
        L.ora_set_well_bhp.argtypes = [vp, _dp]
        L.ora_perforations.argtypes = [vp]
        L.ora_get_well_system.argtypes = [vp, _dp, _dp, _dp, _dp]
        L.ora_well_component_rates.argtypes = [vp, _dp]
        L.ora_component_mass.argtypes = [vp, _dp]
        L.ora_cumulative_well_mass.argtypes = [vp, _dp]
        L.ora_well_rates.argtypes = [vp, _dp]
        L.ora_get_qi.argtypes = [vp, _dp, _dp]
        L.ora_amg_levels.argtypes = [vp]
        L.ora_amg_level_n.argtypes = [vp, C.c_int]
        L.ora_amg_level_nnz.argtypes = [vp, C.c_int]
        L.ora_amg_level_csr.argtypes = [vp, C.c_int, _ip, _ip, _dp]
        L.ora_amg_level_agg.argtypes = [vp, C.c_int, _ip]
        L.ora_ilu_dinv.argtypes = [vp, _dp]
        L.ora_dense_lu_solve.argtypes = [C.c_int, _dp, _dp]
        L.ora_match_pass.argtypes = [C.c_int, _ip, _ip, _dp, C.c_double, C.c_int, _ip]
        L.ora_props_probe.argtypes = [C.POINTER(OraInput), C.c_int, C.c_double, C.c_double, C.c_double,
                                      C.c_int, _dp]
        L.ora_props_probe.restype = C.c_double
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def make_input(case: dict, keep: list, **solver_overrides) -> OraInput:
    """Marshal a synth case into the oracle's input struct (arrays kept alive in `keep`)."""
    inp = OraInput()
    inp.nx, inp.ny, inp.nz = case["nx"], case["ny"], case["nz"]
    inp.dx, inp.dy, inp.dz, inp.top_depth = case["dx"], case["dy"], case["dz"], case["top_depth"]
    inp.model = case["model"]
    for name in ("kx", "ky", "kz", "poro"):
        a, p = _d(case[name]); keep.append(a); setattr(inp, name, p)
    inp.c_rock, inp.p_ref = case["c_rock"], case["p_ref"]
    fl = case["fluid"]
    for name in ("rho_w_ref", "rho_o_ref", "c_w", "c_o", "mu_w", "mu_o", "rho_ws", "rho_os", "rho_gs",
                 "bw_c", "bw_pref", "bo_c_us", "muo_c_us", "swc", "sor", "sgc", "sorg", "nw", "now", "ng", "nog"):
        if name in fl:
            setattr(inp, name, float(fl[name]))
    if case["model"] == 3:
        inp.npvt = len(fl["pvt_p"])
        for name in ("pvt_p", "pvt_bo", "pvt_rs", "pvt_muo", "pvt_bg", "pvt_mug"):
            a, p = _d(fl[name]); keep.append(a); setattr(inp, name, p)
    ws = case["wells"]
    inp.nwells = len(ws)
    for name, key in (("w_i", "i"), ("w_j", "j"), ("w_k0", "k0"), ("w_k1", "k1"), ("w_type", "type")):
        a, p = _i([w[key] for w in ws] or [0]); keep.append(a); setattr(inp, name, p)
    for name, key in (("w_bhp", "bhp"), ("w_rw", "rw"), ("w_skin", "skin")):
        a, p = _d([w[key] for w in ws] or [0.0]); keep.append(a); setattr(inp, name, p)
    a, p = _i([w.get("ctrl", 0) for w in ws] or [0]); keep.append(a); inp.w_ctrl = p
    a, p = _d([w.get("rate", 0.0) for w in ws] or [0.0]); keep.append(a); inp.w_rate = p
    for c in range(3):
        inp.cnv_rho[c] = case["cnv_rho"][c]
    sv = dict(case["solver"]); sv.update(solver_overrides)
    for name in ("newton_tol", "lin_tol", "amg_theta", "chop_ds", "chop_dp", "ew_gamma", "ew_beta", "theta_max"):
        setattr(inp, name, float(sv[name]))
    for name in ("newton_max", "gmres_m", "gmres_max_restarts", "precond", "stage2", "amg_rounds",
                 "amg_coarse_max", "amg_max_levels", "max_cuts", "amg_cycles", "decouple", "cpr_stages",
                 "krylov", "lin_max_iter", "forcing", "orth"):
        setattr(inp, name, int(sv[name]))
    return inp


class Oracle:
    """One oracle simulator instance for a synth case."""

    def __init__(self, case: dict, **solver_overrides):
        self.case = case
        self._keep = []
        self.inp = make_input(case, self._keep, **solver_overrides)
        self.L = lib()
        self.h = self.L.ora_create(C.byref(self.inp))
        if not self.h:
            raise ValueError("oracle: invalid input (see stderr)")
        self.N = case["nx"] * case["ny"] * case["nz"]
        self.nwells = len(case["wells"])
        self.b = self.L.ora_block_size(self.h)
        ini = case["init"]
        self.set_state(ini["p"], ini["sw"], ini["x3"], ini["phase"])

    def __del__(self):
        try:
            if self.h:
                self.L.ora_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # state ------------------------------------------------------------------
    def set_state(self, p, sw, x3, phase):
        p, pp = _d(p); sw, sp = _d(sw); x3, xp = _d(x3)
        ph = np.ascontiguousarray(phase, dtype=np.int8)
        self.L.ora_set_state(self.h, pp, sp, xp, ph.ctypes.data_as(C.c_void_p))

    def get_state(self):
        p = np.zeros(self.N); sw = np.zeros(self.N); x3 = np.zeros(self.N); ph = np.zeros(self.N, np.int8)
        self.L.ora_get_state(self.h, p.ctypes.data_as(_dp), sw.ctypes.data_as(_dp), x3.ctypes.data_as(_dp),
                             ph.ctypes.data_as(C.c_void_p))
        return p, sw, x3, ph

    def set_iterate(self, x, phase):
        x, xp = _d(x)
        ph = np.ascontiguousarray(phase, dtype=np.int8)
        self.L.ora_set_iterate(self.h, xp, ph.ctypes.data_as(C.c_void_p))

    def get_iterate(self):
        x = np.zeros(self.N * self.b); ph = np.zeros(self.N, np.int8)
        self.L.ora_get_iterate(self.h, x.ctypes.data_as(_dp), ph.ctypes.data_as(C.c_void_p))
        return x, ph

    # assembly ---------------------------------------------------------------
    def assemble(self, dt):
        self.L.ora_assemble(self.h, float(dt))

    def residual(self):
        R = np.zeros(self.N * self.b)
        self.L.ora_get_residual(self.h, R.ctypes.data_as(_dp))
        return R

    def jacobian(self):
        J = np.zeros((self.N, 7, self.b, self.b))
        self.L.ora_get_jacobian(self.h, J.ctypes.data_as(_dp))
        return J

    def set_jacobian(self, J):
        J, jp = _d(J)
        self.L.ora_set_jacobian(self.h, jp)

    def cnv(self, dt):
        return self.L.ora_cnv(self.h, float(dt))

    # linear algebra -----------------------------------------------------------
    def spmv(self, x):
        x, xp = _d(x); y = np.zeros_like(x)
        self.L.ora_spmv(self.h, xp, y.ctypes.data_as(_dp))
        return y

    def precond_setup(self):
        self.L.ora_precond_setup(self.h)

    def precond_apply(self, r):
        r, rp = _d(r); z = np.zeros_like(r)
        self.L.ora_precond_apply(self.h, rp, z.ctypes.data_as(_dp))
        return z

    def linear_solve(self, bvec):
        b, bp = _d(bvec); x = np.zeros_like(b); info = LinInfo()
        self.L.ora_linear_solve(self.h, bp, x.ctypes.data_as(_dp), C.byref(info))
        return x, info

    def qi(self):
        w = np.zeros(self.N * self.b); ap = np.zeros((self.N, 7))
        self.L.ora_get_qi(self.h, w.ctypes.data_as(_dp), ap.ctypes.data_as(_dp))
        return w, ap

    def amg_levels(self):
        out = []
        for l in range(self.L.ora_amg_levels(self.h)):
            n = self.L.ora_amg_level_n(self.h, l); nnz = self.L.ora_amg_level_nnz(self.h, l)
            rp = np.zeros(n + 1, np.int32); col = np.zeros(nnz, np.int32); val = np.zeros(nnz)
            self.L.ora_amg_level_csr(self.h, l, rp.ctypes.data_as(_ip), col.ctypes.data_as(_ip),
                                     val.ctypes.data_as(_dp))
            agg = np.full(n, -1, np.int32)
            self.L.ora_amg_level_agg(self.h, l, agg.ctypes.data_as(_ip))
            out.append(dict(n=n, rowptr=rp, col=col, val=val, agg=agg))
        return out

    def ilu_dinv(self):
        d = np.zeros((self.N, self.b, self.b))
        self.L.ora_ilu_dinv(self.h, d.ctypes.data_as(_dp))
        return d

    # nonlinear ----------------------------------------------------------------
    def newton_step(self, dt):
        info = NewtonInfo()
        rc = self.L.ora_newton_step(self.h, float(dt), C.byref(info))
        return rc, info

    def newton_solve(self, dt):
        info = NewtonInfo()
        rc = self.L.ora_newton_solve(self.h, float(dt), C.byref(info))
        return rc, info

    def well_bhp(self):
        p = np.zeros(max(self.nwells, 1))
        self.L.ora_get_well_bhp(self.h, p.ctypes.data_as(_dp))
        return p[:self.nwells]

    def set_well_bhp(self, bhp):
        a, p = _d(np.asarray(bhp, dtype=np.float64).reshape(-1) if self.nwells else [0.0])
        self.L.ora_set_well_bhp(self.h, p)

    def well_component_rates(self):
        q = np.zeros(3 * max(self.nwells, 1))
        self.L.ora_well_component_rates(self.h, q.ctypes.data_as(_dp))
        return q[:3 * self.nwells].reshape(self.nwells, 3)

    def well_system(self):
        """R_w, A_pw [nperf, b], A_wp [nperf, b], A_ww of the last assembly."""
        nw, npf = max(self.nwells, 1), max(self.L.ora_perforations(self.h), 1)
        Rw, Aww = np.zeros(nw), np.zeros(nw)
        Apw, Awp = np.zeros(npf * self.b), np.zeros(npf * self.b)
        self.L.ora_get_well_system(self.h, Rw.ctypes.data_as(_dp), Apw.ctypes.data_as(_dp),
                                   Awp.ctypes.data_as(_dp), Aww.ctypes.data_as(_dp))
        npf = self.L.ora_perforations(self.h)
        return (Rw[:self.nwells], Apw[:npf * self.b].reshape(npf, self.b), Awp[:npf * self.b].reshape(npf, self.b),
                Aww[:self.nwells])

    def forcing_history(self):
        th, bn, rn = np.zeros(64), np.zeros(64), np.zeros(64)
        k = self.L.ora_forcing_history(self.h, th.ctypes.data_as(_dp), bn.ctypes.data_as(_dp),
                                       rn.ctypes.data_as(_dp), 64)
        return th[:k], bn[:k], rn[:k]

    def step(self, dt):
        info = StepInfo()
        rc = self.L.ora_step(self.h, float(dt), C.byref(info))
        return rc, info

    def component_mass(self):
        m = np.zeros(3); self.L.ora_component_mass(self.h, m.ctypes.data_as(_dp)); return m

    def cumulative_well_mass(self):
        m = np.zeros(3); self.L.ora_cumulative_well_mass(self.h, m.ctypes.data_as(_dp)); return m

    def well_rates(self):
        q = np.zeros(3); self.L.ora_well_rates(self.h, q.ctypes.data_as(_dp)); return q


def props_probe(case: dict, what: int, p: float, sw: float, x3: float, ph: int):
    keep = []
    inp = make_input(case, keep)
    g = np.zeros(3)
    v = lib().ora_props_probe(C.byref(inp), what, p, sw, x3, ph, g.ctypes.data_as(_dp))
    return v, g


def dense_lu_solve(A, b):
    A = np.array(A, dtype=np.float64, order="C"); x = np.array(b, dtype=np.float64)
    rc = lib().ora_dense_lu_solve(A.shape[0], A.ctypes.data_as(_dp), x.ctypes.data_as(_dp))
    return rc, x


def match_pass(rowptr, col, val, theta=0.25, rounds=4):
    rp, rpp = _i(rowptr); c, cp = _i(col); v, vp = _d(val)
    n = len(rp) - 1
    partner = np.full(n, -1, np.int32)
    r = lib().ora_match_pass(n, rpp, cp, vp, float(theta), int(rounds), partner.ctypes.data_as(_ip))
    return partner, r
