"""ctypes binding of libsim.so (include/sim.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module only converts
Python / numpy / torch arguments into the C structs and pointers of the ABI.
There is no fallback: if the library or a GPU is missing, calls raise.

Functions keep the ABI's names (sim_create, sim_step, sim_newton_step,
sim_linear_solve, ...).  `Simulator` wraps one handle for a synthetic case
from `synth` and exposes the same operations with numpy / torch arguments.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsim.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sim.h")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_i8p = C.POINTER(C.c_int8)
_vp = C.c_void_p

SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_ENAN, SIM_ENOCONV_LINEAR, SIM_ENOCONV_NEWTON, SIM_ETIMEOUT, SIM_ELIMIT = range(9)
STATUS_NAMES = ["SIM_OK", "SIM_EINVAL", "SIM_ENOMEM", "SIM_ECUDA", "SIM_ENAN", "SIM_ENOCONV_LINEAR",
                "SIM_ENOCONV_NEWTON", "SIM_ETIMEOUT", "SIM_ELIMIT"]


class SimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class sim_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("top_depth", C.c_double)]


class sim_rock(C.Structure):
    _fields_ = [("kx", _dp), ("ky", _dp), ("kz", _dp), ("poro", _dp), ("c_rock", C.c_double), ("p_ref", C.c_double)]


class sim_fluid(C.Structure):
    _fields_ = [("model", C.c_int32),
                ("rho_w_ref", C.c_double), ("rho_o_ref", C.c_double), ("c_w", C.c_double), ("c_o", C.c_double),
                ("mu_w", C.c_double), ("mu_o", C.c_double),
                ("rho_ws", C.c_double), ("rho_os", C.c_double), ("rho_gs", C.c_double), ("bw_c", C.c_double),
                ("bw_pref", C.c_double), ("bo_c_us", C.c_double), ("muo_c_us", C.c_double),
                ("npvt", C.c_int32),
                ("pvt_p", _dp), ("pvt_bo", _dp), ("pvt_rs", _dp), ("pvt_muo", _dp), ("pvt_bg", _dp), ("pvt_mug", _dp),
                ("swc", C.c_double), ("sor", C.c_double), ("sgc", C.c_double), ("sorg", C.c_double),
                ("nw", C.c_double), ("now", C.c_double), ("ng", C.c_double), ("nog", C.c_double),
                ("cnv_rho", C.c_double * 3)]


class sim_well(C.Structure):
    _fields_ = [("i", C.c_int32), ("j", C.c_int32), ("k_top", C.c_int32), ("k_bot", C.c_int32), ("type", C.c_int32),
                ("bhp", C.c_double), ("r_w", C.c_double), ("skin", C.c_double), ("control", C.c_int32),
                ("rate", C.c_double)]


class sim_options(C.Structure):
    _fields_ = [("newton_tol", C.c_double), ("newton_max", C.c_int32), ("lin_tol", C.c_double),
                ("gmres_m", C.c_int32), ("gmres_max_restarts", C.c_int32), ("precond", C.c_int32),
                ("stage2", C.c_int32), ("amg_theta", C.c_double), ("amg_rounds", C.c_int32),
                ("amg_coarse_max", C.c_int32), ("amg_max_levels", C.c_int32), ("chop_ds", C.c_double),
                ("chop_dp", C.c_double), ("max_cuts", C.c_int32), ("precision", C.c_int32),
                ("amg_cycles", C.c_int32), ("graphs", C.c_int32), ("decouple", C.c_int32),
                ("cpr_stages", C.c_int32), ("krylov", C.c_int32), ("lin_max_iter", C.c_int32),
                ("forcing", C.c_int32), ("ew_gamma", C.c_double), ("ew_beta", C.c_double),
                ("theta_max", C.c_double), ("fused_coarse", C.c_int32), ("orth", C.c_int32)]


class sim_linear_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("b_norm", C.c_double), ("r_norm", C.c_double)]


class sim_phase_info(C.Structure):
    _fields_ = [("assemble_us", C.c_double), ("setup_us", C.c_double), ("solve_us", C.c_double),
                ("update_us", C.c_double), ("assemble_bytes", C.c_double), ("setup_bytes", C.c_double),
                ("solve_bytes", C.c_double), ("update_bytes", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class sim_newton_info(C.Structure):
    _fields_ = [("newton_iterations", C.c_int32), ("linear_iterations", C.c_int32), ("converged", C.c_int32),
                ("linear_failures", C.c_int32), ("cnv", C.c_double), ("phase", sim_phase_info),
                ("lin_residual", C.c_double)]


class sim_step_info(C.Structure):
    _fields_ = [("cuts", C.c_int32), ("newton_iterations", C.c_int32), ("linear_iterations", C.c_int32),
                ("substeps", C.c_int32), ("ok", C.c_int32), ("phase", sim_phase_info), ("mb_error", C.c_double)]


class sim_stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("newton_iterations", C.c_int64),
                ("linear_iterations", C.c_int64), ("device_bytes", C.c_int64),
                ("spmv_block", C.c_int32), ("amg_block", C.c_int32), ("stage_block", C.c_int32)]


_SIGS = {
    "sim_create": ([C.POINTER(sim_grid), C.POINTER(sim_rock), C.POINTER(sim_fluid), C.POINTER(sim_well), C.c_int32,
                    C.POINTER(sim_options), _vp, C.POINTER(_vp)], C.c_int),
    "sim_destroy": ([_vp], None),
    "sim_set_state": ([_vp, _dp, _dp, _dp, _i8p], C.c_int),
    "sim_get_state": ([_vp, _dp, _dp, _dp, _i8p], C.c_int),
    "sim_step": ([_vp, C.c_double, C.POINTER(sim_step_info)], C.c_int),
    "sim_newton_solve": ([_vp, C.c_double, C.POINTER(sim_newton_info)], C.c_int),
    "sim_newton_step": ([_vp, C.c_double, C.POINTER(sim_newton_info)], C.c_int),
    "sim_accept_step": ([_vp, C.c_double], C.c_int),
    "sim_linear_solve": ([_vp, _vp, _vp, C.POINTER(sim_linear_info)], C.c_int),
    "sim_set_iterate": ([_vp, _dp, _i8p], C.c_int),
    "sim_get_iterate": ([_vp, _dp, _i8p], C.c_int),
    "sim_assemble": ([_vp, C.c_double], C.c_int),
    "sim_get_residual": ([_vp, _dp], C.c_int),
    "sim_get_jacobian": ([_vp, _dp], C.c_int),
    "sim_set_jacobian": ([_vp, _dp], C.c_int),
    "sim_cnv": ([_vp, C.c_double, _dp], C.c_int),
    "sim_spmv": ([_vp, _vp, _vp], C.c_int),
    "sim_precond_setup": ([_vp], C.c_int),
    "sim_precond_apply": ([_vp, _vp, _vp], C.c_int),
    "sim_get_qi": ([_vp, _dp, _dp], C.c_int),
    "sim_amg_levels": ([_vp], C.c_int32),
    "sim_amg_level_info": ([_vp, C.c_int32, _ip, _ip], C.c_int),
    "sim_amg_level_agg": ([_vp, C.c_int32, _ip], C.c_int),
    "sim_amg_level_ell": ([_vp, C.c_int32, _ip, _dp], C.c_int),
    "sim_component_mass": ([_vp, _dp], C.c_int),
    "sim_cumulative_well_mass": ([_vp, _dp], C.c_int),
    "sim_well_rates": ([_vp, _dp], C.c_int),
    "sim_time_op": ([_vp, C.c_int32, C.c_int32, _dp], C.c_int),
    "sim_run_report": ([_vp, C.c_char_p, C.c_int64, C.POINTER(C.c_int64)], C.c_int),
    "sim_perforations": ([_vp], C.c_int32),
    "sim_get_well_bhp": ([_vp, _dp], C.c_int),
    "sim_set_well_bhp": ([_vp, _dp], C.c_int),
    "sim_well_component_rates": ([_vp, _dp], C.c_int),
    "sim_get_well_system": ([_vp, _dp, _dp, _dp, _dp], C.c_int),
    "sim_set_well_system": ([_vp, _dp, _dp, _dp, _dp], C.c_int),
    "sim_get_stats": ([_vp, C.POINTER(sim_stats)], C.c_int),
    "sim_block_size": ([_vp], C.c_int32),
    "sim_cnv_noalloc": ([C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_int32,
                         _vp, _vp, _dp, C.c_double, _vp, _vp], C.c_int),
    "sim_probe_fma_rates": ([_dp, _dp], C.c_int),
    "sim_probe_fp64_pipe": ([_dp, _dp, _dp], C.c_int),
    "sim_autotune": ([_vp, C.c_double], C.c_int),
    "sim_autotune_cached": ([_vp, C.c_double, C.c_char_p, C.POINTER(C.c_int32)], C.c_int),
    "sim_batch_create": ([C.c_int32, C.POINTER(_vp), C.c_int32, C.POINTER(_vp)], C.c_int),
    "sim_batch_destroy": ([_vp], None),
    "sim_batch_step": ([_vp, _dp, C.POINTER(sim_step_info), C.POINTER(C.c_int)], C.c_int),
    "sim_batch_set_mode": ([_vp, C.c_int32], C.c_int),
    "sim_batch_mode": ([_vp], C.c_int32),
    "sim_batch_stats": ([_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "sim_batch_last_error": ([_vp], C.c_char_p),
    "sim_batch_phase_seconds": ([_vp, _dp, _dp, _dp], C.c_int),
    "sim_net_create": ([C.c_int32, C.c_int32, C.c_int32, C.c_uint64, _vp, C.POINTER(_vp)], C.c_int),
    "sim_net_destroy": ([_vp], None),
    "sim_net_param_count": ([_vp], C.c_int64),
    "sim_net_set_params": ([_vp, C.POINTER(C.c_float)], C.c_int),
    "sim_net_get_params": ([_vp, C.POINTER(C.c_float)], C.c_int),
    "sim_net_forward": ([_vp, _vp, _vp], C.c_int),
    "sim_net_loss_grad": ([_vp, _vp, _vp, _dp, C.POINTER(C.c_float)], C.c_int),
    "sim_net_train_step": ([_vp, _vp, _vp, C.c_float, _dp], C.c_int),
    "sim_net_last_error": ([_vp], C.c_char_p),
    "sim_net_time_conv": ([_vp, C.c_int32, C.c_int32, _dp], C.c_int),
    "sim_net_inject_stall": ([_vp, C.c_int32], C.c_int),
    "sim_set_learned_stage": ([_vp, _vp, C.c_int32], C.c_int),
    "sim_learned_pairs": ([_vp, C.c_int32, _vp, _vp], C.c_int),
    "sim_learned_fallbacks": ([_vp], C.c_int64),
    "sim_learned_available": ([_vp], C.c_int32),
    "sim_last_error": ([_vp], C.c_char_p),
    "sim_clear_error": ([_vp], None),
}

_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/sim.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sim_[a-z0-9_]+)\s*\(", txt)))


def load(path: str = LIB_PATH):
    """Load libsim.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_1606_00548_gb300.build.build())")
    L = C.CDLL(path)
    for name, (args, res) in _SIGS.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(handle, st):
    if st != SIM_OK:
        msg = load().sim_last_error(handle)
        raise SimError(st, msg.decode() if msg else "")


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _ptr(t):
    """Device pointer of a CUDA torch tensor (contiguous float64)."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return _vp(t.data_ptr())


def _ptrf(t):
    """Device pointer of a CUDA torch tensor (contiguous float32)."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return _vp(t.data_ptr())


class Net:
    """The learned pressure stage's network (include/sim.h, sim_net_*)."""

    def __init__(self, nx, ny, nz, seed=0, stream=None):
        self.L = load()
        h = _vp()
        st = self.L.sim_net_create(nx, ny, nz, seed, _vp(stream) if stream else None, C.byref(h))
        if st != SIM_OK:
            raise SimError(st, (self.L.sim_last_error(None) or b"").decode())
        self.h = h
        self.N = nx * ny * nz
        self.nparam = self.L.sim_net_param_count(h)

    def _check(self, st):
        if st != SIM_OK:
            raise SimError(st, (self.L.sim_net_last_error(self.h) or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.sim_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparam
        self._check(self.L.sim_net_set_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float))))

    def get_params(self):
        p = np.zeros(self.nparam, np.float32)
        self._check(self.L.sim_net_get_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float))))
        return p

    def forward(self, x_dev, y_dev):
        self._check(self.L.sim_net_forward(self.h, _ptrf(x_dev), _ptrf(y_dev)))

    def loss_grad(self, x_dev, t_dev):
        loss = C.c_double()
        g = np.zeros(self.nparam, np.float32)
        self._check(self.L.sim_net_loss_grad(self.h, _ptrf(x_dev), _ptrf(t_dev), C.byref(loss),
                                             g.ctypes.data_as(C.POINTER(C.c_float))))
        return loss.value, g

    def inject_stall(self, slab=0):
        """testing hook: the next forward pass's first convolution skips one
        staged copy, so its bounded wait runs out (SIM_ETIMEOUT)"""
        self._check(self.L.sim_net_inject_stall(self.h, int(slab)))

    def time_conv(self, which, reps=10):
        """microseconds per launch of one convolution kernel (0 forward, 1 weight
        gradient with its fold, 2 data gradient) of hidden layer 2"""
        v = C.c_double()
        self._check(self.L.sim_net_time_conv(self.h, int(which), int(reps), C.byref(v)))
        return v.value

    def train_step(self, x_dev, t_dev, lr, want_loss=True):
        loss = C.c_double()
        self._check(self.L.sim_net_train_step(self.h, _ptrf(x_dev), _ptrf(t_dev), float(lr),
                                              C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None


def options_from(solver: dict, precision: int = 0) -> sim_options:
    o = sim_options()
    for name in ("newton_tol", "lin_tol", "amg_theta", "chop_ds", "chop_dp", "ew_gamma", "ew_beta", "theta_max"):
        setattr(o, name, float(solver[name]))
    for name in ("newton_max", "gmres_m", "gmres_max_restarts", "precond", "stage2", "amg_rounds",
                 "amg_coarse_max", "amg_max_levels", "max_cuts", "amg_cycles", "decouple", "cpr_stages",
                 "krylov", "lin_max_iter", "forcing"):
        setattr(o, name, int(solver[name]))
    o.precision = int(precision)
    o.graphs = int(solver.get("graphs", 1))
    o.fused_coarse = int(solver.get("fused_coarse", 1))
    o.orth = int(solver.get("orth", 0))
    return o


class Simulator:
    """One simulator handle for a synth case (inputs copied into the library)."""

    def __init__(self, case: dict, precision: int = 0, stream=None, **solver_overrides):
        L = load()
        self.L = L
        self.case = case
        keep = []
        g = sim_grid(case["nx"], case["ny"], case["nz"], case["dx"], case["dy"], case["dz"], case["top_depth"])
        r = sim_rock()
        for name in ("kx", "ky", "kz", "poro"):
            a, p = _d(case[name]); keep.append(a); setattr(r, name, p)
        r.c_rock, r.p_ref = case["c_rock"], case["p_ref"]
        fl = case["fluid"]
        f = sim_fluid()
        f.model = case["model"]
        for name, _ in sim_fluid._fields_:
            if name in fl and name not in ("pvt_p", "pvt_bo", "pvt_rs", "pvt_muo", "pvt_bg", "pvt_mug"):
                setattr(f, name, float(fl[name]))
        if case["model"] == 3:
            f.npvt = len(fl["pvt_p"])
            for name in ("pvt_p", "pvt_bo", "pvt_rs", "pvt_muo", "pvt_bg", "pvt_mug"):
                a, p = _d(fl[name]); keep.append(a); setattr(f, name, p)
        for c in range(3):
            f.cnv_rho[c] = case["cnv_rho"][c]
        ws = case["wells"]
        W = (sim_well * max(1, len(ws)))()
        for k, w in enumerate(ws):
            W[k] = sim_well(w["i"], w["j"], w["k0"], w["k1"], w["type"], w["bhp"], w["rw"], w["skin"],
                            int(w.get("ctrl", 0)), float(w.get("rate", 0.0)))
        sv = dict(case["solver"]); sv.update(solver_overrides)
        self.opts = options_from(sv, precision)
        h = _vp()
        st = L.sim_create(C.byref(g), C.byref(r), C.byref(f), W, len(ws), C.byref(self.opts),
                          _vp(stream) if stream else None, C.byref(h))
        if st != SIM_OK:
            raise SimError(st, (L.sim_last_error(None) or b"").decode())
        self.h = h
        self.N = case["nx"] * case["ny"] * case["nz"]
        self.b = L.sim_block_size(h)
        ini = case["init"]
        self.set_state(ini["p"], ini["sw"], ini["x3"], ini["phase"])

    def close(self):
        if getattr(self, "h", None):
            self.L.sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clear_error(self):
        self.L.sim_clear_error(self.h)

    # state --------------------------------------------------------------------
    def set_state(self, p, sw, x3, phase):
        p, pp = _d(p); sw, sp = _d(sw); x3, xp = _d(x3)
        ph = np.ascontiguousarray(phase, dtype=np.int8)
        _check(self.h, self.L.sim_set_state(self.h, pp, sp, xp, ph.ctypes.data_as(_i8p)))

    def get_state(self):
        N = self.N
        p = np.zeros(N); sw = np.zeros(N); x3 = np.zeros(N); ph = np.zeros(N, np.int8)
        _check(self.h, self.L.sim_get_state(self.h, p.ctypes.data_as(_dp), sw.ctypes.data_as(_dp),
                                            x3.ctypes.data_as(_dp), ph.ctypes.data_as(_i8p)))
        return p, sw, x3, ph

    def set_iterate(self, x, phase):
        x, xp = _d(x)
        ph = np.ascontiguousarray(phase, dtype=np.int8)
        _check(self.h, self.L.sim_set_iterate(self.h, xp, ph.ctypes.data_as(_i8p)))

    def get_iterate(self):
        x = np.zeros(self.N * self.b); ph = np.zeros(self.N, np.int8)
        _check(self.h, self.L.sim_get_iterate(self.h, x.ctypes.data_as(_dp), ph.ctypes.data_as(_i8p)))
        return x, ph

    # nonlinear ----------------------------------------------------------------
    def step(self, dt):
        info = sim_step_info()
        st = self.L.sim_step(self.h, float(dt), C.byref(info))
        if st not in (SIM_OK, SIM_ENOCONV_NEWTON):
            _check(self.h, st)
        return st, info

    def newton_solve(self, dt):
        info = sim_newton_info()
        st = self.L.sim_newton_solve(self.h, float(dt), C.byref(info))
        if st not in (SIM_OK, SIM_ENOCONV_NEWTON, SIM_ENAN):
            _check(self.h, st)
        return st, info

    def newton_step(self, dt):
        info = sim_newton_info()
        st = self.L.sim_newton_step(self.h, float(dt), C.byref(info))
        if st not in (SIM_OK, SIM_ENAN):
            _check(self.h, st)
        return st, info

    def accept_step(self, dt):
        _check(self.h, self.L.sim_accept_step(self.h, float(dt)))

    # assembly / linear algebra -------------------------------------------------
    def assemble(self, dt):
        _check(self.h, self.L.sim_assemble(self.h, float(dt)))

    def residual(self):
        R = np.zeros(self.N * self.b)
        _check(self.h, self.L.sim_get_residual(self.h, R.ctypes.data_as(_dp)))
        return R

    def jacobian(self):
        J = np.zeros(7 * self.b * self.b * self.N)
        _check(self.h, self.L.sim_get_jacobian(self.h, J.ctypes.data_as(_dp)))
        return J

    def set_jacobian(self, J):
        J, jp = _d(J)
        _check(self.h, self.L.sim_set_jacobian(self.h, jp))

    def cnv(self, dt):
        v = C.c_double()
        _check(self.h, self.L.sim_cnv(self.h, float(dt), C.byref(v)))
        return v.value

    def spmv(self, x_dev, y_dev):
        _check(self.h, self.L.sim_spmv(self.h, _ptr(x_dev), _ptr(y_dev)))

    def precond_setup(self):
        _check(self.h, self.L.sim_precond_setup(self.h))

    def precond_apply(self, r_dev, z_dev):
        _check(self.h, self.L.sim_precond_apply(self.h, _ptr(r_dev), _ptr(z_dev)))

    def linear_solve(self, b_dev, x_dev):
        info = sim_linear_info()
        st = self.L.sim_linear_solve(self.h, _ptr(b_dev), _ptr(x_dev), C.byref(info))
        if st not in (SIM_OK, SIM_ENOCONV_LINEAR):
            _check(self.h, st)
        return st, info

    def qi(self):
        w = np.zeros(self.b * self.N); ap = np.zeros(7 * self.N)
        _check(self.h, self.L.sim_get_qi(self.h, w.ctypes.data_as(_dp), ap.ctypes.data_as(_dp)))
        return w, ap

    def amg_levels(self):
        out = []
        for l in range(self.L.sim_amg_levels(self.h)):
            n = C.c_int32(); w = C.c_int32()
            _check(self.h, self.L.sim_amg_level_info(self.h, l, C.byref(n), C.byref(w)))
            d = dict(n=n.value, width=w.value)
            if l + 1 < self.L.sim_amg_levels(self.h):
                agg = np.zeros(n.value, np.int32)
                _check(self.h, self.L.sim_amg_level_agg(self.h, l, agg.ctypes.data_as(_ip)))
                d["agg"] = agg
            if l >= 1:
                col = np.zeros(w.value * n.value, np.int32); val = np.zeros(w.value * n.value)
                _check(self.h, self.L.sim_amg_level_ell(self.h, l, col.ctypes.data_as(_ip), val.ctypes.data_as(_dp)))
                d["col"] = col.reshape(w.value, n.value); d["val"] = val.reshape(w.value, n.value)
            out.append(d)
        return out

    def component_mass(self):
        m = np.zeros(3); _check(self.h, self.L.sim_component_mass(self.h, m.ctypes.data_as(_dp))); return m

    def cumulative_well_mass(self):
        m = np.zeros(3); _check(self.h, self.L.sim_cumulative_well_mass(self.h, m.ctypes.data_as(_dp))); return m

    def time_op(self, which, reps=20):
        """Average device microseconds of `reps` back-to-back launches (0 SpMV, 1 CPR apply)."""
        us = C.c_double()
        _check(self.h, self.L.sim_time_op(self.h, int(which), int(reps), C.byref(us)))
        return us.value

    def run_report(self):
        """the handle's JSON run report (counters, per-phase device time and bytes), parsed"""
        import json
        n = C.c_int64(0)
        self.L.sim_run_report(self.h, None, 0, C.byref(n))
        buf = C.create_string_buffer(n.value + 1)
        _check(self.h, self.L.sim_run_report(self.h, buf, n.value + 1, C.byref(n)))
        return json.loads(buf.value.decode())

    def well_rates(self):
        q = np.zeros(3); _check(self.h, self.L.sim_well_rates(self.h, q.ctypes.data_as(_dp))); return q

    # well unknowns (host arrays) -------------------------------------------
    @property
    def nwells(self):
        return len(self.case["wells"])

    def perforations(self):
        return int(self.L.sim_perforations(self.h))

    def well_bhp(self):
        p = np.zeros(max(self.nwells, 1))
        _check(self.h, self.L.sim_get_well_bhp(self.h, p.ctypes.data_as(_dp)))
        return p[:self.nwells]

    def set_well_bhp(self, bhp):
        p = np.ascontiguousarray(bhp, dtype=np.float64).reshape(-1)
        if p.size == 0:
            p = np.zeros(1)
        _check(self.h, self.L.sim_set_well_bhp(self.h, p.ctypes.data_as(_dp)))

    def well_component_rates(self):
        q = np.zeros(3 * max(self.nwells, 1))
        _check(self.h, self.L.sim_well_component_rates(self.h, q.ctypes.data_as(_dp)))
        return q[:3 * self.nwells].reshape(self.nwells, 3)

    def well_system(self):
        nw, npf = max(self.nwells, 1), max(self.perforations(), 1)
        Rw, Aww = np.zeros(nw), np.zeros(nw)
        Apw, Awp = np.zeros(npf * self.b), np.zeros(npf * self.b)
        _check(self.h, self.L.sim_get_well_system(self.h, Rw.ctypes.data_as(_dp), Apw.ctypes.data_as(_dp),
                                                  Awp.ctypes.data_as(_dp), Aww.ctypes.data_as(_dp)))
        npf = self.perforations()
        return (Rw[:self.nwells], Apw[:npf * self.b].reshape(npf, self.b), Awp[:npf * self.b].reshape(npf, self.b),
                Aww[:self.nwells])

    def set_well_system(self, Rw, Apw, Awp, Aww):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (Rw, Apw, Awp, Aww)]
        arrs = [a if a.size else np.zeros(1) for a in arrs]
        _check(self.h, self.L.sim_set_well_system(self.h, *[a.ctypes.data_as(_dp) for a in arrs]))

    def set_learned_stage(self, net, enable=True):
        _check(self.h, self.L.sim_set_learned_stage(self.h, net.h if net is not None else None, 1 if enable else 0))

    def learned_pairs(self, k, x_dev, y_dev):
        _check(self.h, self.L.sim_learned_pairs(self.h, int(k), _ptrf(x_dev), _ptrf(y_dev)))

    def learned_available(self):
        return self.L.sim_learned_available(self.h)

    def learned_fallbacks(self):
        return self.L.sim_learned_fallbacks(self.h)

    def stats(self):
        s = sim_stats(); _check(self.h, self.L.sim_get_stats(self.h, C.byref(s))); return s

    def autotune_cached(self, dt, path):
        hit = C.c_int32()
        _check(self.h, self.L.sim_autotune_cached(self.h, float(dt), os.fsencode(path), C.byref(hit)))
        return bool(hit.value)

    def autotune(self, dt):
        _check(self.h, self.L.sim_autotune(self.h, float(dt)))


SIM_BATCH_LOCKSTEP, SIM_BATCH_CONCURRENT = 0, 1


class Batch:
    """Time stepping of independent simulators together (sim_batch_*):
    lockstep rounds with one batched solve per round, or concurrent members."""

    def __init__(self, members, nthreads=0, mode=None):
        self.L = load()
        self.members = list(members)
        arr = (_vp * len(self.members))(*[m.h for m in self.members])
        h = _vp()
        st = self.L.sim_batch_create(len(self.members), arr, int(nthreads), C.byref(h))
        if st != SIM_OK:
            raise SimError(st, (self.L.sim_last_error(None) or b"").decode())
        self.h = h
        if mode is not None:
            st = self.L.sim_batch_set_mode(self.h, int(mode))
            if st != SIM_OK:
                raise SimError(st, "sim_batch_set_mode: mode not available for these members")

    def mode(self):
        return self.L.sim_batch_mode(self.h)

    def stats(self):
        r, s, l = C.c_int64(), C.c_int64(), C.c_int64()
        self.L.sim_batch_stats(self.h, C.byref(r), C.byref(s), C.byref(l))
        return dict(rounds=r.value, solves=s.value, launches=l.value)

    def last_error(self):
        return (self.L.sim_batch_last_error(self.h) or b"").decode()

    def phase_seconds(self):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self.L.sim_batch_phase_seconds(self.h, C.byref(a), C.byref(b), C.byref(c))
        return dict(newton=a.value, solve=b.value, update=c.value)

    def step(self, dts):
        n = len(self.members)
        dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dts, dtype=np.float64), (n,)))
        infos = (sim_step_info * n)()
        sts = (C.c_int * n)()
        self.L.sim_batch_step(self.h, dt.ctypes.data_as(_dp), infos, sts)
        return list(sts), list(infos)

    def close(self):
        if getattr(self, "h", None):
            self.L.sim_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sim_cnv_noalloc(case: dict, b: int, R_dev, poro_dev, dt: float, out_dev, stream=None) -> None:
    """CNV of a residual held in caller-owned device tensors, without any device
    allocation inside the library (see include/sim.h)."""
    L = load()
    rho, rp = _d(case["cnv_rho"][:b])
    st = L.sim_cnv_noalloc(case["nx"], case["ny"], case["nz"], case["dx"], case["dy"], case["dz"], b,
                           _ptr(R_dev), _ptr(poro_dev), rp, float(dt), _ptr(out_dev), _vp(stream) if stream else None)
    _check(None, st)


def sim_probe_fma_rates():
    """(FP64, FP32) fused-multiply-add rates of the current device, per second."""
    L = load()
    a = C.c_double(); b = C.c_double()
    _check(None, L.sim_probe_fma_rates(C.byref(a), C.byref(b)))
    return a.value, b.value


def sim_probe_fp64_pipe():
    """(FP64 FMAs per second, SM MHz during the probe, FMAs per clock per SM)"""
    L = load()
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(None, L.sim_probe_fp64_pipe(C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value
