"""The C-ABI library loads and exports every function include/sim.h declares
(no GPU needed: nothing is called)."""
import ctypes
import os

import pytest


def test_library_exports_every_declared_symbol():
    from paper_1606_00548_gb300 import build, sim
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = sim.header_functions()
    assert "sim_create" in names and "sim_linear_solve" in names and "sim_step" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a signature for every exported function, and nothing else
    assert sorted(sim._SIGS) == names


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1606_00548_gb300 import sim
    saved = sim._lib
    sim._lib = None
    try:
        with pytest.raises(RuntimeError):
            sim.load(str(tmp_path / "missing.so"))
    finally:
        sim._lib = saved


def test_argument_checks_before_any_device_call():
    """Entry points reject bad arguments with SIM_EINVAL before they touch the
    device (host logic only; nothing runs on a GPU): null handles, an empty
    batch, a network on an empty grid, a negative stall slab.  A rejected
    creation leaves its message for sim_last_error(NULL)."""
    from paper_1606_00548_gb300 import build, sim
    lib = ctypes.CDLL(build.build())
    EINVAL = sim.SIM_EINVAL
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.sim_step.argtypes = [vp, dbl, vp]
    lib.sim_get_stats.argtypes = [vp, vp]
    lib.sim_run_report.argtypes = [vp, ctypes.c_char_p, i64, ctypes.POINTER(i64)]
    lib.sim_batch_create.argtypes = [i32, vp, i32, ctypes.POINTER(vp)]
    lib.sim_net_create.argtypes = [i32, i32, i32, ctypes.c_uint64, vp, ctypes.POINTER(vp)]
    lib.sim_net_inject_stall.argtypes = [vp, i32]
    lib.sim_net_time_conv.argtypes = [vp, i32, i32, ctypes.POINTER(dbl)]
    lib.sim_last_error.argtypes = [vp]
    lib.sim_last_error.restype = ctypes.c_char_p
    n = i64(0)
    assert lib.sim_step(None, 1.0, None) == EINVAL
    assert lib.sim_get_stats(None, None) == EINVAL
    assert lib.sim_run_report(None, None, 0, ctypes.byref(n)) == EINVAL
    assert lib.sim_net_inject_stall(None, 0) == EINVAL
    us = dbl(0.0)
    assert lib.sim_net_time_conv(None, 0, 1, ctypes.byref(us)) == EINVAL
    out = vp(123)
    assert lib.sim_batch_create(0, None, 0, ctypes.byref(out)) == EINVAL
    assert b"sim_batch_create" in lib.sim_last_error(None)
    out = vp(123)
    assert lib.sim_net_create(0, 4, 4, 1, None, ctypes.byref(out)) == EINVAL
    assert out.value is None
    assert b"bad grid" in lib.sim_last_error(None)
