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
