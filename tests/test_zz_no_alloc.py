"""sim_cnv_noalloc: the CNV measure for callers that cannot allocate device
memory (their memory belongs to another allocator, or a cudaMalloc's latency
and implicit synchronisation are not acceptable in their loop).

It is checked through the C ABI against sim_cnv, the handle-based entry point
that computes the same quantity, on two calls in a row (two different
residuals).  This file is collected last so that a failure here does not hide
the other tests."""
import numpy as np
import pytest

from paper_1606_00548_gb300 import synth

pytestmark = pytest.mark.gpu


def test_cnv_noalloc_matches_sim_cnv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_00548_gb300 import build
    build.build()
    from paper_1606_00548_gb300 import sim
    case = synth.black_oil_case(nx=33, ny=17, nz=5, seed=71)
    g = sim.Simulator(case)
    dt = 10.0
    poro = torch.tensor(case["poro"], dtype=torch.float64, device="cuda")
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    results = []
    for call in range(2):
        g.assemble(dt)
        expect = g.cnv(dt)
        R = torch.tensor(g.residual(), dtype=torch.float64, device="cuda")
        sim.sim_cnv_noalloc(case, g.b, R, poro, dt, out, stream)
        torch.cuda.synchronize()
        got = float(out.item())
        assert got == pytest.approx(expect, rel=1e-12, abs=0.0), (call, got, expect)
        results.append(got)
        g.newton_step(dt)            # a different residual for the second call
    assert results[0] != results[1]


def test_cnv_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_00548_gb300 import sim
    L = sim.load()
    rho = np.array([1.0, 1.0, 1.0])
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = sim._ptr(dummy)
    st = L.sim_cnv_noalloc(70000, 70000, 1, 1.0, 1.0, 1.0, 3, p, p, rho.ctypes.data_as(sim._dp), 1.0, p, None)
    assert st == sim.SIM_ELIMIT
    assert b"2^31" in L.sim_last_error(None)
