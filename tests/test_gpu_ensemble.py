"""Ensemble runtime and autotuner on the GPU.

Members advanced concurrently by the batch runtime give bit-identical
results to the same members advanced one at a time (members share nothing),
and member results match the oracle; the autotuner changes launch shapes but
not results."""
import numpy as np
import pytest

from paper_1606_00548_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_00548_gb300 import build
    build.build()
    return torch


def small_members():
    return [synth.oil_water_case(nx=nx, ny=ny, nz=nz, sigma=sig, seed=60 + k, nsteps=2)
            for k, (nx, ny, nz, sig) in enumerate([(17, 23, 5, 0.7), (31, 9, 4, 1.5), (12, 12, 8, 2.0),
                                                    (40, 20, 3, 1.0)])]


def test_batch_equals_sequential_and_oracle(torch_cuda):
    import oracle
    from paper_1606_00548_gb300.sim import Batch, Simulator
    cases = small_members()
    A = [Simulator(c) for c in cases]
    B = [Simulator(c) for c in cases]
    batch = Batch(A, nthreads=4)
    for step in range(2):
        sts, infos = batch.step(1.0)
        assert all(s == 0 for s in sts)
        for b, info in zip(B, infos):
            st, ib = b.step(1.0)
            assert ib.newton_iterations == info.newton_iterations
    for a, b in zip(A, B):
        for u, v in zip(a.get_state(), b.get_state()):
            assert np.array_equal(u, v)
    o = oracle.Oracle(cases[1])
    for _ in range(2):
        o.step(1.0)
    po, swo, _, _ = o.get_state()
    pa, swa, _, _ = A[1].get_state()
    assert np.abs(pa - po).max() <= 1e-6 * np.abs(po).max()
    assert np.abs(swa - swo).max() <= 1e-6
    batch.close()


def test_autotune_does_not_change_results(torch_cuda):
    from paper_1606_00548_gb300.sim import Simulator
    case = synth.black_oil_case(nx=26, ny=22, nz=5, nsteps=2, dt=10.0, seed=61)
    a = Simulator(case)
    b = Simulator(case)
    a.autotune(10.0)
    st = a.stats()
    assert st.spmv_block in (64, 128, 256, 512) and st.amg_block in (64, 128, 256)
    for dt in case["dt"]:
        a.step(dt); b.step(dt)
    for u, v in zip(a.get_state(), b.get_state()):
        assert np.array_equal(u, v)
