"""Ensemble runtime and autotuner on the GPU.

Lockstep mode (one batched FGMRES per Newton round, every Krylov operation a
single launch over all members) and concurrent mode both give results
bit-identical to the same members advanced one at a time with sim_step
(each member's arithmetic is that of its own solve), member results match
the oracle, and the batched solves' launch count does not grow with the
number of members; the autotuner changes launch shapes but not results."""
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
    """uneven oil-water members: one with a one-level hierarchy (32 cells), and
    some deep enough for several AMG levels and the fused coarse cycle"""
    shapes = [(17, 23, 5, 0.7), (31, 9, 4, 1.5), (12, 12, 8, 2.0), (40, 20, 3, 1.0), (4, 4, 2, 0.5),
              (48, 40, 10, 1.2)]
    return [synth.oil_water_case(nx=nx, ny=ny, nz=nz, sigma=sig, seed=60 + k, nsteps=2)
            for k, (nx, ny, nz, sig) in enumerate(shapes)]


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_equals_each_member_alone_and_oracle(torch_cuda, mode):
    import oracle
    from paper_1606_00548_gb300.sim import Batch, Simulator
    cases = small_members()
    A = [Simulator(c) for c in cases]
    B = [Simulator(c) for c in cases]
    batch = Batch(A, nthreads=4, mode=mode)
    assert batch.mode() == mode
    for step in range(2):
        sts, infos = batch.step(1.0)
        assert all(s == 0 for s in sts), (sts, batch.last_error())
        for b, info in zip(B, infos):
            st, ib = b.step(1.0)
            assert (ib.newton_iterations, ib.linear_iterations, ib.cuts, ib.substeps) == \
                   (info.newton_iterations, info.linear_iterations, info.cuts, info.substeps)
    for a, b in zip(A, B):
        for u, v in zip(a.get_state(), b.get_state()):
            assert np.array_equal(u, v)
    for k in (1, 4, 5):
        o = oracle.Oracle(cases[k])
        for _ in range(2):
            o.step(1.0)
        po, swo, _, _ = o.get_state()
        pa, swa, _, _ = A[k].get_state()
        assert np.abs(pa - po).max() <= 1e-6 * np.abs(po).max()
        assert np.abs(swa - swo).max() <= 1e-6
    if mode == 0:
        st = batch.stats()
        assert st["rounds"] > 0 and st["solves"] >= st["rounds"]
    batch.close()


def test_lockstep_black_oil_mixed_precision(torch_cuda):
    """black-oil members (3x3 blocks) with the FP32 preconditioner and Z"""
    from paper_1606_00548_gb300.sim import Batch, Simulator
    cases = [synth.black_oil_case(nx=nx, ny=ny, nz=nz, nsteps=2, dt=10.0, seed=70 + k)
             for k, (nx, ny, nz) in enumerate([(24, 20, 6), (13, 29, 4), (30, 30, 5)])]
    A = [Simulator(c, precision=1) for c in cases]
    B = [Simulator(c, precision=1) for c in cases]
    batch = Batch(A, mode=0)
    for dt in cases[0]["dt"]:
        sts, infos = batch.step(dt)
        assert all(s == 0 for s in sts), (sts, batch.last_error())
        for b in B:
            assert b.step(dt)[0] == 0
    for a, b in zip(A, B):
        for u, v in zip(a.get_state(), b.get_state()):
            assert np.array_equal(u, v)
    batch.close()


def test_batched_launches_do_not_grow_with_members(torch_cuda):
    """Eight members stepped in lockstep launch a small fraction of the kernels
    the same members launch stepped one by one, and about as many per round
    as two members do."""
    from paper_1606_00548_gb300.sim import Batch, Simulator

    def members(n):
        return [synth.oil_water_case(nx=30, ny=30, nz=6, sigma=1.0, seed=90 + k, nsteps=1) for k in range(n)]

    per_round = []
    for n in (2, 8):
        sims = [Simulator(c) for c in members(n)]
        batch = Batch(sims, mode=0)
        sts, _ = batch.step(1.0)
        assert all(s == 0 for s in sts)
        st = batch.stats()
        per_round.append(st["launches"] / st["rounds"])
        batch.close()
    assert per_round[1] <= 1.3 * per_round[0], per_round
    # the same eight members: launches of their solves stepped one by one
    # against the batched solves' launches (the per-member assembly, setup and
    # update launches, the same in both runs, are taken out)
    alone = [Simulator(c) for c in members(8)]
    l0 = sum(s.stats().kernel_launches for s in alone)
    for s in alone:
        s.step(1.0)
    l_alone = sum(s.stats().kernel_launches for s in alone) - l0
    sims = [Simulator(c) for c in members(8)]
    m0 = sum(s.stats().kernel_launches for s in sims)
    batch = Batch(sims, mode=0)
    batch.step(1.0)
    per_member = sum(s.stats().kernel_launches for s in sims) - m0
    l_batched = batch.stats()["launches"]
    batch.close()
    l_alone_solves = l_alone - per_member
    print(f"batched solve launches {l_batched} against {l_alone_solves} one member at a time")
    assert l_alone_solves > 0 and l_batched < 0.5 * l_alone_solves, (l_batched, l_alone_solves)


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


def test_autotune_cache_round_trip(torch_cuda, tmp_path):
    """The tuned shapes go into the JSON cache on the first call and come back
    from it, without timing, for another handle of the same grid; results do
    not depend on them."""
    import json
    from paper_1606_00548_gb300.sim import Simulator
    case = synth.black_oil_case(nx=26, ny=22, nz=5, nsteps=2, dt=10.0, seed=62)
    path = str(tmp_path / "tuning.json")
    a = Simulator(case)
    assert a.autotune_cached(10.0, path) is False
    entry = json.load(open(path))["b3_fp64_26x22x5"]
    st = a.stats()
    assert (entry["spmv"], entry["amg"], entry["stage"]) == (st.spmv_block, st.amg_block, st.stage_block)
    assert st.stage_block in (32, 64, 128, 256)
    b = Simulator(case)
    assert b.autotune_cached(10.0, path) is True
    sb = b.stats()
    assert (sb.spmv_block, sb.amg_block, sb.stage_block) == (st.spmv_block, st.amg_block, st.stage_block)
    c = Simulator(case)
    for dt in case["dt"]:
        b.step(dt); c.step(dt)
    for u, v in zip(b.get_state(), c.get_state()):
        assert np.array_equal(u, v)
