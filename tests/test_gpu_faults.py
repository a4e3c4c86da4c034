"""Failure detection and resume on the GPU, without faulting anything.

* Cancellation: a device flag that the walk polls, written by an
  asynchronous copy on another stream while a long walk runs: the kernel
  stops taking work, returns promptly and reports MCG_ERR_CANCELLED (no trap,
  no abandoned wait); every item that did not finish reads NaN, whatever the
  scratch held before.  It runs first in a fresh process on purpose: the
  library loads its kernels before the first launch, so queueing the exit
  kernel behind the running walk does not block the host until the walk
  ends (what CUDA's lazy module loading would otherwise do).
* A bounded wait that runs out: the launch starts with a migration-pool slot
  reserved and never published (the host-side hook fault_unpublished, a
  stand-in for a warp that died between reserving and writing).  The warp
  that claims it waits a bounded time, gives up, and the walk reports
  MCG_ERR_TIMEOUT through mcg_walk, mcgrav_solve and the server; every real
  walk is unaffected.  Nothing faults, traps or hangs.
* Non-finite data (a NaN in the boundary tables) reaches the status word as
  MCG_ERR_NONFINITE; the step cap as MCG_ERR_STEP_CAP.
* Checkpoint / resume: station states (64 bytes each) saved after half the
  paths and restored into a fresh solver give the same result, bit for bit,
  as one uninterrupted solve with the same batches.
"""
import time

import numpy as np
import pytest
import torch

from paper_1709_07469_gb300 import build as B
from paper_1709_07469_gb300 import mcgrav as M
from paper_1709_07469_gb300 import workloads as W
from paper_1709_07469_gb300.device import DeviceSolve
from tests.helpers import smooth_tables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    M.load()
    torch.cuda.init()


def _long_walk(cancel_ptr, stream=None):
    w = W.prism_ore_body()
    ds = DeviceSolve(w, batch=65536, precision=M.MCG_MIXED, stream=stream)   # ~2 s of work uncancelled
    ds.opts.cancel = cancel_ptr
    ds.reset()
    # scratch and outputs hold finite leftovers (zero exit records would read
    # as valid results if the walk did not mark its items first)
    ds.work.zero_()
    ds.pp_u.zero_()
    ds.pp_d.zero_()
    ds.pp_steps.fill_(7)
    torch.cuda.synchronize()
    return ds


def test_cancel_flag_in_device_memory_set_by_a_copy():
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    one = torch.ones(1, dtype=torch.int32).pin_memory()
    walk_stream, side = torch.cuda.Stream(), torch.cuda.Stream()   # two independent streams
    ds = _long_walk(flag.data_ptr(), stream=walk_stream)
    t0 = time.perf_counter()
    ds.walk(0)
    time.sleep(0.2)
    with torch.cuda.stream(side):
        flag.copy_(one, non_blocking=True)   # a copy-engine write while the walk runs
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert int(ds.status[0].item()) & (1 << M.MCG_ERR_CANCELLED), elapsed
    assert elapsed < 1.0
    u, d, steps = ds.per_path()
    unfinished = np.isnan(u)
    assert unfinished.mean() > 0.5                       # cancelled after ~10 % of the work
    assert np.isnan(d[unfinished]).all()
    assert np.isfinite(u[~unfinished]).all() and np.isfinite(d[~unfinished]).all()
    assert (steps[~unfinished] > 0).all()
    assert (steps != 7).all()                            # every item's steps written by this launch
    assert (steps == 0).sum() > 0                        # items never started


def _timeout_opts(w, **kw):
    return M.options(w, precision=M.MCG_MIXED, fault_unpublished=1, **kw)


def test_bounded_pool_wait_gives_up_with_timeout():
    w = W.sphere_line(paths=4096)
    ref = DeviceSolve(w, precision=M.MCG_MIXED)
    ref.reset()
    ref.walk(0)
    u0, d0, s0 = ref.per_path()
    assert int(ref.status[0].item()) == 0
    ds = DeviceSolve(w, precision=M.MCG_MIXED)
    ds.opts.fault_unpublished = 1
    ds.reset()
    t0 = time.perf_counter()
    ds.walk(0)
    u, d, s = ds.per_path()
    elapsed = time.perf_counter() - t0
    assert int(ds.status[0].item()) == 1 << M.MCG_ERR_TIMEOUT
    assert elapsed < 10.0
    # the reserved slot held no walk: every real walk finished unchanged
    assert np.array_equal(s, s0)
    assert np.array_equal(u, u0) and np.array_equal(d, d0)


def test_timeout_reaches_the_solver_and_the_server():
    w = W.sphere_line(paths=2048)
    r = M.mcgrav_solve(M.problem(w), w.stations, 2048, w.dt, 0, _timeout_opts(w), allow=(M.MCG_ERR_TIMEOUT,))
    assert r.status == M.MCG_ERR_TIMEOUT
    assert "bounded wait" in M.last_error()
    model = M.mcg_model_create(M.problem(w), w.dt, w.h)
    sv = M.mcg_server_create(M.server_config(_timeout_opts(w), chunk_paths=1024, min_paths=1024))
    try:
        rq = M.mcg_submit(sv, model, w.stations[:3], 1e-2, 5)
        M.mcg_wait(rq, 3, 60_000)
        done, rc, _ = M.mcg_poll(rq, 3)
        assert done == 1
        M.mcg_request_free(rq)
    finally:
        M.mcg_server_destroy(sv)
        M.mcg_model_destroy(model)
    assert rc == M.MCG_ERR_TIMEOUT      # never finished as a success


def test_nonfinite_boundary_data_is_reported():
    w = W.voxel_survey(shape=(16, 16, 8), table_n=(9, 9), paths=256)
    grid = torch.full((8, 16, 16), 100.0, dtype=torch.float32, device="cuda")
    faces = torch.from_numpy(smooth_tables(w)).cuda()
    faces[5, 4, 4] = float("nan")   # the top face: every walk ends near it
    prob = M.problem(w, grid=grid, faces=faces)
    st = np.array([[0.0, 0.0, 100.0], [10.0, -20.0, 150.0]])
    r = M.mcgrav_solve(prob, st, 2048, w.dt, 0, M.options(w), allow=(M.MCG_ERR_NONFINITE,))
    assert r.status == M.MCG_ERR_NONFINITE
    assert "finite" in M.last_error()


def test_step_cap_is_reported_by_both_precisions():
    w = W.prism_ore_body(paths=64)
    for prec in (M.MCG_FP64, M.MCG_MIXED):
        r = M.mcgrav_solve(M.problem(w), w.stations[:2], 64, w.dt, 0, M.options(w, precision=prec, max_steps=64),
                           allow=(M.MCG_ERR_STEP_CAP,))
        assert r.status == M.MCG_ERR_STEP_CAP


def test_resume_from_saved_station_states_is_exact():
    w = W.sphere_line(paths=8192)
    full = DeviceSolve(w, batch=2048, precision=M.MCG_MIXED).run(paths=8192)
    first = DeviceSolve(w, batch=2048, precision=M.MCG_MIXED)
    first.run(paths=4096)
    saved = first.states.cpu().numpy().copy()            # checkpoint: 64 B per station
    second = DeviceSolve(w, batch=2048, precision=M.MCG_MIXED)
    second.states.copy_(torch.from_numpy(saved))         # resume in a fresh solver
    for k in range(2):
        second.walk(4096 + 2048 * k)
        second.reduce()
    second.finalize()
    resumed = second.result()
    for key in ("u", "gz", "se_u", "se_gz", "n_paths", "path_steps"):
        assert np.array_equal(resumed[key], full[key]), key
