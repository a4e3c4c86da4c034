"""Failure detection and resume on the GPU, without faulting anything.

* Cancellation: a device flag that the walk polls, written by an
  asynchronous copy on another stream while a long walk runs: the kernel
  stops taking work, returns promptly and reports MCG_ERR_CANCELLED (no trap,
  no abandoned wait).  It runs first in a fresh process on purpose: the
  library loads its kernels before the first launch, so queueing the exit
  kernel behind the running walk does not block the host until the walk
  ends (what CUDA's lazy module loading would otherwise do).
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
    ds.work.fill_(255)          # stale records would read as NaN, not as results
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
