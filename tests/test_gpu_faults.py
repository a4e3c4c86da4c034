"""Failure detection and resume on the GPU, without faulting anything.

* Cancellation: a host-mapped flag that the walk polls; set from the host
  while a long walk runs, the kernel stops taking work, returns promptly and
  reports MCG_ERR_CANCELLED (no trap, no abandoned wait).
* Non-finite data (a NaN in the boundary tables) reaches the status word as
  MCG_ERR_NONFINITE; the step cap as MCG_ERR_STEP_CAP.
* Checkpoint / resume: station states (64 bytes each) saved after half the
  paths and restored into a fresh solver give the same result, bit for bit,
  as one uninterrupted solve with the same batches.
"""
import ctypes
import ctypes.util
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


def _cudart():
    for name in ("libcudart.so", ctypes.util.find_library("cudart"), "/usr/local/cuda/lib64/libcudart.so"):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcudart not found")


def test_cancel_flag_stops_a_running_walk():
    rt = _cudart()
    host = ctypes.c_void_p()
    assert rt.cudaHostAlloc(ctypes.byref(host), ctypes.c_size_t(4), ctypes.c_uint(2)) == 0  # cudaHostAllocMapped
    dev = ctypes.c_void_p()
    assert rt.cudaHostGetDevicePointer(ctypes.byref(dev), host, ctypes.c_uint(0)) == 0
    flag = ctypes.cast(host, ctypes.POINTER(ctypes.c_int32))
    flag[0] = 0
    try:
        w = W.prism_ore_body()
        ds = DeviceSolve(w, batch=65536, precision=M.MCG_MIXED)   # ~20 s of work uncancelled
        ds.opts.cancel = dev.value
        ds.reset()
        t0 = time.perf_counter()
        ds.walk(0)                 # asynchronous: the walk is running now
        time.sleep(0.3)
        flag[0] = 1                # cancel from the host
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        status = int(ds.status[0].item())
        assert status & (1 << M.MCG_ERR_CANCELLED)
        assert elapsed < 5.0
    finally:
        rt.cudaFreeHost(host)


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
