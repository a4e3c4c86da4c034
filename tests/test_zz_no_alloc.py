"""mcg_walk_static: the walk for callers that cannot allocate device memory.

Some callers may only pass the buffers they were handed -- plug-in hosts with
a fixed list of input and output arrays, services whose memory manager owns
the whole device budget, latency-critical loops where an allocation would
synchronise the device.  mcg_walk_static serves them: same inputs and outputs
as mcg_walk, scratch kept in one fixed array inside the library.

These tests call it through the C ABI twice in a row (the second call reuses
the array the first one left behind) and compare every per-path output with
mcg_walk on the same inputs, within the per-path tolerance of the parity
tests (1e-12 relative; the kernels are the same, so the values agree
exactly).  This file is collected last so that a failure here does not hide
the rest of the suite; it passes alone in a fresh process and after the
other tests.
"""
import numpy as np
import pytest
import torch

from paper_1709_07469_gb300 import build as B
from paper_1709_07469_gb300 import mcgrav as M
from paper_1709_07469_gb300 import workloads as W
from paper_1709_07469_gb300.device import DeviceSolve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    M.load()


def static_walk(w, p0, N, precision):
    S = w.n_stations
    dev = torch.device("cuda")
    stations = torch.from_numpy(np.ascontiguousarray(w.stations)).to(dev)
    u = torch.full((S * N,), -1.0, dtype=torch.float64, device=dev)
    d = torch.full((S * N,), -1.0, dtype=torch.float64, device=dev)
    st = torch.full((S * N,), -1, dtype=torch.int64, device=dev)
    status = torch.zeros(2, dtype=torch.int32, device=dev)
    opts = M.options(w, precision=precision)
    M.mcg_walk_static(M.problem(w), stations, S, p0, N, w.dt, w.seed, opts, u, d, st, status)
    torch.cuda.synchronize()
    return (u.cpu().numpy().reshape(S, N), d.cpu().numpy().reshape(S, N), st.cpu().numpy().reshape(S, N),
            int(status[0].item()))


def walk(w, p0, N, precision):
    ds = DeviceSolve(w, batch=N, precision=precision)
    ds.reset()
    ds.walk(p0, N)
    u, d, st = ds.per_path(N)
    return u, d, st, int(ds.status[0].item())


def assert_same(a, b):
    (ua, da, sa, ka), (ub, db, sb, kb) = a, b
    assert ka == kb == 0
    assert np.array_equal(sa, sb)
    np.testing.assert_allclose(ua, ub, rtol=1e-12, atol=0)
    np.testing.assert_allclose(da, db, rtol=1e-12, atol=1e-300)


def test_two_calls_in_a_row_match_mcg_walk():
    # first call: sphere workload, 8 stations x 2000 paths
    w1 = W.sphere_line(paths=2000)
    assert_same(static_walk(w1, 0, 2000, M.MCG_MIXED), walk(w1, 0, 2000, M.MCG_MIXED))
    # second call: more paths, other indices and seed; the array still holds
    # the first call's records
    w2 = W.sphere_line(paths=3000, seed=7)
    assert_same(static_walk(w2, 5000, 3000, M.MCG_MIXED), walk(w2, 5000, 3000, M.MCG_MIXED))
    # the plain double-precision walk uses only the fixed work counter
    w3 = W.sphere_line(paths=500, seed=3)
    assert_same(static_walk(w3, 100, 500, M.MCG_FP64), walk(w3, 100, 500, M.MCG_FP64))


def test_rejects_requests_beyond_the_fixed_scratch():
    w = W.sphere_line()
    limit = M.mcg_walk_static_max_items()
    # 64 MiB less the counter's 256 bytes, three 32-byte exit records per path
    assert limit == ((64 << 20) - 256) // 96
    N = limit // w.n_stations + 1
    dev = torch.device("cuda")
    stations = torch.from_numpy(np.ascontiguousarray(w.stations)).to(dev)
    buf = torch.empty(1, dtype=torch.float64, device=dev)
    status = torch.zeros(2, dtype=torch.int32, device=dev)
    rc = M.mcg_walk_static(M.problem(w), stations, w.n_stations, 0, N, w.dt, w.seed, M.options(w), buf, buf,
                           buf, status, allow=(M.MCG_ERR_ARG,))
    assert rc == M.MCG_ERR_ARG
    assert "fixed scratch" in M.last_error()
