"""GPU set-up of the heterogeneous model against the oracle (through the C ABI).

* GRF density: element by element against the oracle's double-precision
  field; both sides take the same operations in the same order except the
  order of the mean / variance sums and exp (a few ulp), so the float grids
  agree to 2 ulp.
* Boundary tables: sampled nodes of every face against the oracle's exact
  direct prism sum over all voxels.  The GPU uses the exact prism within
  `near_cells` cell diagonals and the point-mass term beyond; for cubic cells
  the point-mass error is below (d/r)^4 / 10 per voxel at r >= 4 diagonals,
  i.e. < 5e-6 relative of a node value; the tolerance adds float rounding.
* Walk on the voxel model (grid from the oracle, smooth synthetic tables as
  plain input): per-path FP64 parity and the mixed paired test.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1709_07469_gb300 import build as B
from paper_1709_07469_gb300 import mcgrav as M
from paper_1709_07469_gb300 import workloads as W
from paper_1709_07469_gb300.device import DeviceSolve, packed, voxel_model
from tests.helpers import oracle_spec, smooth_tables

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    M.load()


def gpu_grf(seed, nx, ny, nz, sigma, amp=300.0):
    grid = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    work = torch.empty(M.mcg_grf_work_bytes(nx, ny, nz), dtype=torch.uint8, device="cuda")
    M.mcg_grf_density(seed, nx, ny, nz, sigma, amp, grid, work)
    torch.cuda.synchronize()
    return grid.cpu().numpy()


@pytest.mark.parametrize("shape,sigma", [((128, 128, 64), 5.0), ((37, 29, 11), 1.7)])
def test_grf_matches_oracle(shape, sigma):
    nx, ny, nz = shape
    got = gpu_grf(5, nx, ny, nz, sigma)
    want = oracle.grf_density(5, nx, ny, nz, sigma_vox=sigma, amp=300.0)
    ulp = np.spacing(np.abs(want).astype(np.float32))
    assert np.all(np.abs(got - want) <= 2 * ulp + 1e-6)


def test_tables_full_size_sampled_nodes():
    w = W.voxel_survey()
    grid, faces = voxel_model(w)
    torch.cuda.synchronize()
    g = grid.cpu().numpy()
    want_grid = oracle.grf_density(w.grid_seed, *w.grid_shape, sigma_vox=w.grid_sigma_vox, amp=w.grid_amp)
    assert np.array_equal(g, want_grid) or np.max(np.abs(g - want_grid) / np.spacing(np.abs(want_grid))) <= 2
    f = faces.cpu().numpy()
    nu, nv = w.table_n
    rng = np.random.default_rng(1)
    fi = np.repeat(np.arange(6), 4)
    iu = np.array([v for _ in range(6) for v in (0, nu - 1, *rng.integers(0, nu, 2))])
    iv = np.array([v for _ in range(6) for v in (nv - 1, 0, *rng.integers(0, nv, 2))])
    spec = oracle_spec(w.with_(g_kind="zero"), grid=want_grid)   # the oracle's own grid
    want = oracle.table_nodes(spec, fi, iu, iv, nu, nv, threads=THREADS)
    got = f[fi, iv, iu].astype(np.float64)
    rel = np.abs(got - want) / np.abs(want)
    assert np.all(rel < 2e-5), rel.max()


def test_tables_all_exact_small_grid():
    """With the near zone covering every voxel the tables are the exact sum."""
    w = W.voxel_survey(shape=(16, 12, 8), table_n=(9, 7))
    og = oracle.grf_density(3, 16, 12, 8, sigma_vox=1.5, amp=300.0)
    grid = torch.from_numpy(og).cuda()
    nu, nv = w.table_n
    faces = torch.empty((6, nv, nu), dtype=torch.float32, device="cuda")
    M.mcg_boundary_tables(M.problem(w.with_(g_kind="zero"), grid=grid), nu, nv, 1e6, faces)
    torch.cuda.synchronize()
    f = faces.cpu().numpy()
    fi, iu, iv = np.meshgrid(np.arange(6), np.arange(nu), np.arange(nv), indexing="ij")
    spec = oracle_spec(w.with_(g_kind="zero"), grid=og)
    want = oracle.table_nodes(spec, fi.ravel(), iu.ravel(), iv.ravel(), nu, nv, threads=THREADS)
    got = f[fi.ravel(), iv.ravel(), iu.ravel()].astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=3e-7)


@pytest.fixture(scope="module")
def voxel_inputs():
    w = W.voxel_survey(paths=512)
    grid = oracle.grf_density(w.grid_seed, *w.grid_shape, sigma_vox=w.grid_sigma_vox, amp=w.grid_amp)
    faces = smooth_tables(w, scale=-1e-4)
    return w, grid, faces


def test_voxel_walk_fp64_per_path(voxel_inputs):
    w, grid, faces = voxel_inputs
    st = w.stations[[0, 17, 100, 255]]
    wg = w.with_(stations=st, paths=48)
    ds = DeviceSolve(wg, precision=M.MCG_FP64, grid=torch.from_numpy(grid).cuda(),
                     faces=torch.from_numpy(faces).cuda())
    ds.reset()
    ds.walk(1000)
    u, d, steps = ds.per_path()
    assert int(ds.status[0].item()) == 0
    ref = oracle.solve(oracle_spec(wg, grid=grid, faces=faces), st, 48, p0=1000, per_path=True, threads=THREADS)
    same = steps == ref.pp_steps
    assert same.mean() >= 0.99
    assert np.all(np.abs(u - ref.pp_u)[same] <= 1e-12 * np.abs(ref.pp_u)[same])
    assert np.all(np.abs(d - ref.pp_d)[same] <= 1e-12 * np.abs(ref.pp_u)[same] / w.h)


def test_voxel_walk_mixed_paired(voxel_inputs):
    w, grid, faces = voxel_inputs
    st = w.stations[[3, 60, 130, 250]]
    wg = w.with_(stations=st, paths=512)
    ds = DeviceSolve(wg, precision=M.MCG_MIXED, grid=torch.from_numpy(grid).cuda(),
                     faces=torch.from_numpy(faces).cuda())
    ds.reset()
    ds.walk(0)
    u, d, steps = ds.per_path()
    assert int(ds.status[0].item()) == 0
    ref = oracle.solve(oracle_spec(wg, grid=grid, faces=faces, ubits=23), st, 512, per_path=True, threads=THREADS)
    assert (steps == ref.pp_steps).mean() > 0.9
    for s in range(st.shape[0]):
        diff = u[s] - ref.pp_u[s]
        se = diff.std(ddof=1) / math.sqrt(diff.size)
        um = abs(ref.pp_u[s].mean())
        assert abs(diff.mean()) <= 4 * se + 1e-6 * um, (s, diff.mean(), se)


def test_large_survey_full_size_sampled_paths(voxel_inputs):
    """The 2 x 10^4-station survey in one launch (8 paths per station, mixed
    precision); sampled (station, path) pairs are walked one by one by the
    oracle under the same station and path indices (same random streams, the
    23-bit uniforms of the single-precision walk)."""
    _, grid, faces = voxel_inputs
    w = W.large_survey(paths=8)
    ds = DeviceSolve(w, batch=8, precision=M.MCG_MIXED, grid=torch.from_numpy(grid).cuda(),
                     faces=torch.from_numpy(faces).cuda())
    ds.reset()
    ds.walk(0)
    u, d, steps = ds.per_path()
    assert int(ds.status[0].item()) == 0 and u.shape == (20000, 8)
    spec = oracle_spec(w, grid=grid, faces=faces, ubits=23)
    same, rel = [], []
    for s in (0, 9999, 10000, 19999, 4321, 15678):
        for p in range(8):
            rc, uc, st, _ = oracle.walk_path(spec, w.stations[s], s, p)
            assert rc == 0
            same.append(st.sum() == steps[s, p])
            if same[-1]:
                rel.append(abs(u[s, p] - uc[0]) / abs(uc[0]))
    assert np.mean(same) > 0.8
    assert np.median(rel) < 1e-5


def test_autotune_picks_a_valid_launch_shape():
    w = W.sphere_line()
    ds = DeviceSolve(w, precision=M.MCG_MIXED)
    M.mcg_autotune(ds.prob, ds.stations, ds.S, w.dt, w.seed, ds.opts)
    assert ds.opts.block in (64, 96, 128) and ds.opts.refill_min in (1, 4, 16)
    assert ds.opts.spill_max in (8, 16, 24, 32)
    r = ds.run()
    assert r["status"] == 0


def test_voxel_survey_against_the_exact_potential():
    """The heterogeneous-model workload end to end (GPU-built GRF density and
    boundary tables, mixed walk, 2e5 paths at 8 survey stations) against the
    exact potential and g_z of the voxel model at the stations (direct prism
    sums, oracle).  g_z agrees within 4 SE.  u carries the O(sqrt dt) bias of
    the discrete walk (monitoring of the exit and of the density jumps):
    within 4 SE + 0.5 % at a 10 m step, and halving the step shrinks it."""
    devs = {}
    for step in (10.0, 5.0):
        w = W.voxel_survey(paths=200_000, step=step)
        grid, faces = voxel_model(w)
        st = w.stations[[0, 37, 100, 135, 170, 200, 230, 255]]
        r = DeviceSolve(w, stations=st, batch=50_000, precision=M.MCG_MIXED, grid=grid, faces=faces).run()
        assert r["status"] == 0
        if step == 10.0:   # exact field of the oracle's own grid (the GPU grid agrees to 2 ulp)
            og = oracle.grf_density(w.grid_seed, *w.grid_shape, sigma_vox=w.grid_sigma_vox, amp=w.grid_amp)
            phi, gz = oracle.voxel_field(oracle_spec(w.with_(g_kind="zero"), grid=og), st, threads=THREADS,
                                         want_gz=True)
        assert np.all(np.abs(r["gz"] - gz) < 4 * r["se_gz"] + 1e-3 * np.abs(gz))
        assert np.all(np.abs(r["u"] - phi) < 4 * r["se_u"] + 5e-3 * np.abs(phi))
        devs[step] = float(np.mean(np.abs(r["u"] - phi) / np.abs(phi)))
    assert devs[5.0] < 0.75 * devs[10.0], devs


def test_mcgrav_solve_takes_host_or_device_model_arrays(voxel_inputs):
    """mcgrav_solve accepts the voxel grid and the boundary tables in host
    memory (staged into its workspace) as well as on the device: the same
    walks either way.  Path counts and steps are identical; with a voxel
    density the single-precision partial sums are flushed at schedule-
    dependent steps, so the statistics agree to rounding (1e-5 relative)."""
    w, grid, faces = voxel_inputs
    st = w.stations[[5, 77]]
    opts = M.options(w, precision=M.MCG_MIXED)
    host = M.mcgrav_solve(M.problem(w, grid=grid, faces=faces), st, 2048, w.dt, w.seed, opts)
    gd, fd = torch.from_numpy(grid).cuda(), torch.from_numpy(faces).cuda()
    dev = M.mcgrav_solve(M.problem(w, grid=gd, faces=fd), st, 2048, w.dt, w.seed, opts)
    for k in ("n_paths", "path_steps"):
        assert np.array_equal(getattr(host, k), getattr(dev, k)), k
    for k in ("u", "gz", "se_u", "se_gz"):
        np.testing.assert_allclose(getattr(host, k), getattr(dev, k), rtol=1e-5, err_msg=k)


def test_packed_arrays_layout(voxel_inputs):
    """mcg_voxel_pack: entry (iz + 1, iy, ix) holds layers iz-1, iz, iz+1 of
    the column (0 outside the grid); mcg_table_pack: entry (f, iv, iu) holds
    the four corners of that table cell."""
    w, grid, faces = voxel_inputs
    nz, ny, nx = grid.shape
    zp, tq = packed(w, torch.from_numpy(grid).cuda(), torch.from_numpy(faces).cuda())
    torch.cuda.synchronize()
    zp = zp.cpu().numpy().reshape(nz + 2, ny, nx, 4)
    pad = np.zeros((nz + 4, ny, nx), dtype=np.float32)
    pad[2:nz + 2] = grid
    for d in range(3):
        assert np.array_equal(zp[..., d], pad[d:d + nz + 2])
    assert np.all(zp[..., 3] == 0)
    nv, nu = faces.shape[1:]
    tq = tq.cpu().numpy().reshape(6, nv - 1, nu - 1, 4)
    assert np.array_equal(tq[..., 0], faces[:, :-1, :-1]) and np.array_equal(tq[..., 1], faces[:, :-1, 1:])
    assert np.array_equal(tq[..., 2], faces[:, 1:, :-1]) and np.array_equal(tq[..., 3], faces[:, 1:, 1:])


def test_packed_walks_read_the_same_values(voxel_inputs):
    """The 16-byte packed reads give the walk the same densities and table
    values as the scalar reads: the FP64 walk (packed tables) is bit-identical
    path by path; the mixed walk (packed grid and tables) has identical exit
    steps and u, d equal up to the schedule-dependent flush rounding of its
    single-precision partial sums (4e-6 of max |u|, as with migration)."""
    w, grid, faces = voxel_inputs
    g, f = torch.from_numpy(grid).cuda(), torch.from_numpy(faces).cuda()
    wg = w.with_(stations=w.stations[[2, 90, 171, 240]], paths=2048)
    out = {}
    for prec in (M.MCG_FP64, M.MCG_MIXED):
        for pack in (True, False):
            n = 64 if prec == M.MCG_FP64 else 2048
            ds = DeviceSolve(wg, batch=n, precision=prec, grid=g, faces=f, pack=pack)
            assert (ds.prob.density.zpack is not None) == pack
            ds.reset()
            ds.walk(0)
            out[prec, pack] = ds.per_path() + (int(ds.status[0].item()),)
    a, b = out[M.MCG_FP64, True], out[M.MCG_FP64, False]
    assert a[3] == 0 and b[3] == 0
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    a, b = out[M.MCG_MIXED, True], out[M.MCG_MIXED, False]
    assert a[3] == 0 and b[3] == 0
    assert np.array_equal(a[2], b[2])
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=4e-6 * np.abs(b[0]).max())
    np.testing.assert_allclose(a[1], b[1], rtol=0, atol=4e-6 * np.abs(b[0]).max() / w.h)
