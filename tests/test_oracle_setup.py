"""Pins of the oracle's heterogeneous-model set-up (CPU only).

* Gaussian random field: the smoothed field is rescaled to zero mean and unit
  population variance exactly; white noise smoothed by a normalised Gaussian
  of std sigma has autocorrelation exp(-d^2 / (4 sigma^2)) at lag d (the
  convolution of two Gaussians), checked on a grid large enough for the
  sampling error; rho = amp (exp(Z) - 1) exactly; the noise itself is the
  Box-Muller output of the documented counters.
* Boundary-table nodes by direct prism summation: a grid of constant density
  equals the closed form of the union prism (additivity of the potential); a
  single non-zero voxel equals that voxel's prism; nodes lie on the faces.
"""
import math

import numpy as np
import pytest

import oracle


def test_grf_normalised_and_transformed():
    grid, z = oracle.grf_density(seed=3, nx=24, ny=20, nz=16, sigma_vox=2.0, amp=300.0, want_z=True)
    assert abs(z.mean()) < 1e-12
    assert abs(z.std() - 1.0) < 1e-12
    np.testing.assert_allclose(grid, (300.0 * np.expm1(z)).astype(np.float32), rtol=2e-7, atol=1e-4)


def test_grf_noise_is_documented_box_muller():
    """A tiny smoothing width leaves the (rescaled) white noise: compare with
    Box-Muller of counters (q, 0, 0, 1), voxels 4q..4q+3."""
    seed, nx, ny, nz = 11, 8, 4, 2
    _, z = oracle.grf_density(seed, nx, ny, nz, sigma_vox=0.05, amp=1.0, want_z=True)
    n = nx * ny * nz
    q = np.arange(n // 4, dtype=np.uint32)
    ctr = np.stack([q, 0 * q, 0 * q, 0 * q + 1], 1).astype(np.uint32)
    key = np.tile(np.array([seed, 0], dtype=np.uint32), (q.size, 1))
    w = oracle.philox(ctr, key).astype(np.float64)
    u = (w + 0.5) * 2.0**-32
    noise = np.empty((q.size, 4))
    for j in (0, 2):
        r = np.sqrt(-2 * np.log(u[:, j]))
        noise[:, j] = r * np.cos(2 * np.pi * u[:, j + 1])
        noise[:, j + 1] = r * np.sin(2 * np.pi * u[:, j + 1])
    noise = noise.reshape(-1)
    want = (noise - noise.mean()) / noise.std()
    np.testing.assert_allclose(z.reshape(-1), want, rtol=0, atol=1e-12)


def test_grf_autocorrelation_is_gaussian():
    """Bounds are ~4x the seed-to-seed spread of the estimator on this grid;
    a kernel of the wrong width (sigma sqrt 2) would miss lag 4 by 0.24."""
    sigma = 2.0
    _, z = oracle.grf_density(seed=7, nx=96, ny=96, nz=96, sigma_vox=sigma, amp=1.0, want_z=True)
    core = z[6:-6, 6:-6, 6:-6]  # away from the zero-padded edges
    core = core - core.mean()
    for d, tol in ((1, 0.01), (2, 0.03), (4, 0.06)):
        for axis in (0, 1, 2):
            a = np.moveaxis(core, axis, 0)
            c = np.mean(a[d:] * a[:-d]) / np.mean(a * a)
            want = math.exp(-d * d / (4 * sigma * sigma))
            assert abs(c - want) < tol, (d, axis, c, want)


def _spec(grid, origin, spacing, lo, hi, G=1.0):
    return oracle.Spec(lo=lo, hi=hi, rho_kind=oracle.RHO_VOXEL, G=G, grid=grid, origin=origin, spacing=spacing)


def test_table_nodes_constant_grid_equals_union_prism():
    grid = np.full((2, 3, 4), 250.0, dtype=np.float32)   # nz=2, ny=3, nx=4
    origin, spacing = (-40.0, -30.0, -50.0), (20.0, 20.0, 25.0)
    lo, hi = (-100.0, -100.0, -100.0), (100.0, 100.0, 50.0)
    spec = _spec(grid, origin, spacing, lo, hi)
    nu, nv = 5, 4
    faces = np.repeat(np.arange(6), 4)
    iu = np.tile([0, 1, 2, 4], 6)
    iv = np.tile([0, 3, 1, 2], 6)
    got = oracle.table_nodes(spec, faces, iu, iv, nu, nv)
    plo = origin
    phi = (origin[0] + 4 * 20.0, origin[1] + 3 * 20.0, origin[2] + 2 * 25.0)
    for q in range(faces.size):
        f = faces[q]
        k, a, b = f // 2, (1 if f // 2 == 0 else 0), (1 if f // 2 == 2 else 2)
        x = [0.0, 0.0, 0.0]
        x[k] = hi[k] if f % 2 else lo[k]
        x[a] = lo[a] + (hi[a] - lo[a]) * iu[q] / (nu - 1)
        x[b] = lo[b] + (hi[b] - lo[b]) * iv[q] / (nv - 1)
        want = oracle.prism_phi(1.0, 250.0, plo, phi, x)
        assert abs(got[q] - want) < 1e-10 * abs(want), (q, got[q], want)


def test_table_nodes_single_voxel():
    grid = np.zeros((3, 3, 3), dtype=np.float32)
    grid[1, 2, 0] = -120.0
    origin, spacing = (0.0, 0.0, 0.0), (10.0, 10.0, 10.0)
    lo, hi = (-50.0, -50.0, -50.0), (80.0, 80.0, 80.0)
    spec = _spec(grid, origin, spacing, lo, hi)
    got = oracle.table_nodes(spec, [5, 0], [3, 1], [2, 2], 7, 7)
    vlo, vhi = (0.0, 20.0, 10.0), (10.0, 30.0, 20.0)
    x_top = (lo[0] + 130.0 * 3 / 6, lo[1] + 130.0 * 2 / 6, 80.0)
    x_mx = (-50.0, lo[1] + 130.0 * 1 / 6, lo[2] + 130.0 * 2 / 6)
    assert abs(got[0] - oracle.prism_phi(1.0, -120.0, vlo, vhi, x_top)) < 1e-12
    assert abs(got[1] - oracle.prism_phi(1.0, -120.0, vlo, vhi, x_mx)) < 1e-12


def test_table_nodes_reject_bad_index():
    grid = np.ones((1, 1, 1), dtype=np.float32)
    spec = _spec(grid, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (-5.0,) * 3, (5.0,) * 3)
    with pytest.raises(ValueError):
        oracle.table_nodes(spec, [6], [0], [0], 4, 4)


def test_voxel_field_equals_prism_closed_form_for_a_uniform_block():
    grid = np.full((2, 2, 3), 400.0, dtype=np.float32)
    origin, spacing = (-30.0, -20.0, -60.0), (20.0, 20.0, 25.0)
    spec = _spec(grid, origin, spacing, (-500.0,) * 3, (500.0,) * 3)
    pts = np.array([[0.0, 0.0, 10.0], [50.0, -70.0, -20.0], [5.0, 3.0, -40.0]])
    phi, gz = oracle.voxel_field(spec, pts, want_gz=True)
    hi = (origin[0] + 60.0, origin[1] + 40.0, origin[2] + 50.0)
    for q, x in enumerate(pts):
        assert abs(phi[q] - oracle.prism_phi(1.0, 400.0, origin, hi, x)) < 1e-10 * abs(phi[q])
        assert abs(gz[q] - oracle.prism_gz(1.0, 400.0, origin, hi, x)) < 1e-9 * abs(gz[q]) + 1e-12
