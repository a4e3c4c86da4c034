"""mcg_density_at: the walks' own density samplers (Sec. 2.3 step 3: rho at
the walk's points; half-open cells, 0 outside) against the oracle's density,
point by point, at the points and at their common-random-number copies
z + h, z - h.  Interior points, exact cell faces, copies that cross a layer,
points outside the grid, and points far outside it (beyond 2^22 cells, where
the single-precision cell index is read from the bits of a float) for the
voxel grid, plain and packed; the sphere and the prism on exact faces.  The
coordinates sit on a binary grid, so the single-precision sampler's
arithmetic is exact and must pick the oracle's cell everywhere."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_07469_gb300 import build as B
from paper_1709_07469_gb300 import mcgrav as M
from paper_1709_07469_gb300 import workloads as W
from paper_1709_07469_gb300.device import packed
from tests.helpers import oracle_spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    M.load()


def sample(prob, pts, h, precision):
    x = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float64)).cuda()
    out = torch.empty(3 * len(pts), dtype=torch.float64, device="cuda")
    M.mcg_density_at(prob, h, precision, x, len(pts), out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(-1, 3)


def oracle_rho(w, pts, h, grid=None):
    spec = oracle_spec(w, grid=grid)
    return np.array([[oracle.rho(spec, (p[0], p[1], p[2] + o)) for o in (0.0, h, -h)] for p in pts])


def small_voxel():
    """8 x 6 x 5 cells of 0.5 m from (-2, -1.5, -2), a distinct density per
    cell, in Omega = [-4, 4]^2 x [-4, 2] (centre z = -1)."""
    nx, ny, nz = 8, 6, 5
    w = W.voxel_survey(shape=(nx, ny, nz), table_n=(9, 9)).with_(
        g_kind="zero", lo=(-4.0, -4.0, -4.0), hi=(4.0, 4.0, 2.0), grid_origin=(-2.0, -1.5, -2.0),
        grid_spacing=(0.5, 0.5, 0.5), h=0.2)
    grid = (1.0 + np.arange(nx * ny * nz, dtype=np.float32)).reshape(nz, ny, nx)
    return w, grid


def binary_points():
    """Every point of the 0.125 m lattice over [-2.5, 2.5] x [-2, 2] x [-2.75, 1]
    (cell faces, interiors, the grid's outside), plus points far outside:
    2^22 cells and beyond on either side, 1e30, and a coordinate that
    overflows single precision."""
    a = np.arange(-2.5, 2.5 + 1e-9, 0.125)
    b = np.arange(-2.0, 2.0 + 1e-9, 0.125)
    c = np.arange(-2.75, 1.0 + 1e-9, 0.125)
    pts = np.stack(np.meshgrid(a, b, c, indexing="ij"), -1).reshape(-1, 3)
    far = []
    for t in (2.0**22, 2.0**22 + 1, 2.0**23, 2.0**24 + 3):
        for sgn in (1.0, -1.0):
            x = -2.0 + sgn * t * 0.5
            far += [[x, 0.25, -1.25], [0.25, x, -1.25], [0.25, 0.25, x]]
    far += [[1e30, 0.0, -1.0], [0.0, -1e30, -1.0], [0.0, 0.0, 1e300], [-1e300, 0.0, 0.0]]
    return np.concatenate([pts, np.array(far)])


def test_voxel_samplers_equal_the_oracle():
    w, grid = small_voxel()
    g = torch.from_numpy(grid).cuda()
    pts = binary_points()
    want = oracle_rho(w, pts, w.h, grid=grid)
    assert np.count_nonzero(want) > 1000 and np.count_nonzero(want == 0) > 1000
    plain = sample(M.problem(w, grid=g), pts, w.h, M.MCG_MIXED)
    np.testing.assert_array_equal(plain, want)
    zpack, _ = packed(w, g, None)
    assert zpack is not None
    torch.cuda.synchronize()
    pk = sample(M.problem(w, grid=g, zpack=zpack), pts, w.h, M.MCG_MIXED)
    np.testing.assert_array_equal(pk, want)
    f64 = sample(M.problem(w, grid=g), pts, w.h, M.MCG_FP64)
    np.testing.assert_array_equal(f64, want)


def test_voxel_copies_cross_layers_at_random_points():
    """Random points away from cell faces (more than 1e-3 cells, also for the
    copies), h = 0.2 m = 0.4 cells: about 40 % of the copies inside the grid
    sit in another layer than their point (31 % of all)."""
    w, grid = small_voxel()
    g = torch.from_numpy(grid).cuda()
    rng = np.random.default_rng(11)
    pts = rng.uniform((-2.2, -1.7, -2.4), (2.2, 1.7, 0.7), (20000, 3))
    org, sp = np.array(w.grid_origin), np.array(w.grid_spacing)
    keep = np.ones(len(pts), bool)
    for dz in (0.0, w.h, -w.h):
        t = (pts + np.array([0.0, 0.0, dz]) - org) / sp
        keep &= np.all(np.abs(t - np.round(t)) > 1e-3, axis=1)
    pts = pts[keep]
    want = oracle_rho(w, pts, w.h, grid=grid)
    assert np.mean(want[:, 1] != want[:, 0]) > 0.25 and np.mean(want[:, 2] != want[:, 0]) > 0.25
    zpack, _ = packed(w, g, None)
    torch.cuda.synchronize()
    for prob in (M.problem(w, grid=g), M.problem(w, grid=g, zpack=zpack)):
        np.testing.assert_array_equal(sample(prob, pts, w.h, M.MCG_MIXED), want)


@pytest.mark.parametrize("kind", ["prism", "sphere"])
def test_analytic_samplers_on_exact_faces(kind):
    if kind == "prism":
        w = W.prism_ore_body().with_(lo=(-4.0, -4.0, -4.0), hi=(4.0, 4.0, 2.0), plo=(-1.0, -0.5, -2.0),
                                     phi=(1.5, 1.0, -0.75), h=0.25)
    else:
        w = W.sphere_line().with_(lo=(-4.0, -4.0, -4.0), hi=(4.0, 4.0, 2.0), center=(0.5, -0.25, -1.0),
                                  radius=1.25, h=0.25)
    pts = binary_points()
    want = oracle_rho(w, pts, w.h)
    assert np.count_nonzero(want) > 500
    prob = M.problem(w)
    np.testing.assert_array_equal(sample(prob, pts, w.h, M.MCG_MIXED), want)
    np.testing.assert_array_equal(sample(prob, pts, w.h, M.MCG_FP64), want)


def test_edge_cases():
    w, grid = small_voxel()
    g = torch.from_numpy(grid).cuda()
    assert M.mcg_density_at(M.problem(w, grid=g), w.h, M.MCG_MIXED, None, 0, None) == M.MCG_OK
    none = W.unit_box([[0.0, 0.0, 0.0]]).with_(rho_kind="none")
    np.testing.assert_array_equal(sample(M.problem(none), np.zeros((5, 3)), 0.01, M.MCG_MIXED), 0.0)
