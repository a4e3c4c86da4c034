"""mcg_field: the exact potential and dPhi/dz of the density models on the GPU
against the oracle's closed forms (sphere, Nagy's prism) and its direct sum of
voxel prisms.  The voxel kernel regroups that sum by grid node (one corner
evaluation per node), so it must equal the direct sum to rounding, at points
off, on and between grid nodes, including the boundary-table nodes."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_07469_gb300 import build as B
from paper_1709_07469_gb300 import mcgrav as M
from paper_1709_07469_gb300 import workloads as W
from tests.helpers import oracle_spec

pytestmark = pytest.mark.gpu
THREADS = 16


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    M.load()


def field(prob, pts):
    x = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float64)).cuda()
    n = x.shape[0]
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    gz = torch.empty(n, dtype=torch.float64, device="cuda")
    M.mcg_field(prob, x, n, phi, gz)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), gz.cpu().numpy()


def test_sphere_closed_form():
    w = W.sphere_line()
    rng = np.random.default_rng(0)
    pts = np.concatenate([rng.uniform(-1, 1, (200, 3)), rng.uniform(-0.25, 0.25, (50, 3)), w.stations])
    phi, gz = field(M.problem(w), pts)
    for x, p, g in zip(pts, phi, gz):
        assert p == pytest.approx(oracle.sphere_phi(1.0, 1.0, w.center, w.radius, x), rel=1e-14)
        assert g == pytest.approx(oracle.sphere_gz(1.0, 1.0, w.center, w.radius, x), rel=1e-13, abs=1e-16)


def test_prism_closed_form_incl_edges_and_faces():
    w = W.prism_ore_body()
    rng = np.random.default_rng(1)
    pts = [rng.uniform(-1000, 1000, 3) for _ in range(200)] + list(w.stations)
    # on the prism's face planes, edges and corners (the limit forms)
    for x in (-100.0, 0.0, 100.0):
        for y in (-100.0, 37.0, 100.0):
            for z in (-250.0, -150.0, -200.0, 0.0):
                pts.append([x, y, z])
    pts = np.array(pts)
    phi, gz = field(M.problem(w), pts)
    for x, p, g in zip(pts, phi, gz):
        want_p = oracle.prism_phi(w.G, w.rho0, w.plo, w.phi, x)
        want_g = oracle.prism_gz(w.G, w.rho0, w.plo, w.phi, x)
        assert p == pytest.approx(want_p, rel=1e-12)
        assert g == pytest.approx(want_g, rel=1e-11, abs=1e-12 * abs(want_p) / 100.0)


def _small_voxel():
    w = W.voxel_survey(shape=(16, 16, 8), table_n=(9, 9)).with_(g_kind="zero")
    grid = oracle.grf_density(5, 16, 16, 8, sigma_vox=1.5, amp=300.0)
    return w, grid


def test_voxel_node_sum_equals_direct_prism_sum():
    w, grid = _small_voxel()
    rng = np.random.default_rng(2)
    sp = np.array(w.grid_spacing)
    org = np.array(w.grid_origin)
    pts = [rng.uniform(w.lo, w.hi) for _ in range(24)]
    pts += [org + sp * np.array([3, 5, 8]), org + sp * np.array([16, 0, 4]),      # grid nodes
            org + sp * np.array([7.5, 2, 6.25]), [0.0, 0.0, 0.0], [12.5, -40.0, 150.0]]
    pts = np.array(pts)
    prob = M.problem(w, grid=torch.from_numpy(grid).cuda())
    phi, gz = field(prob, pts)
    ref_phi, ref_gz = oracle.voxel_field(oracle_spec(w.with_(g_kind="zero"), grid=grid), pts, threads=THREADS,
                                         want_gz=True)
    np.testing.assert_allclose(phi, ref_phi, rtol=1e-10)
    np.testing.assert_allclose(gz, ref_gz, rtol=1e-9, atol=1e-9 * np.abs(ref_gz).max())


def test_voxel_field_at_table_nodes():
    """The node-summation field at boundary-table nodes equals the oracle's
    direct-sum table nodes (the exact reference the walk's tables are built
    to approximate)."""
    w, grid = _small_voxel()
    nu, nv = w.table_n
    rng = np.random.default_rng(3)
    face = rng.integers(0, 6, 40)
    iu, iv = rng.integers(0, nu, 40), rng.integers(0, nv, 40)
    ref = oracle.table_nodes(oracle_spec(w.with_(g_kind="zero"), grid=grid), face, iu, iv, nu, nv,
                             threads=THREADS)
    pts = []
    for f, a, b in zip(face, iu, iv):
        k = f // 2
        ua, va = (1, 2) if k == 0 else ((0, 2) if k == 1 else (0, 1))
        x = [0.0, 0.0, 0.0]
        x[k] = w.hi[k] if f % 2 else w.lo[k]
        x[ua] = w.lo[ua] + (w.hi[ua] - w.lo[ua]) * a / (nu - 1)
        x[va] = w.lo[va] + (w.hi[va] - w.lo[va]) * b / (nv - 1)
        pts.append(x)
    phi, _ = field(M.problem(w, grid=torch.from_numpy(grid).cuda()), np.array(pts))
    np.testing.assert_allclose(phi, ref, rtol=1e-10)


def test_voxel_full_size_sampled_points():
    """The full 128 x 128 x 64 heterogeneous model at four survey stations."""
    w = W.voxel_survey().with_(g_kind="zero")
    grid = oracle.grf_density(w.grid_seed, *w.grid_shape, sigma_vox=w.grid_sigma_vox, amp=w.grid_amp)
    pts = w.stations[[0, 100, 187, 255]]
    phi, gz = field(M.problem(w, grid=torch.from_numpy(grid).cuda()), pts)
    ref_phi, ref_gz = oracle.voxel_field(oracle_spec(w.with_(g_kind="zero"), grid=grid), pts, threads=THREADS,
                                         want_gz=True)
    np.testing.assert_allclose(phi, ref_phi, rtol=1e-10)
    np.testing.assert_allclose(gz, ref_gz, rtol=1e-8)


def test_edge_cases():
    w = W.prism_ore_body()
    prob = M.problem(w)
    assert M.mcg_field(prob, None, 0, None, None) == M.MCG_OK
    none = M.problem(W.unit_box([[0.0, 0.0, 0.0]]).with_(rho_kind="none"))
    phi, gz = field(none, np.zeros((3, 3)))
    assert np.all(phi == 0.0) and np.all(gz == 0.0)
