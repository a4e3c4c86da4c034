"""GPU walk against the oracle, through the C ABI (the parity gate).

Tolerances:
* plain FP64 walk, per path: the two sides run the same operation sequence
  and differ only in the last bits of log / sin / cos, so where the exit step
  matches, |du| <= 1e-12 |u| and |dd| <= 1e-12 |u| / h (the centred
  difference divides by 2h); the fraction of paths whose exit step flips
  must stay below 1e-4;
* mixed walk, per path, against the oracle run on the same 23-bit uniforms:
  most paths agree to single-precision rounding; the paired mean difference
  must be within 4 standard errors of the differences plus the shift that
  single-precision inputs alone cause (station coordinates and step scale
  rounded to 2^-24 relative move u by ~1e-8 relative; allowance 1e-6 |u|,
  and 1e-6 |u| / h for the centred difference);
* station statistics: within 4 standard errors of the closed form where the
  estimator is exactly unbiased.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1709_07469_gb300 import build as B
from paper_1709_07469_gb300 import mcgrav as M
from paper_1709_07469_gb300 import workloads as W
from paper_1709_07469_gb300.device import DeviceSolve
from tests.helpers import oracle_spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    M.load()


def gpu_per_path(w, precision, paths=None, stations=None, p0=0, **kw):
    ds = DeviceSolve(w, stations=stations, batch=paths or w.paths, precision=precision, **kw)
    ds.reset()
    ds.walk(p0)
    u, d, st = ds.per_path()
    return u, d, st, int(ds.status[0].item())


def compare_fp64(w, paths, stations=None, p0=0):
    u, d, st, status = gpu_per_path(w, M.MCG_FP64, paths, stations, p0)
    assert status == 0
    S = u.shape[0]
    ref = oracle.solve(oracle_spec(w), w.stations if stations is None else stations, paths, p0=p0, per_path=True)
    same = st == ref.pp_steps
    flips = 1.0 - same.mean()
    tol_u = 1e-12 * np.abs(ref.pp_u)
    tol_d = 1e-12 * np.abs(ref.pp_u) / w.h + 1e-300
    assert np.all(np.abs(u - ref.pp_u)[same] <= tol_u[same])
    assert np.all(np.abs(d - ref.pp_d)[same] <= tol_d[same])
    return flips, S * paths


def test_fp64_per_path_sphere_line_full():
    """Sphere workload, all 8 stations x 2e4 paths (the full configuration)."""
    w = W.sphere_line()
    flips, n = compare_fp64(w, w.paths)
    assert flips < 1e-4, flips


def prism_rounding_bound(w, x, ulps=16):
    """Error bound of the prism's closed form at x from the rounding of its
    terms: `ulps` units of roundoff of the absolute sum of the 48 terms of
    Nagy's corner sum (Sec. 4.2), times G rho.  At exit points on the domain's
    faces that sum is up to ~3e4 |u|, so two correct evaluations that differ
    only in their log / atan implementations (CUDA's and the host's libm) or
    in fused multiply-adds differ by far more than 1e-12 |u|."""
    tot = 0.0
    for c in range(8):
        X, Y, Z = [(w.phi[k] if (c >> k) & 1 else w.plo[k]) - x[k] for k in range(3)]
        r = np.sqrt(X * X + Y * Y + Z * Z)
        for a, b, q in ((X, Y, Z), (Y, Z, X), (Z, X, Y)):
            if a * b != 0.0:  # ln(q + r), q + r = (a^2 + b^2) / (r - q) for q < 0
                ln = np.log(q + r) if q >= 0.0 else np.log(a * a + b * b) - np.log(r - q)
                tot += abs(a * b * ln)
            if a != 0.0:
                tot += abs(0.5 * a * a * np.arctan(b * q / (a * r)))
    return ulps * np.finfo(np.float64).eps * abs(w.G * w.rho0) * tot


def test_fp64_per_path_prism_sampled_paths():
    """Prism ore body (step 1 m, ~1.4e5 RNG-steps per path): all 30 stations x
    16 paths at the highest path indices of the full 10^6-path configuration
    (480 walks; the bench line checks paths 0-255 of every station).  Where
    the exit steps agree, u and d agree to 1e-12 |u| plus the closed form's
    own rounding bound at the copies' exit points."""
    w = W.prism_ore_body()
    N, p0 = 16, 999_984
    u, d, steps, status = gpu_per_path(w, M.MCG_FP64, N, p0=p0)
    assert status == 0
    spec = oracle_spec(w)
    flips, worst = 0, 0.0
    for s in range(w.n_stations):
        for j in range(N):
            rc, uc, st, xe = oracle.walk_path(spec, w.stations[s], s, p0 + j)
            assert rc == 0
            if st.sum() != steps[s, j]:
                flips += 1
                continue
            b = [prism_rounding_bound(w, xe[c]) for c in range(3)]
            tol_u = 1e-12 * abs(uc[0]) + b[0]
            tol_d = (2e-12 * abs(uc[0]) + b[1] + b[2]) / (2.0 * w.h)
            err_u = abs(u[s, j] - uc[0])
            err_d = abs(d[s, j] - (uc[1] - uc[2]) / (2.0 * w.h))
            assert err_u <= tol_u and err_d <= tol_d, (s, j, err_u, tol_u, err_d, tol_d)
            worst = max(worst, err_u / abs(uc[0]))
    print(f"max relative |u - oracle| over matched paths: {worst:.3e}; flips {flips} of {w.n_stations * N}")
    assert flips <= 1


@pytest.mark.parametrize("name,poly", [("linear", (0.3, 1.0, 2.0, -1.0, 0, 0, 0, 0, 0, 0, 0)),
                                       ("xyz", (0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 3.0))])
def test_fp64_per_path_harmonic_ragged(name, poly):
    """clip = 0 and crn on, a ragged path count (not a multiple of 32)."""
    st = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.5], [0.8, 0.7, -0.6]])
    w = W.unit_box(st, g_kind="poly", poly=poly, dt=0.02, paths=1001, clip=0, h=0.05)
    flips, n = compare_fp64(w, w.paths)
    assert flips < 1e-3


def test_mixed_vs_oracle_paired_sphere_line():
    w = W.sphere_line(paths=20000)
    u, d, st, status = gpu_per_path(w, M.MCG_MIXED)
    assert status == 0
    ref = oracle.solve(oracle_spec(w, ubits=23), w.stations, w.paths, per_path=True)
    same = st == ref.pp_steps
    assert same.mean() > 0.97, same.mean()
    rel = np.abs(u - ref.pp_u)[same] / np.abs(ref.pp_u)[same]
    assert np.quantile(rel, 0.99) < 1e-4
    for s in range(w.n_stations):
        diff = u[s] - ref.pp_u[s]
        se = diff.std(ddof=1) / math.sqrt(diff.size)
        um = abs(ref.pp_u[s].mean())
        assert abs(diff.mean()) <= 4 * se + 1e-6 * um, (s, diff.mean(), se)
        dd = d[s] - ref.pp_d[s]
        se_d = dd.std(ddof=1) / math.sqrt(dd.size)
        assert abs(dd.mean()) <= 4 * se_d + 1e-6 * um / w.h, (s, dd.mean(), se_d)
        # the shift is below a thousandth of the estimate's own standard error
        assert abs(diff.mean()) < 1e-3 * ref.pp_u[s].std(ddof=1) / math.sqrt(diff.size)


@pytest.mark.parametrize("precision", [M.MCG_FP64, M.MCG_MIXED])
def test_sphere_line_vs_closed_form(precision):
    w = W.sphere_line()
    r = DeviceSolve(w, precision=precision).run()
    assert r["status"] == 0
    Mass = 4 / 3 * math.pi * 0.25**3
    z = w.stations[:, 2]
    assert np.all(np.abs(r["u"] + Mass / z) < 4 * r["se_u"] + 2e-4), (r["u"] + Mass / z) / r["se_u"]
    assert np.all(np.abs(r["gz"] - Mass / z**2) < 4 * r["se_gz"])
    assert np.all(r["n_paths"] == w.paths)


@pytest.mark.parametrize("precision", [M.MCG_FP64, M.MCG_MIXED])
def test_station_statistics_match_oracle(precision):
    """Means, standard errors and step totals against the oracle's two-pass
    statistics on the same paths (FP64: 1e-12; mixed: within 4 SE)."""
    w = W.sphere_line(paths=5000)
    r = DeviceSolve(w, precision=precision, batch=1237).run()   # ragged batches
    ref = oracle.solve(oracle_spec(w, ubits=32 if precision == M.MCG_FP64 else 23), w.stations, w.paths)
    if precision == M.MCG_FP64:
        np.testing.assert_allclose(r["u"], ref.u, rtol=1e-11)
        np.testing.assert_allclose(r["se_u"], ref.se_u, rtol=1e-9)
        np.testing.assert_allclose(r["gz"], ref.gz, rtol=1e-9)
        assert np.array_equal(r["path_steps"], ref.path_steps)
    else:
        assert np.all(np.abs(r["u"] - ref.u) < 4 * ref.se_u)
        assert np.all(np.abs(r["gz"] - ref.gz) < 4 * ref.se_gz)
        np.testing.assert_allclose(r["se_u"], ref.se_u, rtol=0.05)


HARMONIC = [(0.3, 1.0, 2.0, -1.0, 0, 0, 0, 0, 0, 0, 0), (0, 0, 0, 0, 1.0, -1.0, 0, 0, 0, 0, 0),
            (0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 3.0), (0, 0, 0, 0, 1.0, 1.0, -2.0, 0, 0, 0, 0)]


def poly_eval(c, x):
    X, Y, Z = x
    return (c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * X + c[5] * Y * Y + c[6] * Z * Z
            + c[7] * X * Y + c[8] * Y * Z + c[9] * Z * X + c[10] * X * Y * Z)


@pytest.mark.parametrize("precision", [M.MCG_FP64, M.MCG_MIXED])
@pytest.mark.parametrize("k", range(4))
def test_harmonic_unbiased_gpu(precision, k):
    st = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.5], [0.8, 0.7, -0.6], [-0.9, 0.1, 0.85]])
    w = W.unit_box(st, g_kind="poly", poly=HARMONIC[k], dt=0.01, paths=200_000, clip=0, h=0.05)
    r = DeviceSolve(w, precision=precision).run()
    assert r["status"] == 0
    for s, x in enumerate(st):
        assert abs(r["u"][s] - poly_eval(HARMONIC[k], x)) < 4 * r["se_u"][s] + 1e-12
        want_d = (poly_eval(HARMONIC[k], x + [0, 0, w.h]) - poly_eval(HARMONIC[k], x - [0, 0, w.h])) / (2 * w.h)
        assert abs(r["gz"][s] - want_d) < 4 * r["se_gz"][s] + 1e-12


@pytest.mark.parametrize("precision", [M.MCG_FP64, M.MCG_MIXED])
def test_constant_density_quadratic_gpu(precision):
    A = 2 * math.pi / 3
    st = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.5], [0.8, 0.7, -0.6]])
    w = W.unit_box(st, rho_kind="prism", rho0=1.0, g_kind="poly", poly=(0, 0, 0, 0, A, A, A, 0, 0, 0, 0),
                   dt=0.01, paths=200_000, clip=0, h=0.05)
    r = DeviceSolve(w, precision=precision).run()
    for s, x in enumerate(st):
        assert abs(r["u"][s] - A * np.dot(x, x)) < 4 * r["se_u"][s]
        assert abs(r["gz"][s] - 2 * A * x[2]) < 4 * r["se_gz"][s] + 1e-12


def test_mcgrav_solve_matches_device_path_and_is_deterministic():
    w = W.sphere_line(paths=3000)
    prob = M.problem(w)
    a = M.mcgrav_solve(prob, w.stations, w.paths, w.dt, w.seed, M.options(w, batch_paths=3000))
    b = M.mcgrav_solve(prob, w.stations, w.paths, w.dt, w.seed, M.options(w, batch_paths=3000))
    c = DeviceSolve(w, precision=M.MCG_MIXED).run()
    for k in ("u", "gz", "se_u", "se_gz"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
        assert np.array_equal(getattr(a, k), c[k])
    assert np.array_equal(a.path_steps, c["path_steps"])
    # batching changes only the merge order of the statistics
    d = M.mcgrav_solve(prob, w.stations, w.paths, w.dt, w.seed, M.options(w, batch_paths=777))
    np.testing.assert_allclose(d.u, a.u, rtol=1e-12)
    assert np.array_equal(d.path_steps, a.path_steps)


def test_per_path_values_independent_of_launch_shape():
    w = W.sphere_line(paths=2000)
    u1, d1, s1, _ = gpu_per_path(w, M.MCG_MIXED, block=128)
    u2, d2, s2, _ = gpu_per_path(w, M.MCG_MIXED, block=32)
    assert np.array_equal(u1, u2) and np.array_equal(d1, d2) and np.array_equal(s1, s2)


def test_edge_cases():
    w = W.sphere_line(paths=1)
    r = M.mcgrav_solve(M.problem(w), w.stations[:1], 1, w.dt, w.seed, M.options(w))
    assert r.n_paths[0] == 1 and math.isnan(r.se_u[0])
    r = M.mcgrav_solve(M.problem(w), np.zeros((0, 3)), 5, w.dt, w.seed, M.options(w))
    assert r.u.size == 0
    # step cap: every path stopped early -> status and NaN
    w = W.sphere_line(paths=64)
    r = M.mcgrav_solve(M.problem(w), w.stations, 64, w.dt, w.seed, M.options(w, max_steps=8),
                       allow=(M.MCG_ERR_STEP_CAP,))
    assert r.status == M.MCG_ERR_STEP_CAP and np.all(np.isnan(r.u))
    # no common random numbers: g_z is NaN, u unchanged vs the crn run
    a = M.mcgrav_solve(M.problem(w), w.stations, 64, w.dt, w.seed, M.options(w))
    b = M.mcgrav_solve(M.problem(w), w.stations, 64, w.dt, w.seed, M.options(w, crn_gz=0))
    assert np.all(np.isnan(b.gz)) and np.array_equal(a.u, b.u)


def test_device_station_outside_flags_status():
    w = W.sphere_line(paths=32)
    st = w.stations.copy()
    st[3] = [0.0, 0.0, 1.5]
    ds = DeviceSolve(w, stations=st, precision=M.MCG_MIXED)
    ds.reset()
    ds.walk(0)
    u, d, s, status = *ds.per_path(), int(ds.status[0].item())
    assert status & (1 << M.MCG_ERR_ARG)
    assert np.all(np.isnan(u[3])) and np.all(np.isfinite(u[[0, 1, 2, 4, 5, 6, 7]]))


# --- Brownian-bridge exit test ------------------------------------------------

def test_bridge_fp64_per_path():
    """Stations near faces (where the bridge acts) and the sphere line, FP64
    walk per path against the oracle with the bridge on."""
    st = np.array([[0.95, 0.2, 0.0], [0.1, -0.93, 0.4], [0.0, 0.0, 0.0]])
    w = W.unit_box(st, g_kind="poly", poly=HARMONIC[1], dt=2e-3, paths=2000, clip=1, h=0.02).with_(bridge=1)
    flips, _ = compare_fp64(w, w.paths)
    assert flips < 1e-3
    w = W.sphere_line(paths=2000).with_(bridge=1)
    flips, _ = compare_fp64(w, w.paths)
    assert flips < 1e-3


def test_bridge_mixed_paired():
    w = W.sphere_line(paths=20000).with_(bridge=1)
    u, d, st, status = gpu_per_path(w, M.MCG_MIXED)
    assert status == 0
    ref = oracle.solve(oracle_spec(w, ubits=23), w.stations, w.paths, per_path=True)
    assert (st == ref.pp_steps).mean() > 0.95
    for s in range(w.n_stations):
        diff = u[s] - ref.pp_u[s]
        se = diff.std(ddof=1) / math.sqrt(diff.size)
        assert abs(diff.mean()) <= 4 * se + 1e-6 * abs(ref.pp_u[s].mean()), (s, diff.mean(), se)


@pytest.mark.parametrize("precision", [M.MCG_FP64, M.MCG_MIXED])
def test_bridge_slab_exit_time_gpu(precision):
    """E[N dt] of the slab equals (a - z)(a + z) without overshoot correction."""
    a = 0.5
    st = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.3]])
    w = W.Workload(name="slab", lo=(-20.0, -20.0, -a), hi=(20.0, 20.0, a), rho_kind="prism", g_kind="zero",
                   G=1.0, stations=st, dt=1e-3, h=0.01, seed=5, paths=200_000 if precision else 50_000,
                   rho0=1.0, plo=(-100.0,) * 3, phi=(100.0,) * 3, clip=0, crn=0, bridge=1)
    r = DeviceSolve(w, precision=precision).run()
    for s, z in enumerate(st[:, 2]):
        got, se = -r["u"][s] / (2 * math.pi), r["se_u"][s] / (2 * math.pi)
        assert abs(got - (a - z) * (a + z)) < 4 * se + 2e-4, (z, got, se)


# --- ball domain (the paper's own Omega) -------------------------------------

def _ball_cube(paths, dt=1e-4, a=0.05):
    st = np.array([[0.0, 0.0, 0.3], [0.25, 0.0, -0.2], [0.0, 0.0, 0.6]])
    return W.Workload(name="ball", lo=(-1.0,) * 3, hi=(1.0,) * 3, rho_kind="prism", g_kind="zero", G=1.0,
                      stations=st, dt=dt, h=0.01, seed=4, paths=paths, rho0=1.0, plo=(-a,) * 3, phi=(a,) * 3,
                      domain="ball", ball_radius=1.0)


def test_ball_fp64_per_path():
    flips, _ = compare_fp64(_ball_cube(400), 400)
    assert flips < 1e-3


def test_ball_mixed_paired():
    w = _ball_cube(4000)
    u, d, st, status = gpu_per_path(w, M.MCG_MIXED)
    assert status == 0
    ref = oracle.solve(oracle_spec(w, ubits=23), w.stations, w.paths, per_path=True)
    assert (st == ref.pp_steps).mean() > 0.9
    for s in range(w.n_stations):
        diff = u[s] - ref.pp_u[s]
        se = diff.std(ddof=1) / math.sqrt(diff.size)
        assert abs(diff.mean()) <= 4 * se + 1e-6 * abs(ref.pp_u[s].mean())


@pytest.mark.parametrize("precision", [M.MCG_MIXED])
def test_ball_zero_data_offset_GM_over_R_gpu(precision):
    """Sec. 2.2: zero Dirichlet data on the ball adds G M / R to the potential
    (a constant) and leaves g_z alone -- at 2e5 paths per station."""
    a = 0.05
    w = _ball_cube(200_000, a=a)
    r = DeviceSolve(w, precision=precision).run()
    assert r["status"] == 0
    M_ = (2 * a) ** 3
    for s, x in enumerate(w.stations):
        phi = oracle.prism_phi(1.0, 1.0, (-a,) * 3, (a,) * 3, x)
        gz = oracle.prism_gz(1.0, 1.0, (-a,) * 3, (a,) * 3, x)
        assert abs(r["u"][s] - (phi + M_)) < 4 * r["se_u"][s] + 2e-5
        assert r["u"][s] - phi > 20 * r["se_u"][s]
        assert abs(r["gz"][s] - gz) < 4 * r["se_gz"][s] + 2e-4 * abs(gz)


def test_paper_experiment_1_line():
    """The paper's experiment 1 geometry (cube [0,100]^3 m, 2000 kg/m^3, ball
    of 10 km, zero data, 31 stations on y = 50, z = 200): FP64 per path on a
    sample, and the mixed estimate against Phi_cube + G M / R (the paper's
    ~1 % offset) within 4 SE plus the time-step bias of a 20 m step."""
    w = W.paper_cube_ball(paths=8192)
    flips, _ = compare_fp64(w.with_(stations=w.stations[[0, 15, 30]]), 2)
    assert flips <= 1.0 / 6 + 1e-12
    r = DeviceSolve(w, precision=M.MCG_MIXED).run()
    assert r["status"] == 0
    Mass = 2000.0 * 100.0**3
    off = W.G_SI * Mass / 10_000.0
    phi = np.array([oracle.prism_phi(W.G_SI, 2000.0, (0, 0, 0), (100, 100, 100), x) for x in w.stations])
    rel_offset = off / np.abs(phi)
    assert np.all((rel_offset > 0.008) & (rel_offset < 0.03))     # the paper's offset of about 1 %
    assert np.all(np.abs(r["u"] - (phi + off)) < 4 * r["se_u"] + 0.01 * np.abs(phi))


def test_mcgrav_solve_graph_equals_stream_launches():
    """Several batches (the last one ragged) alternate between two streams
    inside mcgrav_solve; captured into one CUDA graph or issued directly,
    they give the same numbers as the same batches run one after another on
    one stream through the device-level entry points (same per-path values,
    reductions in batch order)."""
    w = W.sphere_line(paths=6500)
    prob = M.problem(w)
    a = M.mcgrav_solve(prob, w.stations, w.paths, w.dt, w.seed, M.options(w, batch_paths=1000, graph=1))
    b = M.mcgrav_solve(prob, w.stations, w.paths, w.dt, w.seed, M.options(w, batch_paths=1000, graph=0))
    ds = DeviceSolve(w, batch=1000, precision=M.MCG_MIXED)
    c = ds.run()
    for k in ("u", "gz", "se_u", "se_gz", "n_paths", "path_steps"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
        assert np.array_equal(getattr(a, k), c[k]), k
    assert np.all(a.n_paths == 6500)


def _per_path_migrate(w, migrate, **kw):
    ds = DeviceSolve(w, precision=M.MCG_MIXED, **kw)
    ds.opts.migrate = migrate
    ds.reset()
    ds.work.fill_(255)   # stale pool flags must not read as ready
    ds.walk(0)
    u, d, st = ds.per_path()
    return u, d, st, int(ds.status[0].item())


@pytest.mark.parametrize("name,w", [
    # fewer walks than lanes: the work list is used up at once and warps spill from the start
    ("prism, 30 x 512", W.prism_ore_body(paths=512)),
    # a few walks per lane, then the exit-time tail
    ("prism, 30 x 8192", W.prism_ore_body(paths=8192)),
    # less than one warp of work, and a ragged count
    ("prism, 3 x 7", W.prism_ore_body(paths=7).with_(stations=W.prism_ore_body().stations[:3])),
    ("sphere, 8 x 20000", W.sphere_line(paths=20000)),
])
def test_migration_leaves_every_path_unchanged(name, w):
    """Walks handed between warps keep their numbers: with a piecewise-constant
    density the partial sums are exact, so every per-path value is bit-identical
    with and without migration."""
    a = _per_path_migrate(w, 1)
    b = _per_path_migrate(w, 0)
    assert a[3] == 0 and b[3] == 0
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    assert np.all(np.isfinite(a[0])) and np.all(a[2] > 0)


def test_migration_voxel_rounding_only():
    """Voxel density: migration moves the flush points of the single-precision
    partial sums, which changes u by rounding only; exit steps are identical.
    A flush of up to 64 single-precision terms carries a relative error of at
    most 64 * 2^-24 ~ 4e-6 of the source integral, whose term in u is below
    max |u| here; the allowance is 4e-6 max |u|, absolute (u itself can be
    near zero where g and the integral cancel)."""
    from tests.helpers import smooth_tables
    w = W.voxel_survey(shape=(32, 32, 16), table_n=(33, 33), paths=256, n_side=8)
    grid = torch.from_numpy(oracle.grf_density(1, 32, 32, 16, sigma_vox=2.0, amp=300.0)).cuda()
    faces = torch.from_numpy(smooth_tables(w, scale=-1e-4)).cuda()
    a = _per_path_migrate(w, 1, grid=grid, faces=faces)
    b = _per_path_migrate(w, 0, grid=grid, faces=faces)
    assert a[3] == 0 and b[3] == 0
    assert np.array_equal(a[2], b[2])
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=4e-6 * np.abs(b[0]).max())
    assert np.mean(a[0] == b[0]) > 0.2   # paths that never migrated are bit-identical


def test_prism_full_size_launch_sampled_paths_mixed():
    """The benchmark's launch: prism ore body, 30 stations x 131072 paths in one
    mixed-precision launch (migration on), at a path range of a later step.
    Sampled (station, path) pairs are walked one by one by the oracle under
    the same indices and the 23-bit uniforms of the single-precision walk:
    most exit steps agree exactly, and where they do u agrees to single-
    precision rounding of ~1e5 steps."""
    w = W.prism_ore_body()
    N, p0 = 131072, 5 * 131072
    ds = DeviceSolve(w, batch=N, precision=M.MCG_MIXED)
    ds.reset()
    ds.walk(p0)
    u, d, steps = ds.per_path()
    assert int(ds.status[0].item()) == 0
    assert np.all(np.isfinite(u)) and np.all(steps > 0)
    spec = oracle_spec(w, ubits=23)
    rng = np.random.default_rng(3)
    picks = [(0, 0), (29, N - 1), (14, N // 2)] + [(int(a), int(b)) for a, b in
                                                 zip(rng.integers(0, 30, 37), rng.integers(0, N, 37))]
    same, rel = [], []
    for s, j in picks:
        rc, uc, st, _ = oracle.walk_path(spec, w.stations[s], s, p0 + j)
        assert rc == 0
        same.append(st.sum() == steps[s, j])
        if same[-1]:
            rel.append(abs(u[s, j] - uc[0]) / abs(uc[0]))
    assert np.mean(same) > 0.8
    assert np.median(rel) < 1e-5


def test_largest_path_indices_and_seed():
    """The last 40 path indices a launch may use (p0 + N = 2^32) under the
    all-ones seed (key words 0xFFFFFFFF): the FP64 walk equals the oracle path
    by path, and the mixed walk follows the oracle's 23-bit-uniform walk of
    the same indices (same exit step for most paths, u to single-precision
    rounding where it does)."""
    w = W.sphere_line().with_(seed=2**64 - 1)
    N, p0 = 40, 2**32 - 40
    flips, n = compare_fp64(w, N, p0=p0)
    assert flips * n <= 1.0 + 1e-9, flips * n
    u, d, steps, status = gpu_per_path(w, M.MCG_MIXED, N, p0=p0)
    assert status == 0
    spec = oracle_spec(w, ubits=23)
    same, rel = [], []
    for s in range(w.n_stations):
        for j in range(N):
            rc, uc, st, _ = oracle.walk_path(spec, w.stations[s], s, p0 + j)
            assert rc == 0
            same.append(st.sum() == steps[s, j])
            if same[-1]:
                rel.append(abs(u[s, j] - uc[0]) / abs(uc[0]))
    assert np.mean(same) > 0.8
    assert np.median(rel) < 1e-4
