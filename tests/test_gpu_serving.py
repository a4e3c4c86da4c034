"""Continuous batching (mcg_server_*): requests of different station counts,
models and targets overlap on the GPU; each result must be the same alone and
in the mix (bit for bit: a request's paths, chunks and merge order depend only
on its own seed, stations and target), equal to the device-level solve with
the same chunking, stop at its target, and honour cancellation and the HBM
budget.  Rounds of compatible requests share walk launches (a segment table
gives each walk its request's stations, seed and model arrays): the results
equal those of a server that launches every round alone."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1709_07469_gb300 import build as B
from paper_1709_07469_gb300 import mcgrav as M
from paper_1709_07469_gb300 import workloads as W
from paper_1709_07469_gb300.device import DeviceSolve
from tests.helpers import smooth_tables

pytestmark = pytest.mark.gpu
CHUNK = 2048


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    M.load()


@pytest.fixture(scope="module")
def models():
    sph = W.sphere_line()
    pri = W.prism_ore_body()
    vox = W.voxel_survey(shape=(32, 32, 16), table_n=(33, 33))
    grid = oracle.grf_density(1, 32, 32, 16, sigma_vox=2.0, amp=300.0)
    faces = smooth_tables(vox, scale=-1e-4)
    grid2 = oracle.grf_density(2, 32, 32, 16, sigma_vox=2.0, amp=300.0)   # same geometry, other grid
    faces2 = smooth_tables(vox, seed=5, scale=-1e-4)
    m = {"sphere": (sph, M.mcg_model_create(M.problem(sph), sph.dt, sph.h)),
         "prism": (pri, M.mcg_model_create(M.problem(pri), pri.dt, pri.h)),
         "voxel": (vox, M.mcg_model_create(M.problem(vox, grid=grid, faces=faces), vox.dt, vox.h)),
         "voxel2": (vox, M.mcg_model_create(M.problem(vox, grid=grid2, faces=faces2), vox.dt, vox.h))}
    yield m
    for _, h in m.values():
        M.mcg_model_destroy(h)


def server(w, **kw):
    cfg = M.server_config(M.options(w), chunk_paths=CHUNK, min_paths=2 * CHUNK, **kw)
    return M.mcg_server_create(cfg)


def run_alone(w, model, stations, target, seed):
    sv = server(w)
    try:
        rq = M.mcg_submit(sv, model, stations, target, seed)
        rc, out = M.mcg_wait(rq, len(stations), 120_000)
        info = M.mcg_request_info(rq)
        M.mcg_request_free(rq)
    finally:
        M.mcg_server_destroy(sv)
    assert rc == M.MCG_OK
    return out, info


def test_alone_equals_in_mix(models):
    w, h = models["sphere"]
    st = w.stations[:5]
    alone, info = run_alone(w, h, st, 5e-3, 11)
    assert info[0] % CHUNK == 0 and info[0] >= 2 * CHUNK
    # the same request among others (other models, station counts, targets)
    sv = server(w, streams=4)
    try:
        reqs = []
        wv, hv = models["voxel"]
        reqs.append((M.mcg_submit(sv, hv, wv.stations[:7], 2e-2, 3), 7))
        reqs.append((M.mcg_submit(sv, h, w.stations[2:8], 1e-2, 5), 6))
        target = M.mcg_submit(sv, h, st, 5e-3, 11)
        reqs.append((M.mcg_submit(sv, hv, wv.stations[10:12], 1e-2, 9), 2))
        rc, mixed = M.mcg_wait(target, 5, 120_000)
        assert rc == M.MCG_OK
        for rq, S in reqs:
            assert M.mcg_wait(rq, S, 120_000)[0] == M.MCG_OK
            M.mcg_request_free(rq)
        M.mcg_request_free(target)
    finally:
        M.mcg_server_destroy(sv)
    for k in ("u", "gz", "se_u", "se_gz", "n_paths", "path_steps"):
        assert np.array_equal(alone[k], mixed[k]), k


def test_server_equals_device_solve(models):
    """Same paths as the device-level solve over the same number of paths;
    rounds past min_paths group several chunks into one batch, so the merged
    statistics agree to rounding and the counts exactly."""
    w, h = models["sphere"]
    st = w.stations[:3]
    out, (paths, rounds, _) = run_alone(w, h, st, 8e-3, 2)
    ds = DeviceSolve(w.with_(seed=2), stations=st, batch=CHUNK, precision=M.MCG_MIXED)
    ref = ds.run(paths=paths)
    for k in ("u", "gz", "se_u", "se_gz"):
        np.testing.assert_allclose(out[k], ref[k], rtol=1e-12, err_msg=k)
    for k in ("n_paths", "path_steps"):
        assert np.array_equal(out[k], ref[k]), k


def test_stops_at_target_and_respects_cap(models):
    w, h = models["sphere"]
    out, (paths, rounds, _) = run_alone(w, h, w.stations[:4], 4e-3, 1)
    assert np.all(out["se_u"] <= 4e-3 * np.abs(out["u"]))
    # the adaptive rounds do not overshoot much: at most half again the paths
    # the final spread says are needed, plus two chunks
    need = np.max((out["se_u"] * np.sqrt(paths) / (4e-3 * np.abs(out["u"]))) ** 2)
    assert paths <= 1.5 * need + 2 * CHUNK
    assert rounds < paths // CHUNK or paths == 2 * CHUNK   # several chunks went in one round
    # max_paths caps an unreachable target
    sv = server(w, max_paths=3 * CHUNK)
    try:
        rq = M.mcg_submit(sv, h, w.stations[:2], 1e-9, 1)
        rc, out = M.mcg_wait(rq, 2, 120_000)
        assert rc == M.MCG_OK and np.all(out["n_paths"] == 3 * CHUNK)
        M.mcg_request_free(rq)
    finally:
        M.mcg_server_destroy(sv)


def test_cancel_and_budget_queueing(models):
    w, h = models["prism"]
    sv = server(w, hbm_budget=1 << 20, streams=2)   # one request in flight at a time
    try:
        long_rq = M.mcg_submit(sv, h, w.stations[:2], 1e-7, 4)
        small = [M.mcg_submit(sv, models["sphere"][1], models["sphere"][0].stations[:1], 2e-2, s) for s in range(3)]
        time.sleep(0.5)
        M.mcg_cancel(long_rq)
        rc, out = M.mcg_wait(long_rq, 2, 300_000)
        assert rc == M.MCG_ERR_CANCELLED
        for rq in small:
            assert M.mcg_wait(rq, 1, 300_000)[0] == M.MCG_OK
            M.mcg_request_free(rq)
        M.mcg_request_free(long_rq)
    finally:
        M.mcg_server_destroy(sv)


def test_submit_validation(models):
    w, h = models["sphere"]
    sv = server(w)
    try:
        with pytest.raises(M.McgError):
            M.mcg_submit(sv, h, np.array([[0.0, 0.0, 2.0]]), 1e-2, 0)
        with pytest.raises(M.McgError):
            M.mcg_submit(sv, h, w.stations[:1], -1.0, 0)
    finally:
        M.mcg_server_destroy(sv)


def _run_all(models, reqs, batch, graph=1, **kw):
    """All requests submitted at once; (results in order, (launches, rounds))."""
    sph_w = models["sphere"][0]
    cfg = M.server_config(M.options(sph_w, graph=graph), chunk_paths=CHUNK, min_paths=2 * CHUNK,
                          max_paths=4 * CHUNK, batch=batch, **kw)
    sv = M.mcg_server_create(cfg)
    out = []
    try:
        hs = [M.mcg_submit(sv, models[name][1], st, target, seed) for name, st, target, seed in reqs]
        for h, (name, st, _, _) in zip(hs, reqs):
            rc, res = M.mcg_wait(h, len(st), 120_000)
            assert rc == M.MCG_OK, (name, rc, M.last_error())
            out.append(res)
            M.mcg_request_free(h)
        stats = M.mcg_server_stats(sv)
    finally:
        M.mcg_server_destroy(sv)
    return out, stats


def test_shared_launches_equal_separate_launches(models):
    """Eight requests (sphere, prism and two voxel models of one geometry with
    different grids and tables, different seeds, station sets and targets)
    through a server that shares walk launches between compatible rounds and
    through one that launches every round alone.  Sphere and prism results are
    bit for bit the same; voxel results agree to the flush rounding of the
    single-precision partial sums (which follows the warp schedule), with
    identical path and step counts (their targets are out of reach, so both
    servers stop them at max_paths).  A voxel walk read through the wrong
    request's grid or tables would differ by far more."""
    sw, pw, vw = models["sphere"][0], models["prism"][0], models["voxel"][0]
    reqs = [("sphere", sw.stations[:3], 5e-3, 21), ("voxel", vw.stations[:9], 1e-9, 22),
            ("sphere", sw.stations[3:8], 1e-2, 23), ("voxel2", vw.stations[100:104], 1e-9, 24),
            ("prism", pw.stations[:2], 2e-2, 25), ("voxel", vw.stations[50:51], 1e-9, 26),
            ("voxel2", vw.stations[7:20], 1e-9, 27), ("sphere", sw.stations[:1], 1e-2, 28)]
    shared, (launches, rounds) = _run_all(models, reqs, 1, streams=2)
    alone, (launches0, rounds0) = _run_all(models, reqs, 0, streams=2)
    assert launches0 == rounds0
    assert launches < rounds, (launches, rounds)       # rounds did share launches
    for (name, _, _, _), a, b in zip(reqs, shared, alone):
        for k in ("n_paths", "path_steps"):
            assert np.array_equal(a[k], b[k]), (name, k)
        if name.startswith("voxel"):
            for k in ("u", "gz"):
                np.testing.assert_allclose(a[k], b[k], rtol=1e-6, atol=1e-6 * np.abs(b["u"]).max(),
                                           err_msg=f"{name} {k}")
        else:
            for k in ("u", "gz", "se_u", "se_gz"):
                assert np.array_equal(a[k], b[k]), (name, k)


def test_graph_batches_equal_stream_batches(models):
    """Each batch of rounds (segment table, shared walk, every request's
    reduction, finalize and result copies) captured and launched as one CUDA
    graph -- the slot's instantiated graph updated in place from batch to batch
    -- gives what the same batches issued on the stream give: sphere and prism
    bit for bit, voxel to the flush rounding, path and step counts equal, and
    the same number of walk launches for the same rounds."""
    sw, pw, vw = models["sphere"][0], models["prism"][0], models["voxel"][0]
    reqs = [("voxel", vw.stations[:5], 1e-9, 41), ("sphere", sw.stations[:4], 5e-3, 42),
            ("voxel2", vw.stations[60:63], 1e-9, 43), ("prism", pw.stations[3:5], 2e-2, 44),
            ("sphere", sw.stations[4:6], 1e-2, 45), ("voxel", vw.stations[200:201], 1e-9, 46)]
    g, (launches_g, rounds_g) = _run_all(models, reqs, 1, graph=1, streams=2)
    n, (launches_n, rounds_n) = _run_all(models, reqs, 1, graph=0, streams=2)
    assert rounds_g == rounds_n and launches_g < rounds_g
    for (name, _, _, _), a, b in zip(reqs, g, n):
        for k in ("n_paths", "path_steps"):
            assert np.array_equal(a[k], b[k]), (name, k)
        if name.startswith("voxel"):
            for k in ("u", "gz"):
                np.testing.assert_allclose(a[k], b[k], rtol=1e-6, atol=1e-6 * np.abs(b["u"]).max(),
                                           err_msg=f"{name} {k}")
        else:
            for k in ("u", "gz", "se_u", "se_gz"):
                assert np.array_equal(a[k], b[k]), (name, k)
