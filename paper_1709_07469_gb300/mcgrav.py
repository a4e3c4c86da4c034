"""ctypes binding of libmcgrav (include/mcgrav.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts numpy
arrays / torch tensors into the C structures and pointers and turns status
codes into exceptions.  Loading fails loudly if the library has not been
built (``python -m paper_1709_07469_gb300.build``): there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

MCG_OK, MCG_ERR_ARG, MCG_ERR_OOM, MCG_ERR_CUDA = 0, 1, 2, 3
MCG_ERR_STEP_CAP, MCG_ERR_TIMEOUT, MCG_ERR_NONFINITE, MCG_ERR_CANCELLED = 4, 5, 6, 7
MCG_RHO_NONE, MCG_RHO_SPHERE, MCG_RHO_PRISM, MCG_RHO_VOXEL = 0, 1, 2, 3
MCG_DOMAIN_BOX, MCG_DOMAIN_BALL = 0, 1
MCG_G_ZERO, MCG_G_SPHERE, MCG_G_PRISM, MCG_G_TABLE, MCG_G_POLY = 0, 1, 2, 3, 4
MCG_FP64, MCG_MIXED = 0, 1

_RHO = {"none": MCG_RHO_NONE, "sphere": MCG_RHO_SPHERE, "prism": MCG_RHO_PRISM, "voxel": MCG_RHO_VOXEL}
_G = {"zero": MCG_G_ZERO, "sphere": MCG_G_SPHERE, "prism": MCG_G_PRISM, "table": MCG_G_TABLE, "poly": MCG_G_POLY}

D3 = C.c_double * 3


class mcg_domain(C.Structure):
    _fields_ = [("lo", D3), ("hi", D3), ("kind", C.c_int32), ("center", D3), ("radius", C.c_double)]


class mcg_density(C.Structure):
    _fields_ = [("kind", C.c_int32), ("G", C.c_double), ("rho0", C.c_double), ("center", D3),
                ("radius", C.c_double), ("lo", D3), ("hi", D3), ("grid", C.c_void_p),
                ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64), ("origin", D3), ("spacing", D3),
                ("zpack", C.c_void_p)]


class mcg_boundary(C.Structure):
    _fields_ = [("kind", C.c_int32), ("faces", C.c_void_p), ("nu", C.c_int32), ("nv", C.c_int32),
                ("poly", C.c_double * 11), ("quads", C.c_void_p)]


class mcg_options(C.Structure):
    _fields_ = [("h", C.c_double), ("sigma", C.c_double), ("precision", C.c_int32), ("clip", C.c_int32),
                ("crn_gz", C.c_int32), ("block", C.c_int32), ("max_steps", C.c_int64),
                ("batch_paths", C.c_int64), ("stream", C.c_void_p), ("cancel", C.c_void_p),
                ("bridge", C.c_int32), ("refill_min", C.c_int32), ("graph", C.c_int32),
                ("migrate", C.c_int32), ("fault_unpublished", C.c_int32), ("spill_max", C.c_int32)]


class mcg_result(C.Structure):
    _fields_ = [("u", C.c_void_p), ("gz", C.c_void_p), ("se_u", C.c_void_p), ("se_gz", C.c_void_p),
                ("n_paths", C.c_void_p), ("path_steps", C.c_void_p)]


class mcg_server_config(C.Structure):
    _fields_ = [("streams", C.c_int32), ("max_active", C.c_int32), ("hbm_budget", C.c_int64),
                ("chunk_paths", C.c_int64), ("min_paths", C.c_int64), ("max_paths", C.c_int64),
                ("max_round_paths", C.c_int64), ("walk", mcg_options), ("batch", C.c_int32),
                ("batch_items", C.c_int64)]


class mcg_station_state(C.Structure):
    _fields_ = [("n", C.c_double), ("mean_u", C.c_double), ("m2_u", C.c_double), ("mean_d", C.c_double),
                ("m2_d", C.c_double), ("steps", C.c_double), ("pad", C.c_double * 2)]


STATE_BYTES = C.sizeof(mcg_station_state)


class McgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mcgrav status {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libmcgrav.so (raises if it is missing: there is no CPU path)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise ImportError(f"libmcgrav.so not built at {p}; run paper_1709_07469_gb300.build.build()")
    lib = C.CDLL(p)
    vp, i32, i64, u32, u64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
    P = C.POINTER
    lib.mcg_options_default.argtypes = [P(mcg_options)]
    lib.mcg_options_default.restype = None
    lib.mcg_last_error.restype = C.c_char_p
    lib.mcg_version.restype = C.c_char_p
    lib.mcgrav_solve.argtypes = [P(mcg_domain), P(mcg_density), P(mcg_boundary), vp, i64, i64, d, u64,
                                 P(mcg_options), P(mcg_result)]
    lib.mcgrav_solve.restype = C.c_int
    lib.mcg_walk.argtypes = [P(mcg_domain), P(mcg_density), P(mcg_boundary), vp, i64, i64, i64, d, u64,
                             P(mcg_options), vp, vp, vp, vp, vp, vp]
    lib.mcg_walk.restype = C.c_int
    lib.mcg_walk_work_bytes.argtypes = [i64, i64, i32]
    lib.mcg_walk_work_bytes.restype = C.c_size_t
    lib.mcg_walk_static.argtypes = [P(mcg_domain), P(mcg_density), P(mcg_boundary), vp, i64, i64, i64, d, u64,
                                    P(mcg_options), vp, vp, vp, vp]
    lib.mcg_walk_static.restype = C.c_int
    lib.mcg_walk_static_max_items.argtypes = []
    lib.mcg_walk_static_max_items.restype = C.c_int64
    lib.mcg_autotune.argtypes = [P(mcg_domain), P(mcg_density), P(mcg_boundary), vp, i64, d, u64, P(mcg_options)]
    lib.mcg_autotune.restype = C.c_int
    lib.mcg_smooth_moving_average.argtypes = [vp, i64, i32, vp]
    lib.mcg_smooth_moving_average.restype = C.c_int
    lib.mcg_states_merge.argtypes = [vp, i64, i64, vp]
    lib.mcg_states_merge.restype = C.c_int
    lib.mcg_server_config_default.argtypes = [P(mcg_server_config)]
    lib.mcg_server_config_default.restype = None
    lib.mcg_model_create.argtypes = [P(mcg_domain), P(mcg_density), P(mcg_boundary), d, d, P(vp)]
    lib.mcg_model_create.restype = C.c_int
    lib.mcg_model_destroy.argtypes = [vp]
    lib.mcg_model_destroy.restype = C.c_int
    lib.mcg_server_create.argtypes = [P(mcg_server_config), P(vp)]
    lib.mcg_server_create.restype = C.c_int
    lib.mcg_server_destroy.argtypes = [vp]
    lib.mcg_server_destroy.restype = C.c_int
    lib.mcg_submit.argtypes = [vp, vp, vp, i64, d, u64, P(vp)]
    lib.mcg_submit.restype = C.c_int
    lib.mcg_poll.argtypes = [vp, P(mcg_result), P(C.c_int)]
    lib.mcg_poll.restype = C.c_int
    lib.mcg_wait.argtypes = [vp, P(mcg_result), i64]
    lib.mcg_wait.restype = C.c_int
    lib.mcg_cancel.argtypes = [vp]
    lib.mcg_cancel.restype = C.c_int
    lib.mcg_request_info.argtypes = [vp, P(i64), P(i64), P(d)]
    lib.mcg_request_info.restype = C.c_int
    lib.mcg_server_stats.argtypes = [vp, P(i64), P(i64)]
    lib.mcg_server_stats.restype = C.c_int
    lib.mcg_request_free.argtypes = [vp]
    lib.mcg_request_free.restype = C.c_int
    lib.mcg_grf_work_bytes.argtypes = [i64, i64, i64]
    lib.mcg_grf_work_bytes.restype = C.c_size_t
    lib.mcg_grf_density.argtypes = [u64, i64, i64, i64, d, d, vp, vp, vp]
    lib.mcg_grf_density.restype = C.c_int
    lib.mcg_boundary_tables.argtypes = [P(mcg_domain), P(mcg_density), i32, i32, d, vp, vp]
    lib.mcg_boundary_tables.restype = C.c_int
    lib.mcg_reduce.argtypes = [vp, vp, vp, i64, i64, vp, vp]
    lib.mcg_reduce.restype = C.c_int
    lib.mcg_finalize.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp]
    lib.mcg_finalize.restype = C.c_int
    lib.mcg_workspace_bytes.argtypes = [i64, i64]
    lib.mcg_workspace_bytes.restype = C.c_size_t
    lib.mcg_voxel_pack_bytes.argtypes = [i64, i64, i64]
    lib.mcg_voxel_pack_bytes.restype = C.c_size_t
    lib.mcg_voxel_pack.argtypes = [P(mcg_density), vp, vp]
    lib.mcg_voxel_pack.restype = C.c_int
    lib.mcg_table_pack_bytes.argtypes = [i32, i32]
    lib.mcg_table_pack_bytes.restype = C.c_size_t
    lib.mcg_table_pack.argtypes = [P(mcg_boundary), vp, vp]
    lib.mcg_table_pack.restype = C.c_int
    lib.mcg_issue_probe.argtypes = [i32, i32, P(d), P(d)]
    lib.mcg_issue_probe.restype = C.c_int
    lib.mcg_field.argtypes = [P(mcg_density), vp, i64, vp, vp, vp]
    lib.mcg_field.restype = C.c_int
    lib.mcg_density_at.argtypes = [P(mcg_domain), P(mcg_density), d, i32, vp, i64, vp, vp]
    lib.mcg_density_at.restype = C.c_int
    lib.mcg_philox.argtypes = [vp, vp, i64, vp, vp]
    lib.mcg_philox.restype = C.c_int
    lib.mcg_normals.argtypes = [u64, u32, u32, u32, i64, i32, vp, vp]
    lib.mcg_normals.restype = C.c_int
    _lib = lib
    return lib


def _check(rc: int, allow=()):
    if rc != MCG_OK and rc not in allow:
        raise McgError(rc, load().mcg_last_error().decode())
    return rc


def last_error() -> str:
    return load().mcg_last_error().decode()


def version() -> str:
    return load().mcg_version().decode()


def _ptr(x) -> int | None:
    """Device pointer of a torch tensor, host pointer of a numpy array, or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# --- problem description ----------------------------------------------------

@dataclass
class Problem:
    domain: mcg_domain
    density: mcg_density
    boundary: mcg_boundary
    keep: tuple = ()


def problem(w, grid=None, faces=None, zpack=None, quads=None) -> Problem:
    """C structures of a workload (paper_1709_07469_gb300.workloads.Workload).
    `grid` / `faces` are device tensors (float32) when the workload uses them;
    `zpack` / `quads` their optional packed copies (mcg_voxel_pack /
    mcg_table_pack, device tensors)."""
    dom = mcg_domain(D3(*w.lo), D3(*w.hi), 1 if getattr(w, "domain", "box") == "ball" else 0,
                     D3(*getattr(w, "ball_center", (0.0, 0.0, 0.0))), getattr(w, "ball_radius", 0.0))
    den = mcg_density()
    den.kind = _RHO[w.rho_kind]
    den.G, den.rho0 = w.G, w.rho0
    den.center, den.radius = D3(*w.center), w.radius
    if w.rho_kind == "prism":
        den.lo, den.hi = D3(*w.plo), D3(*w.phi)
    if w.rho_kind == "voxel":
        if grid is None:
            raise ValueError("voxel workload needs a device grid")
        nz, ny, nx = grid.shape
        den.grid = _ptr(grid)
        den.nx, den.ny, den.nz = nx, ny, nz
        den.origin, den.spacing = D3(*w.grid_origin), D3(*w.grid_spacing)
        den.zpack = _ptr(zpack)
    bnd = mcg_boundary()
    bnd.kind = _G[w.g_kind]
    bnd.poly = (C.c_double * 11)(*[float(c) for c in w.poly])
    if w.g_kind == "table":
        if faces is None:
            raise ValueError("table workload needs device faces")
        bnd.faces = _ptr(faces)
        bnd.nv, bnd.nu = faces.shape[1], faces.shape[2]
        bnd.quads = _ptr(quads)
    return Problem(dom, den, bnd, (grid, faces, zpack, quads))


def options(w=None, precision: int = MCG_MIXED, stream=None, **kw) -> mcg_options:
    o = mcg_options()
    load().mcg_options_default(C.byref(o))
    o.precision = precision
    if w is not None:
        o.h, o.sigma, o.clip, o.crn_gz, o.bridge = w.h, w.sigma, w.clip, w.crn, w.bridge
    o.stream = _stream_handle(stream)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


# --- entry points -------------------------------------------------------------

@dataclass
class SolveResult:
    status: int
    u: np.ndarray
    gz: np.ndarray
    se_u: np.ndarray
    se_gz: np.ndarray
    n_paths: np.ndarray
    path_steps: np.ndarray


def mcgrav_solve(prob: Problem, stations: np.ndarray, paths: int, dt: float, seed: int, opts: mcg_options,
                 allow=()) -> SolveResult:
    """Blocking one-call solve with HOST stations and HOST results."""
    lib = load()
    st = np.ascontiguousarray(stations, dtype=np.float64).reshape(-1, 3)
    S = st.shape[0]
    out = {k: np.full(S, np.nan) for k in ("u", "gz", "se_u", "se_gz")}
    out["n_paths"] = np.zeros(S, dtype=np.int64)
    out["path_steps"] = np.zeros(S, dtype=np.int64)
    res = mcg_result(*[out[k].ctypes.data for k in ("u", "gz", "se_u", "se_gz", "n_paths", "path_steps")])
    rc = lib.mcgrav_solve(C.byref(prob.domain), C.byref(prob.density), C.byref(prob.boundary), st.ctypes.data,
                          S, paths, dt, seed & 0xFFFFFFFFFFFFFFFF, C.byref(opts), C.byref(res))
    _check(rc, allow)
    return SolveResult(rc, **out)


def mcg_walk(prob: Problem, stations_dev, S: int, p0: int, N: int, dt: float, seed: int, opts: mcg_options,
             pp_u, pp_d, pp_steps, work_dev, status_dev, counter_dev) -> int:
    """Asynchronous walk launch on device buffers (torch tensors)."""
    rc = load().mcg_walk(C.byref(prob.domain), C.byref(prob.density), C.byref(prob.boundary), _ptr(stations_dev),
                         S, p0, N, dt, seed & 0xFFFFFFFFFFFFFFFF, C.byref(opts), _ptr(pp_u), _ptr(pp_d),
                         _ptr(pp_steps), _ptr(work_dev), _ptr(status_dev), _ptr(counter_dev))
    return _check(rc)


def mcg_walk_work_bytes(S: int, N: int, precision: int) -> int:
    return int(load().mcg_walk_work_bytes(S, N, precision))


def mcg_walk_static(prob: Problem, stations_dev, S: int, p0: int, N: int, dt: float, seed: int, opts: mcg_options,
                    pp_u, pp_d, pp_steps, status_dev, allow=()) -> int:
    """The walk with the library's fixed scratch (no device allocation)."""
    rc = load().mcg_walk_static(C.byref(prob.domain), C.byref(prob.density), C.byref(prob.boundary),
                                _ptr(stations_dev), S, p0, N, dt, seed & 0xFFFFFFFFFFFFFFFF, C.byref(opts),
                                _ptr(pp_u), _ptr(pp_d), _ptr(pp_steps), _ptr(status_dev))
    return _check(rc, allow)


def mcg_walk_static_max_items() -> int:
    return int(load().mcg_walk_static_max_items())


def mcg_reduce(pp_u, pp_d, pp_steps, S: int, N: int, states_dev, stream=None) -> int:
    return _check(load().mcg_reduce(_ptr(pp_u), _ptr(pp_d), _ptr(pp_steps), S, N, _ptr(states_dev),
                                    _stream_handle(stream)))


def mcg_finalize(states_dev, S: int, u=None, gz=None, se_u=None, se_gz=None, n_paths=None, path_steps=None,
                 stream=None) -> int:
    return _check(load().mcg_finalize(_ptr(states_dev), S, _ptr(u), _ptr(gz), _ptr(se_u), _ptr(se_gz),
                                      _ptr(n_paths), _ptr(path_steps), _stream_handle(stream)))


def mcg_workspace_bytes(S: int, batch: int) -> int:
    return int(load().mcg_workspace_bytes(S, batch))


def mcg_philox(ctr_dev, key_dev, n: int, out_dev, stream=None) -> int:
    return _check(load().mcg_philox(_ptr(ctr_dev), _ptr(key_dev), n, _ptr(out_dev), _stream_handle(stream)))


def mcg_normals(seed: int, s: int, p: int, b0: int, nblocks: int, precision: int, out_dev, stream=None) -> int:
    return _check(load().mcg_normals(seed & 0xFFFFFFFFFFFFFFFF, s, p, b0, nblocks, precision, _ptr(out_dev),
                                     _stream_handle(stream)))


def mcg_grf_work_bytes(nx: int, ny: int, nz: int) -> int:
    return int(load().mcg_grf_work_bytes(nx, ny, nz))


def mcg_grf_density(seed: int, nx: int, ny: int, nz: int, sigma_vox: float, amp: float, grid_out, work,
                    stream=None) -> int:
    return _check(load().mcg_grf_density(seed & 0xFFFFFFFFFFFFFFFF, nx, ny, nz, sigma_vox, amp, _ptr(grid_out),
                                         _ptr(work), _stream_handle(stream)))


def mcg_boundary_tables(prob: Problem, nu: int, nv: int, near_cells: float, faces_out, stream=None) -> int:
    return _check(load().mcg_boundary_tables(C.byref(prob.domain), C.byref(prob.density), nu, nv, near_cells,
                                             _ptr(faces_out), _stream_handle(stream)))


def mcg_issue_probe(kind: int, iters: int = 4096):
    """(lane-instructions per second, seconds) of the issue-rate probe."""
    rate, secs = C.c_double(), C.c_double()
    _check(load().mcg_issue_probe(kind, iters, C.byref(rate), C.byref(secs)))
    return rate.value, secs.value


def mcg_voxel_pack_bytes(nx: int, ny: int, nz: int) -> int:
    return int(load().mcg_voxel_pack_bytes(nx, ny, nz))


def mcg_voxel_pack(prob: Problem, out_dev, stream=None) -> int:
    return _check(load().mcg_voxel_pack(C.byref(prob.density), _ptr(out_dev), _stream_handle(stream)))


def mcg_table_pack_bytes(nu: int, nv: int) -> int:
    return int(load().mcg_table_pack_bytes(nu, nv))


def mcg_table_pack(prob: Problem, out_dev, stream=None) -> int:
    return _check(load().mcg_table_pack(C.byref(prob.boundary), _ptr(out_dev), _stream_handle(stream)))


def mcg_field(prob: Problem, points_dev, n: int, phi_dev=None, gz_dev=None, stream=None) -> int:
    """Exact Phi and dPhi/dz of the problem's density model at n device points."""
    return _check(load().mcg_field(C.byref(prob.density), _ptr(points_dev), n, _ptr(phi_dev), _ptr(gz_dev),
                                   _stream_handle(stream)))


def mcg_density_at(prob: Problem, h: float, precision: int, points_dev, n: int, out_dev, stream=None) -> int:
    """The walks' density sampler at n device points and their copies z +- h
    (out: 3 n doubles on the device)."""
    return _check(load().mcg_density_at(C.byref(prob.domain), C.byref(prob.density), h, precision,
                                        _ptr(points_dev), n, _ptr(out_dev), _stream_handle(stream)))


STATE_FIELDS = ("n", "mean_u", "m2_u", "mean_d", "m2_d", "steps")


def mcg_states_merge(parts: np.ndarray) -> np.ndarray:
    """Merge per-rank station states (float64 array [R, S, 8]) in rank order."""
    p = np.ascontiguousarray(parts, dtype=np.float64)
    if p.ndim != 3 or p.shape[2] != STATE_BYTES // 8:
        raise ValueError("parts must be [R, S, 8] float64")
    out = np.zeros(p.shape[1:], dtype=np.float64)
    _check(load().mcg_states_merge(p.ctypes.data, p.shape[0], p.shape[1], out.ctypes.data))
    return out


# --- serving --------------------------------------------------------------------

def server_config(opts: mcg_options | None = None, **kw) -> mcg_server_config:
    c = mcg_server_config()
    load().mcg_server_config_default(C.byref(c))
    if opts is not None:
        c.walk = opts
    for k, v in kw.items():
        setattr(c, k, v)
    if "chunk_paths" in kw and "max_round_paths" not in kw:
        c.max_round_paths = 16 * c.chunk_paths
    return c


def mcg_model_create(prob: Problem, dt: float, h: float) -> int:
    out = C.c_void_p()
    _check(load().mcg_model_create(C.byref(prob.domain), C.byref(prob.density), C.byref(prob.boundary), dt, h,
                                   C.byref(out)))
    return out.value


def mcg_model_destroy(model: int) -> int:
    return _check(load().mcg_model_destroy(model))


def mcg_server_create(cfg: mcg_server_config) -> int:
    h = C.c_void_p()
    _check(load().mcg_server_create(C.byref(cfg), C.byref(h)))
    return h.value


def mcg_server_stats(server: int):
    """(walk launches, request rounds) of the server so far."""
    a, b = C.c_int64(), C.c_int64()
    _check(load().mcg_server_stats(server, C.byref(a), C.byref(b)))
    return a.value, b.value


def mcg_server_destroy(server: int) -> int:
    return _check(load().mcg_server_destroy(server))


def mcg_submit(server: int, model: int, stations: np.ndarray, target_rel_se: float, seed: int) -> int:
    st = np.ascontiguousarray(stations, dtype=np.float64).reshape(-1, 3)
    h = C.c_void_p()
    _check(load().mcg_submit(server, model, st.ctypes.data, st.shape[0], target_rel_se,
                             seed & 0xFFFFFFFFFFFFFFFF, C.byref(h)))
    return h.value


def _result_buffers(S: int):
    out = {k: np.full(S, np.nan) for k in ("u", "gz", "se_u", "se_gz")}
    out["n_paths"] = np.zeros(S, dtype=np.int64)
    out["path_steps"] = np.zeros(S, dtype=np.int64)
    res = mcg_result(*[out[k].ctypes.data for k in ("u", "gz", "se_u", "se_gz", "n_paths", "path_steps")])
    return out, res


def mcg_poll(request: int, S: int):
    """(done, status, result dict or None)."""
    out, res = _result_buffers(S)
    done = C.c_int(0)
    rc = load().mcg_poll(request, C.byref(res), C.byref(done))
    return bool(done.value), rc, (out if done.value else None)


def mcg_wait(request: int, S: int, timeout_ms: int = -1):
    """(status, result dict); MCG_ERR_TIMEOUT leaves the dict unfilled."""
    out, res = _result_buffers(S)
    rc = load().mcg_wait(request, C.byref(res), timeout_ms)
    return rc, out


def mcg_cancel(request: int) -> int:
    return _check(load().mcg_cancel(request))


def mcg_request_info(request: int):
    paths, rounds, secs = C.c_int64(), C.c_int64(), C.c_double()
    _check(load().mcg_request_info(request, C.byref(paths), C.byref(rounds), C.byref(secs)))
    return paths.value, rounds.value, secs.value


def mcg_request_free(request: int) -> int:
    return _check(load().mcg_request_free(request))


def mcg_autotune(prob: Problem, stations_dev, S: int, dt: float, seed: int, opts: mcg_options) -> mcg_options:
    """Picks block and refill_min in place (returns opts)."""
    _check(load().mcg_autotune(C.byref(prob.domain), C.byref(prob.density), C.byref(prob.boundary),
                               _ptr(stations_dev), S, dt, seed & 0xFFFFFFFFFFFFFFFF, C.byref(opts)))
    return opts


def mcg_smooth_moving_average(y, span: int = 5) -> np.ndarray:
    a = np.ascontiguousarray(y, dtype=np.float64)
    out = np.empty_like(a)
    _check(load().mcg_smooth_moving_average(a.ctypes.data, a.size, span, out.ctypes.data))
    return out
