"""Plain FP64 CPU oracle for the Feynman-Kac gravity walk (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never touches it, and the two share no code.

The oracle is plain C (``mcg_oracle.c``) compiled with gcc, without
floating-point contraction, and wrapped here with ctypes.  Each function cites
the part of the paper (arXiv:1709.07469) it follows in the C source:

* Philox4x32-10 and Box-Muller normals (the paper names no generator),
* the walk of Sec. 2.3 (Euler-Maruyama, trapezoid rule, exit check) with the
  last segment clipped to the box and common random numbers for g_z,
* Eq. 7 (Monte Carlo mean) with the sample variance and standard error,
* the closed forms of the homogeneous sphere and the rectangular prism,
* the heterogeneous model set-up: Gaussian random field density and boundary
  tables by direct prism summation.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

RHO_NONE, RHO_SPHERE, RHO_PRISM, RHO_VOXEL = 0, 1, 2, 3
G_ZERO, G_SPHERE, G_PRISM, G_TABLE, G_POLY = 0, 1, 2, 3, 4
OK, ERR_ARG, ERR_STEP_CAP = 0, 1, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available).  Returns the .so path."""
    src = os.path.join(_HERE, "mcg_oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src),
                                                   os.path.getmtime(os.path.join(_HERE, "mcg_oracle.h")))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Problem(C.Structure):
    _fields_ = [
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("domain_kind", C.c_int), ("bc", C.c_double * 3), ("R", C.c_double),
        ("rho_kind", C.c_int), ("G", C.c_double), ("rho0", C.c_double),
        ("center", C.c_double * 3), ("radius", C.c_double),
        ("plo", C.c_double * 3), ("phi", C.c_double * 3),
        ("grid", C.POINTER(C.c_float)), ("n", C.c_int64 * 3),
        ("origin", C.c_double * 3), ("spacing", C.c_double * 3),
        ("g_kind", C.c_int), ("faces", C.POINTER(C.c_float)),
        ("nu", C.c_int32), ("nv", C.c_int32), ("poly", C.c_double * 11),
        ("dt", C.c_double), ("sigma", C.c_double), ("h", C.c_double),
        ("seed", C.c_uint64), ("clip", C.c_int), ("crn", C.c_int), ("ubits", C.c_int),
        ("max_steps", C.c_int64), ("bridge", C.c_int),
    ]


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i64, u32, u64 = C.c_double, C.c_int64, C.c_uint32, C.c_uint64
            P = C.POINTER
            lib.orc_philox_fill.argtypes = [P(u32), P(u32), i64, P(u32)]
            lib.orc_normals_fill.argtypes = [u64, u32, u32, u32, i64, u32, C.c_int, P(d)]
            lib.orc_rho.argtypes = [P(Problem), P(d)]
            lib.orc_rho.restype = d
            lib.orc_g.argtypes = [P(Problem), P(d)]
            lib.orc_g.restype = d
            for nm in ("orc_sphere_phi", "orc_sphere_gz"):
                getattr(lib, nm).argtypes = [d, d, P(d), d, P(d)]
                getattr(lib, nm).restype = d
            for nm in ("orc_prism_phi", "orc_prism_gz"):
                getattr(lib, nm).argtypes = [d, d, P(d), P(d), P(d)]
                getattr(lib, nm).restype = d
            lib.orc_walk_path.argtypes = [P(Problem), P(d), u32, u32, P(d), P(i64), P(d)]
            lib.orc_walk_path.restype = C.c_int
            lib.orc_solve.argtypes = [P(Problem), P(d), i64, i64, i64, C.c_int,
                                      P(d), P(d), P(d), P(d), P(i64), P(d), P(d), P(i64), P(i64)]
            lib.orc_solve.restype = C.c_int
            lib.orc_grf_density.argtypes = [u64, i64, i64, i64, d, d, P(C.c_float), P(d)]
            lib.orc_table_nodes.argtypes = [P(Problem), P(i64), P(i64), P(i64), i64, C.c_int, P(d)]
            lib.orc_table_nodes.restype = C.c_int
            lib.orc_voxel_field.argtypes = [P(Problem), P(d), i64, C.c_int, P(d), P(d)]
            lib.orc_voxel_field.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def _v3(x):
    return (C.c_double * 3)(*[float(t) for t in x])


@dataclass
class Spec:
    """Problem description in plain Python (mirrors the oracle's struct)."""
    lo: tuple
    hi: tuple
    domain_kind: int = 0                  # 0 box, 1 ball |x - bc| < R
    bc: tuple = (0.0, 0.0, 0.0)
    R: float = 0.0
    rho_kind: int = RHO_NONE
    G: float = 1.0
    rho0: float = 0.0
    center: tuple = (0.0, 0.0, 0.0)
    radius: float = 0.0
    plo: tuple = (0.0, 0.0, 0.0)
    phi: tuple = (0.0, 0.0, 0.0)
    grid: np.ndarray | None = None        # float32 [nz, ny, nx]
    origin: tuple = (0.0, 0.0, 0.0)
    spacing: tuple = (1.0, 1.0, 1.0)
    g_kind: int = G_ZERO
    faces: np.ndarray | None = None       # float32 [6, nv, nu]
    poly: tuple = (0.0,) * 11
    dt: float = 1e-3
    sigma: float = 1.0
    h: float = 0.01
    seed: int = 0
    clip: int = 1
    crn: int = 1
    ubits: int = 32
    max_steps: int = 1 << 40
    bridge: int = 0
    _keep: list = field(default_factory=list, repr=False)

    def struct(self) -> Problem:
        p = Problem()
        p.lo, p.hi = _v3(self.lo), _v3(self.hi)
        p.domain_kind, p.bc, p.R = self.domain_kind, _v3(self.bc), self.R
        p.rho_kind, p.G, p.rho0 = self.rho_kind, self.G, self.rho0
        p.center, p.radius = _v3(self.center), self.radius
        p.plo, p.phi = _v3(self.plo), _v3(self.phi)
        self._keep = []
        if self.grid is not None:
            g = np.ascontiguousarray(self.grid, dtype=np.float32)
            self._keep.append(g)
            p.grid = _ptr(g, C.c_float)
            nz, ny, nx = g.shape
            p.n = (C.c_int64 * 3)(nx, ny, nz)
        p.origin, p.spacing = _v3(self.origin), _v3(self.spacing)
        p.g_kind = self.g_kind
        if self.faces is not None:
            f = np.ascontiguousarray(self.faces, dtype=np.float32)
            self._keep.append(f)
            p.faces = _ptr(f, C.c_float)
            p.nv, p.nu = f.shape[1], f.shape[2]
        p.poly = (C.c_double * 11)(*[float(t) for t in self.poly])
        p.dt, p.sigma, p.h = self.dt, self.sigma, self.h
        p.seed, p.clip, p.crn, p.ubits = self.seed, self.clip, self.crn, self.ubits
        p.max_steps = self.max_steps
        p.bridge = self.bridge
        return p


def philox(ctrs: np.ndarray, keys: np.ndarray) -> np.ndarray:
    """Philox4x32-10 of n counters [n,4] under n keys [n,2] -> [n,4] uint32."""
    lib = _lib_handle()
    c = np.ascontiguousarray(ctrs, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(keys, dtype=np.uint32).reshape(-1, 2)
    out = np.empty_like(c)
    lib.orc_philox_fill(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), c.shape[0], _ptr(out, C.c_uint32))
    return out


def normals(seed: int, s: int, p: int, b0: int, nblocks: int, tag: int = 0, ubits: int = 32) -> np.ndarray:
    """Normals of step blocks b0..b0+nblocks-1 of path (s, p): [nblocks*12]."""
    lib = _lib_handle()
    z = np.empty(12 * nblocks, dtype=np.float64)
    lib.orc_normals_fill(seed, s, p, b0, nblocks, tag, ubits, _ptr(z, C.c_double))
    return z


def rho(spec: Spec, x) -> float:
    st = spec.struct()
    return _lib_handle().orc_rho(C.byref(st), _v3(x))


def g(spec: Spec, x) -> float:
    st = spec.struct()
    return _lib_handle().orc_g(C.byref(st), _v3(x))


def sphere_phi(G, rho0, c, a, x):
    return _lib_handle().orc_sphere_phi(G, rho0, _v3(c), a, _v3(x))


def sphere_gz(G, rho0, c, a, x):
    return _lib_handle().orc_sphere_gz(G, rho0, _v3(c), a, _v3(x))


def prism_phi(G, rho0, lo, hi, x):
    return _lib_handle().orc_prism_phi(G, rho0, _v3(lo), _v3(hi), _v3(x))


def prism_gz(G, rho0, lo, hi, x):
    return _lib_handle().orc_prism_gz(G, rho0, _v3(lo), _v3(hi), _v3(x))


def walk_path(spec: Spec, x0, s: int, p: int):
    """One path: (status, u[3], steps[3], xexit[3,3])."""
    st = spec.struct()
    u = (C.c_double * 3)()
    steps = (C.c_int64 * 3)()
    xe = (C.c_double * 9)()
    rc = _lib_handle().orc_walk_path(C.byref(st), _v3(x0), s, p, u, steps, xe)
    return rc, np.array(u[:]), np.array(steps[:]), np.array(xe[:]).reshape(3, 3)


@dataclass
class Result:
    status: int
    u: np.ndarray
    gz: np.ndarray
    se_u: np.ndarray
    se_gz: np.ndarray
    path_steps: np.ndarray
    pp_u: np.ndarray | None = None
    pp_d: np.ndarray | None = None
    pp_steps: np.ndarray | None = None
    pp_copy_steps: np.ndarray | None = None


def solve(spec: Spec, stations, paths: int, p0: int = 0, threads: int = 0, per_path: bool = False) -> Result:
    """Station means, g_z and standard errors over paths p0..p0+paths-1."""
    lib = _lib_handle()
    st = spec.struct()
    x = np.ascontiguousarray(stations, dtype=np.float64).reshape(-1, 3)
    S = x.shape[0]
    u, gz, se_u, se_gz = (np.empty(S) for _ in range(4))
    ps = np.empty(S, dtype=np.int64)
    ppu = ppd = pps = ppc = None
    if per_path:
        ppu, ppd = np.empty(S * paths), np.empty(S * paths)
        pps = np.empty(S * paths, dtype=np.int64)
        ppc = np.empty(S * paths * 3, dtype=np.int64)
    rc = lib.orc_solve(C.byref(st), _ptr(x, C.c_double), S, p0, paths, threads,
                       _ptr(u, C.c_double), _ptr(gz, C.c_double), _ptr(se_u, C.c_double),
                       _ptr(se_gz, C.c_double), _ptr(ps, C.c_int64),
                       _ptr(ppu, C.c_double), _ptr(ppd, C.c_double), _ptr(pps, C.c_int64),
                       _ptr(ppc, C.c_int64))
    res = Result(rc, u, gz, se_u, se_gz, ps)
    if per_path:
        res.pp_u, res.pp_d = ppu.reshape(S, paths), ppd.reshape(S, paths)
        res.pp_steps = pps.reshape(S, paths)
        res.pp_copy_steps = ppc.reshape(S, paths, 3)
    return res


def grf_density(seed: int, nx: int, ny: int, nz: int, sigma_vox: float = 5.0, amp: float = 300.0,
                want_z: bool = False):
    """Gaussian-random-field density grid float32 [nz, ny, nx] (and Z if asked)."""
    lib = _lib_handle()
    grid = np.empty((nz, ny, nx), dtype=np.float32)
    z = np.empty((nz, ny, nx), dtype=np.float64) if want_z else None
    lib.orc_grf_density(seed, nx, ny, nz, sigma_vox, amp, _ptr(grid, C.c_float), _ptr(z, C.c_double))
    return (grid, z) if want_z else grid


def table_nodes(spec: Spec, face, iu, iv, nu: int, nv: int, threads: int = 0) -> np.ndarray:
    """Potential at face-table nodes by direct prism summation over all voxels."""
    lib = _lib_handle()
    st = spec.struct()
    st.nu, st.nv = nu, nv
    f = np.ascontiguousarray(face, dtype=np.int64)
    a = np.ascontiguousarray(iu, dtype=np.int64)
    b = np.ascontiguousarray(iv, dtype=np.int64)
    out = np.empty(f.shape[0])
    rc = lib.orc_table_nodes(C.byref(st), _ptr(f, C.c_int64), _ptr(a, C.c_int64), _ptr(b, C.c_int64),
                             f.shape[0], threads, _ptr(out, C.c_double))
    if rc != OK:
        raise ValueError(f"orc_table_nodes status {rc}")
    return out


def voxel_field(spec: Spec, points, threads: int = 0, want_gz: bool = False):
    """Phi (and dPhi/dz) of the voxel model at points [n,3] by direct prism sums."""
    lib = _lib_handle()
    st = spec.struct()
    x = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    phi = np.empty(x.shape[0])
    gz = np.empty(x.shape[0]) if want_gz else None
    rc = lib.orc_voxel_field(C.byref(st), _ptr(x, C.c_double), x.shape[0], threads, _ptr(phi, C.c_double),
                             _ptr(gz, C.c_double))
    if rc != OK:
        raise ValueError(f"orc_voxel_field status {rc}")
    return (phi, gz) if want_gz else phi
