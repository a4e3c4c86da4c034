"""Seeded synthetic workloads (problem descriptions only, no method arithmetic).

Each workload is plain data: the box domain, the density model, the Dirichlet
data, the stations and the walk parameters.  Tests, the smoke check and the
benchmark build both the CUDA call and the oracle call from the same object.
Nothing here computes any part of the walk, the closed forms or the set-up.

Shapes follow the paper's experiments (a compact ore body under a survey
line, Sec. 3 and Sec. 4) scaled to the workloads this library is measured on:

* ``sphere_line``     homogeneous sphere in the cube [-1,1]^3, G = 1,
                      8 stations on the z axis, dt = 1e-3, FP64 parity case;
* ``prism_ore_body``  200x200x100 m prism (density contrast 500 kg/m^3, top
                      150 m deep) in [-1000,1000]^2 x [-1000,200] m, 30
                      stations, step 1 m, 10^6 paths per station;
* ``voxel_survey``    128x128x64 Gaussian-random-field density over a
                      4000x4000x2000 m block, 256x256 boundary tables per
                      face, 256 surface stations, step 10 m.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

G_SI = 6.67430e-11  # CODATA 2018, m^3 kg^-1 s^-2


@dataclass(frozen=True)
class Workload:
    name: str
    lo: tuple
    hi: tuple
    rho_kind: str                 # "none" | "sphere" | "prism" | "voxel"
    g_kind: str                   # "zero" | "sphere" | "prism" | "table" | "poly"
    G: float
    stations: np.ndarray = field(repr=False)
    dt: float = 1e-3
    sigma: float = 1.0
    h: float = 0.01
    seed: int = 0
    paths: int = 1000
    rho0: float = 0.0
    center: tuple = (0.0, 0.0, 0.0)
    radius: float = 0.0
    plo: tuple = (0.0, 0.0, 0.0)
    phi: tuple = (0.0, 0.0, 0.0)
    grid_shape: tuple = (0, 0, 0)       # (nx, ny, nz)
    grid_origin: tuple = (0.0, 0.0, 0.0)
    grid_spacing: tuple = (1.0, 1.0, 1.0)
    grid_seed: int = 0
    grid_sigma_vox: float = 5.0
    grid_amp: float = 300.0
    table_n: tuple = (256, 256)         # (nu, nv) nodes per face
    poly: tuple = (0.0,) * 11
    clip: int = 1
    crn: int = 1
    bridge: int = 0
    domain: str = "box"                 # "box" (lo, hi) or "ball" (ball_center, ball_radius)
    ball_center: tuple = (0.0, 0.0, 0.0)
    ball_radius: float = 0.0

    @property
    def n_stations(self) -> int:
        return int(self.stations.shape[0])

    @property
    def step_length(self) -> float:
        return float(self.sigma * np.sqrt(self.dt))

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def sphere_line(paths: int = 20000, dt: float = 1e-3, seed: int = 0) -> Workload:
    """Homogeneous sphere (a = 0.25, rho = 1, G = 1) at the centre of [-1,1]^3;
    Dirichlet data = the sphere's own potential; stations (0, 0, z),
    z = 0.30 .. 0.65 step 0.05; h = 0.01."""
    z = 0.30 + 0.05 * np.arange(8)
    st = np.stack([np.zeros(8), np.zeros(8), z], axis=1)
    return Workload(name="sphere_line", lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0),
                    rho_kind="sphere", g_kind="sphere", G=1.0, stations=st, dt=dt, h=0.01,
                    seed=seed, paths=paths, rho0=1.0, radius=0.25)


def prism_ore_body(paths: int = 1_000_000, seed: int = 0, step: float = 1.0) -> Workload:
    """Prism [-100,100]^2 x [-250,-150] m, density contrast 500 kg/m^3, in
    [-1000,1000]^2 x [-1000,200] m; Dirichlet data = the prism's potential;
    stations on x in {-200..200 step 100}, y in {-100, 0, 100}, z in {0, 50};
    step length sigma sqrt(dt) = 1 m; h = 1 m."""
    xs = np.array([-200.0, -100.0, 0.0, 100.0, 200.0])
    ys = np.array([-100.0, 0.0, 100.0])
    pts = [(x, y, z) for z in (0.0, 50.0) for y in ys for x in xs]
    return Workload(name="prism_ore_body", lo=(-1000.0, -1000.0, -1000.0), hi=(1000.0, 1000.0, 200.0),
                    rho_kind="prism", g_kind="prism", G=G_SI, stations=np.array(pts),
                    dt=step * step, h=1.0, seed=seed, paths=paths, rho0=500.0,
                    plo=(-100.0, -100.0, -250.0), phi=(100.0, 100.0, -150.0))


def voxel_survey(paths: int = 1_000_000, seed: int = 0, step: float = 10.0, grid_seed: int = 0,
                 shape=(128, 128, 64), table_n=(256, 256), n_side: int = 16) -> Workload:
    """Gaussian-random-field density on a voxel grid over [-2000,2000]^2 x
    [-2000,0] m inside Omega = [-2000,2000]^2 x [-2000,200] m (200 m of air);
    tabulated boundary data; an n_side x n_side station grid at z = 0 with
    125 m spacing (scaled with n_side) centred on the origin; h = 1 m."""
    nx, ny, nz = shape
    spacing = (4000.0 / nx, 4000.0 / ny, 2000.0 / nz)
    sp = 2000.0 / n_side
    c = -1000.0 + sp / 2 + sp * np.arange(n_side)
    pts = [(x, y, 0.0) for y in c for x in c]
    return Workload(name="voxel_survey", lo=(-2000.0, -2000.0, -2000.0), hi=(2000.0, 2000.0, 200.0),
                    rho_kind="voxel", g_kind="table", G=G_SI, stations=np.array(pts),
                    dt=step * step, h=1.0, seed=seed, paths=paths,
                    grid_shape=(nx, ny, nz), grid_origin=(-2000.0, -2000.0, -2000.0),
                    grid_spacing=spacing, grid_seed=grid_seed, table_n=table_n)


def large_survey(paths: int = 1_000_000, seed: int = 0, step: float = 10.0, grid_seed: int = 0,
                 shape=(128, 128, 64), table_n=(256, 256)) -> Workload:
    """The voxel model of voxel_survey with 2 x 10^4 stations: a 100 x 100
    surface grid at 20 m spacing (x, y = -990 + 20 i) at z = 0 and the same
    grid airborne at z = +100 m."""
    base = voxel_survey(paths=paths, seed=seed, step=step, grid_seed=grid_seed, shape=shape, table_n=table_n)
    c = -990.0 + 20.0 * np.arange(100)
    pts = [(x, y, z) for z in (0.0, 100.0) for y in c for x in c]
    return base.with_(name="large_survey", stations=np.array(pts))


def paper_cube_ball(paths: int = 4096, seed: int = 0, step: float = 20.0, line: str = "horizontal",
                    R: float = 10_000.0) -> Workload:
    """The paper's own experiment (Sec. 3): a cube [0,100]^3 m of density
    2000 kg/m^3 inside a ball of radius 10 km with zero Dirichlet data.
    Experiment 1: stations on y = 50, z = 200, x = -100 .. 200 step 10 (31
    points); experiment 2: the vertical line x = y = 50, z = -100 .. 200 step
    10.  The paper's time step is given without units; here the step length
    sigma sqrt(dt) is stated in metres."""
    t = -100.0 + 10.0 * np.arange(31)
    if line == "horizontal":
        pts = np.stack([t, np.full(31, 50.0), np.full(31, 200.0)], axis=1)
    else:
        pts = np.stack([np.full(31, 50.0), np.full(31, 50.0), t], axis=1)
    return Workload(name="paper_cube_ball", lo=(-R, -R, -R), hi=(R, R, R), rho_kind="prism", g_kind="zero",
                    G=G_SI, stations=pts, dt=step * step, h=1.0, seed=seed, paths=paths, rho0=2000.0,
                    plo=(0.0, 0.0, 0.0), phi=(100.0, 100.0, 100.0), domain="ball", ball_radius=R)


def unit_box(stations, rho_kind="none", g_kind="poly", poly=(0.0,) * 11, dt=1e-2, paths=4000,
             seed=7, clip=0, crn=1, h=0.05, rho0=0.0, half=1.0, plo=None, phi=None) -> Workload:
    """Small test problems on the cube [-half, half]^3 (G = 1)."""
    lo = (-half,) * 3
    hi = (half,) * 3
    return Workload(name="unit_box", lo=lo, hi=hi, rho_kind=rho_kind, g_kind=g_kind, G=1.0,
                    stations=np.asarray(stations, dtype=np.float64).reshape(-1, 3), dt=dt, h=h,
                    seed=seed, paths=paths, rho0=rho0, poly=tuple(poly), clip=clip, crn=crn,
                    plo=plo if plo is not None else tuple(-10 * half for _ in range(3)),
                    phi=phi if phi is not None else tuple(10 * half for _ in range(3)))
