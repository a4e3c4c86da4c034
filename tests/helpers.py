"""Test helpers: map a workload description onto the oracle's problem spec.

Only the tests use this module.  It holds no arithmetic of the method.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1709_07469_gb300.workloads import Workload

_RHO = {"none": oracle.RHO_NONE, "sphere": oracle.RHO_SPHERE, "prism": oracle.RHO_PRISM,
        "voxel": oracle.RHO_VOXEL}
_G = {"zero": oracle.G_ZERO, "sphere": oracle.G_SPHERE, "prism": oracle.G_PRISM,
      "table": oracle.G_TABLE, "poly": oracle.G_POLY}


def oracle_spec(w: Workload, grid=None, faces=None, ubits: int = 32, max_steps: int = 1 << 40) -> oracle.Spec:
    return oracle.Spec(
        lo=w.lo, hi=w.hi, domain_kind=1 if w.domain == "ball" else 0, bc=w.ball_center, R=w.ball_radius,
        rho_kind=_RHO[w.rho_kind], G=w.G, rho0=w.rho0, center=w.center,
        radius=w.radius, plo=w.plo, phi=w.phi, grid=grid, origin=w.grid_origin,
        spacing=w.grid_spacing, g_kind=_G[w.g_kind], faces=faces, poly=w.poly, dt=w.dt,
        sigma=w.sigma, h=w.h, seed=w.seed, clip=w.clip, crn=w.crn, ubits=ubits,
        max_steps=max_steps, bridge=w.bridge)


def smooth_tables(w: Workload, seed: int = 1, scale: float = 1e-4) -> np.ndarray:
    """A seeded smooth synthetic boundary table [6, nv, nu] (float32): a few
    low-order Fourier modes per face.  Used as plain input data for the walk
    parity tests; it is not a solution of anything."""
    rng = np.random.default_rng(seed)
    nu, nv = w.table_n
    s = np.linspace(0.0, 1.0, nu)[None, :]
    t = np.linspace(0.0, 1.0, nv)[:, None]
    out = np.empty((6, nv, nu), dtype=np.float32)
    for f in range(6):
        a = rng.normal(size=(3, 3))
        acc = np.full((nv, nu), -1.0)
        for i in range(3):
            for j in range(3):
                acc = acc + 0.1 * a[i, j] * np.cos(np.pi * i * s) * np.cos(np.pi * j * t)
        out[f] = (scale * acc).astype(np.float32)
    return out
