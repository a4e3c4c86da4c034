"""Device-resident solve through the C ABI (torch provides memory and streams).

``DeviceSolve`` owns the per-path buffers of one launch (S stations x N paths),
the running station states and the status / work-counter words, and calls
mcg_walk -> mcg_reduce -> mcg_finalize.  Nothing here computes: it allocates,
passes pointers, and reads results back.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mcgrav as M


def packed(w, grid, faces, stream=None):
    """Packed copies of a device voxel grid and device boundary tables for the
    walk's 16-byte loads (mcg_voxel_pack / mcg_table_pack): (zpack, quads),
    None where the workload has no such array or the packed grid does not
    apply (h > half a cell height)."""
    zpack = quads = None
    if grid is not None and w.rho_kind == "voxel" and grid.is_cuda and w.h <= 0.5 * w.grid_spacing[2]:
        nz, ny, nx = grid.shape
        zpack = torch.empty(M.mcg_voxel_pack_bytes(nx, ny, nz) // 4, dtype=torch.float32, device=grid.device)
        M.mcg_voxel_pack(M.problem(w.with_(g_kind="zero"), grid=grid), zpack, stream)
    if faces is not None and w.g_kind == "table" and faces.is_cuda:
        quads = torch.empty(M.mcg_table_pack_bytes(faces.shape[2], faces.shape[1]) // 4, dtype=torch.float32,
                            device=faces.device)
        M.mcg_table_pack(M.problem(w.with_(rho_kind="none"), faces=faces), quads, stream)
    return zpack, quads


class DeviceSolve:
    def __init__(self, w, stations=None, batch: int | None = None, precision: int = M.MCG_MIXED,
                 grid=None, faces=None, device: str = "cuda", stream=None, block: int = 0, pack: bool = True):
        self.w = w
        self.dev = torch.device(device)
        st = np.asarray(w.stations if stations is None else stations, dtype=np.float64).reshape(-1, 3)
        self.S = st.shape[0]
        self.stations = torch.from_numpy(st).to(self.dev)
        self.batch = int(batch or w.paths)
        self.precision = precision
        self.stream = stream
        zpack, quads = packed(w, grid, faces, stream) if pack else (None, None)
        self.prob = M.problem(w, grid=grid, faces=faces, zpack=zpack, quads=quads)
        self.opts = M.options(w, precision=precision, stream=stream, block=block)
        n = self.S * self.batch
        self.pp_u = torch.empty(n, dtype=torch.float64, device=self.dev)
        self.pp_d = torch.empty(n, dtype=torch.float64, device=self.dev)
        self.pp_steps = torch.empty(n, dtype=torch.int64, device=self.dev)
        self.states = torch.zeros(self.S * M.STATE_BYTES // 8, dtype=torch.float64, device=self.dev)
        self.status = torch.zeros(2, dtype=torch.int32, device=self.dev)
        self.counter = torch.zeros(1, dtype=torch.int64, device=self.dev)
        self.res = torch.empty((6, self.S), dtype=torch.float64, device=self.dev)
        wb = M.mcg_walk_work_bytes(self.S, self.batch, precision)
        # torch allocations are 512-byte aligned, as mcg_walk requires
        self.work = torch.empty(max(wb, 1), dtype=torch.uint8, device=self.dev) if wb else None

    def reset(self):
        self.states.zero_()
        self.status.zero_()

    def walk(self, p0: int, N: int | None = None):
        """Launch the walk for paths p0 .. p0+N-1 of every station."""
        N = self.batch if N is None else N
        M.mcg_walk(self.prob, self.stations, self.S, p0, N, self.w.dt, self.w.seed, self.opts,
                   self.pp_u, self.pp_d, self.pp_steps, self.work, self.status, self.counter)
        return N

    def reduce(self, N: int | None = None):
        N = self.batch if N is None else N
        M.mcg_reduce(self.pp_u, self.pp_d, self.pp_steps, self.S, N, self.states, self.stream)

    def finalize(self):
        r = self.res
        M.mcg_finalize(self.states, self.S, r[0], r[1], r[2], r[3], r[4], r[5], self.stream)

    def run(self, paths: int | None = None, p0: int = 0):
        """Whole solve over paths p0 .. p0+paths-1 in batches; returns host dict."""
        paths = self.w.paths if paths is None else paths
        self.reset()
        done = 0
        while done < paths:
            nb = min(self.batch, paths - done)
            self.walk(p0 + done, nb)
            self.reduce(nb)
            done += nb
        self.finalize()
        return self.result()

    def result(self):
        torch.cuda.synchronize(self.dev)
        r = self.res.cpu().numpy()
        return {"u": r[0].copy(), "gz": r[1].copy(), "se_u": r[2].copy(), "se_gz": r[3].copy(),
                "n_paths": r[4].view(np.int64).copy(), "path_steps": r[5].view(np.int64).copy(),
                "status": int(self.status[0].item())}

    def per_path(self, N: int | None = None):
        N = self.batch if N is None else N
        torch.cuda.synchronize(self.dev)
        k = self.S * N
        return (self.pp_u[:k].cpu().numpy().reshape(self.S, N), self.pp_d[:k].cpu().numpy().reshape(self.S, N),
                self.pp_steps[:k].cpu().numpy().reshape(self.S, N))


def voxel_model(w, device: str = "cuda", stream=None, near_cells: float = 4.0):
    """Device-resident heterogeneous model of a voxel workload: the GRF density
    grid [nz, ny, nx] and the boundary tables [6, nv, nu] (float32), built by
    mcg_grf_density and mcg_boundary_tables."""
    nx, ny, nz = w.grid_shape
    dev = torch.device(device)
    grid = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
    work = torch.empty(M.mcg_grf_work_bytes(nx, ny, nz), dtype=torch.uint8, device=dev)
    M.mcg_grf_density(w.grid_seed, nx, ny, nz, w.grid_sigma_vox, w.grid_amp, grid, work, stream)
    nu, nv = w.table_n
    faces = torch.empty((6, nv, nu), dtype=torch.float32, device=dev)
    prob = M.problem(w.with_(g_kind="zero"), grid=grid)
    M.mcg_boundary_tables(prob, nu, nv, near_cells, faces, stream)
    return grid, faces
