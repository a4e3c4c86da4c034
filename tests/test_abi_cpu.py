"""The C-ABI library builds, loads and exports every symbol include/mcgrav.h
declares; the ctypes structures match the C layout; host-side argument checks
answer without a GPU.  No compute call is made here."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1709_07469_gb300 import build as B
from paper_1709_07469_gb300 import mcgrav as M
from paper_1709_07469_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.load()


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        names += re.findall(r"^MCG_API\s+[\w\s\*]+?\b(mcg\w*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "mcgrav_solve" in names and "mcg_walk" in names
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    structs = {"mcg_domain": M.mcg_domain, "mcg_density": M.mcg_density, "mcg_boundary": M.mcg_boundary,
               "mcg_options": M.mcg_options, "mcg_result": M.mcg_result, "mcg_station_state": M.mcg_station_state,
               "mcg_server_config": M.mcg_server_config}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mcgrav.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.split("\n") if l)
    for name, cls in structs.items():
        assert int(out[name]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_defaults_and_workspace(lib):
    o = M.mcg_options()
    lib.mcg_options_default(C.byref(o))
    assert o.h == 1e-2 and o.sigma == 1.0 and o.precision == M.MCG_MIXED and o.clip == 1 and o.crn_gz == 1
    assert o.max_steps == 1 << 31
    assert o.graph == 1 and o.refill_min == 1 and o.bridge == 0 and o.migrate == 1
    assert M.mcg_workspace_bytes(0, 10) == 0
    b = M.mcg_workspace_bytes(30, 1000)
    # two per-batch sets; per path: u, d, steps (24 B) + the mixed walk's exit
    # records (3 x 32 B) + a migration-pool slot (80 B) and its ready flag (4 B)
    assert b >= 2 * 30 * 1000 * 204 and b < 2 * 30 * 1000 * 204 + 64 * 1024
    assert M.mcg_walk_work_bytes(30, 1000, M.MCG_FP64) == 0
    assert M.mcg_walk_work_bytes(30, 1000, M.MCG_MIXED) >= 30 * 1000 * 180
    # the pool stops growing at 2^19 slots
    big = M.mcg_walk_work_bytes(1000, 10_000, M.MCG_MIXED)
    assert big >= 10**7 * 96 + (1 << 19) * 84 and big < 10**7 * 96 + (1 << 19) * 84 + 64 * 1024
    assert "sm_103a" in M.version()


def _solve_status(w, **kw):
    prob = M.problem(w)
    opts = M.options(w, **kw)
    lib = M.load()
    st = np.ascontiguousarray(w.stations, dtype=np.float64)
    res = M.mcg_result()
    return lib.mcgrav_solve(C.byref(prob.domain), C.byref(prob.density), C.byref(prob.boundary), st.ctypes.data,
                            st.shape[0], w.paths, w.dt, 0, C.byref(opts), C.byref(res))


def test_argument_checks_without_gpu(lib):
    w = W.sphere_line(paths=10)
    assert _solve_status(w.with_(dt=-1.0)) == M.MCG_ERR_ARG
    assert "dt" in M.last_error()
    assert _solve_status(w.with_(stations=np.array([[0.0, 0.0, 1.0]]))) == M.MCG_ERR_ARG
    assert "inside" in M.last_error()
    assert _solve_status(w.with_(stations=np.array([[0.0, 0.0, 0.995]]))) == M.MCG_ERR_ARG  # +h copy outside
    assert _solve_status(w.with_(lo=(1.0, -1.0, -1.0))) == M.MCG_ERR_ARG
    assert _solve_status(w.with_(g_kind="prism")) == M.MCG_ERR_ARG
    assert _solve_status(w, block=48) == M.MCG_ERR_ARG
    assert _solve_status(w, precision=7) == M.MCG_ERR_ARG
    assert _solve_status(w.with_(paths=0)) == M.MCG_ERR_ARG
    # empty station list is a no-op
    assert _solve_status(w.with_(stations=np.zeros((0, 3)))) == M.MCG_OK


def test_product_path_fails_loudly_without_library(tmp_path):
    saved = M._lib
    try:
        M._lib = None
        with pytest.raises(ImportError):
            M.load(str(tmp_path / "missing.so"))
    finally:
        M._lib = saved


def test_new_entry_points_check_arguments_without_gpu(lib):
    """Host-side checks of the packed-array, exact-field, probe and server
    entry points answer before any launch."""
    assert M.mcg_voxel_pack_bytes(128, 128, 64) == 16 * 128 * 128 * 66
    assert M.mcg_voxel_pack_bytes(0, 1, 1) == 0
    assert M.mcg_table_pack_bytes(256, 256) == 16 * 6 * 255 * 255
    assert M.mcg_table_pack_bytes(1, 5) == 0
    w = W.voxel_survey(shape=(4, 4, 2), table_n=(3, 3)).with_(g_kind="zero")
    grid = np.zeros((2, 4, 4), dtype=np.float32)
    prob = M.problem(w, grid=grid)
    with pytest.raises(M.McgError):                       # 16-byte alignment of the output
        M.mcg_voxel_pack(prob, grid.ctypes.data + 4)
    sph = M.problem(W.sphere_line())
    with pytest.raises(M.McgError):                       # not a voxel density
        M.mcg_voxel_pack(sph, grid.ctypes.data)
    assert M.mcg_field(sph, None, 0) == M.MCG_OK
    with pytest.raises(M.McgError):
        M.mcg_field(sph, None, -1, grid.ctypes.data)
    for kind in (-1, 3, 7):
        with pytest.raises(M.McgError):
            M.mcg_issue_probe(kind)
    c = M.server_config()
    assert c.batch == 1 and c.batch_items == 1 << 22 and c.walk.spill_max == 24
    assert c.walk.fault_unpublished == 0


def test_walk_option_ranges_without_gpu(lib):
    w = W.sphere_line(paths=10)
    assert _solve_status(w, fault_unpublished=256) == M.MCG_ERR_ARG
    assert "fault_unpublished" in M.last_error()
    assert _solve_status(w, spill_max=33) == M.MCG_ERR_ARG
    assert "spill_max" in M.last_error()


def test_walk_index_limits_without_gpu(lib):
    """Path indices are the 32-bit counter word p: p0 + N may reach 2^32 but
    not pass it; checked before any device pointer is touched."""
    w = W.sphere_line(paths=10)
    prob = M.problem(w)
    opts = M.options(w)
    fake = 0x1000  # never dereferenced: the checks fail first
    for p0, N in ((2**32 - 10, 11), (2**32, 1), (-1, 5)):
        rc = lib.mcg_walk(C.byref(prob.domain), C.byref(prob.density), C.byref(prob.boundary), fake, 8, p0, N,
                          w.dt, 0, C.byref(opts), fake, fake, fake, fake, fake, fake)
        assert rc == M.MCG_ERR_ARG, (p0, N)
        assert ("non-negative" if p0 < 0 else "32 bits") in M.last_error()


def test_density_at_checks_arguments_without_gpu(lib):
    w = W.sphere_line()
    prob = M.problem(w)
    for h, prec in ((0.01, 7), (-1.0, M.MCG_MIXED), (float("nan"), M.MCG_FP64)):
        with pytest.raises(M.McgError):
            M.mcg_density_at(prob, h, prec, None, 3, None)
    with pytest.raises(M.McgError):  # n > 0 with null buffers
        M.mcg_density_at(prob, 0.01, M.MCG_MIXED, None, 3, None)
    assert M.mcg_density_at(prob, 0.01, M.MCG_MIXED, None, 0, None) == M.MCG_OK
