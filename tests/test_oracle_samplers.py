"""Pins of the oracle's two table-driven samplers (CPU only).

* Dirichlet data read from face tables (MCG_G_TABLE): six node-centred
  tables, face order -x, +x, -y, +y, -z, +z; face +-x tabulated over (y, z),
  +-y over (x, z), +-z over (x, y); u is the fast index; read bilinearly; a
  point on two faces takes the face of the lowest axis.  Each face's table is
  filled from its own asymmetric bilinear function of the node indices, so
  bilinear interpolation reproduces that function exactly everywhere on the
  face; a swapped u / v axis, a swapped face, a transposed table or a wrong
  clamp at the last node changes the value by O(1).
* Voxel density (MCG_RHO_VOXEL): grid[ix + nx (iy + ny iz)] on half-open
  cells [origin + i spacing, origin + (i + 1) spacing), 0 outside.  Every
  cell holds a different value, so a wrong stride or axis fails.

Both are the boundary-data and density readings that the walk uses on the
heterogeneous workloads (Sec. 2.3 step 3 reads rho along the path; the
Dirichlet data enter Eq. 5 at the exit point).
"""
import itertools

import numpy as np
import pytest

import oracle

LO = (-3.0, -2.0, -1.5)
HI = (4.0, 5.0, 2.5)
NU, NV = 7, 5                       # u and v node counts differ on purpose
UV_AXES = {0: (1, 2), 1: (0, 2), 2: (0, 1)}   # face axis k -> (u axis, v axis)


def face_coeffs():
    """Per face: value(i, j) = a + b i + c j + d i j at node (u index i, v
    index j).  Small integers: every node value is exact in float32."""
    return [(10.0 * (f + 1), 1.0 + f, -(2.0 + 3 * f), 0.5 * (f + 2)) for f in range(6)]


def tables():
    t = np.empty((6, NV, NU), dtype=np.float32)
    i = np.arange(NU)[None, :]
    j = np.arange(NV)[:, None]
    for f, (a, b, c, d) in enumerate(face_coeffs()):
        t[f] = a + b * i + c * j + d * i * j
    return t


def spec_table():
    return oracle.Spec(lo=LO, hi=HI, g_kind=oracle.G_TABLE, faces=tables())


def expected_on_face(f, x):
    """The face's bilinear function at the boundary point x (continuous node
    coordinates along the face's documented u / v axes)."""
    k = f // 2
    ua, va = UV_AXES[k]
    i = (x[ua] - LO[ua]) / (HI[ua] - LO[ua]) * (NU - 1)
    j = (x[va] - LO[va]) / (HI[va] - LO[va]) * (NV - 1)
    a, b, c, d = face_coeffs()[f]
    return a + b * i + c * j + d * i * j


def expected(x):
    """The value the documented reading gives at a boundary point: the face
    of the lowest axis on which x lies on lo or hi."""
    for k in range(3):
        if x[k] == LO[k]:
            return expected_on_face(2 * k, x)
        if x[k] == HI[k]:
            return expected_on_face(2 * k + 1, x)
    raise ValueError("not on the boundary")


def point_on_face(f, s, t):
    """Boundary point of face f at fractions (s, t) of its u / v extents."""
    k = f // 2
    ua, va = UV_AXES[k]
    x = [0.0, 0.0, 0.0]
    x[k] = HI[k] if f % 2 else LO[k]
    x[ua] = LO[ua] + s * (HI[ua] - LO[ua])
    x[va] = LO[va] + t * (HI[va] - LO[va])
    return x


@pytest.mark.parametrize("f", range(6))
def test_table_interior_points_reproduce_the_face_function(f):
    rng = np.random.default_rng(100 + f)
    sp = spec_table()
    for s, t in rng.uniform(0.001, 0.999, size=(40, 2)):
        x = point_on_face(f, s, t)
        assert oracle.g(sp, x) == pytest.approx(expected_on_face(f, x), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("f", range(6))
def test_table_nodes_and_the_last_node_clamp(f):
    """At a node the reading is the stored value; at the far edge (u index
    nu - 1 or v index nv - 1) the cell index is clamped to the last cell and
    the weight is 1.  Nodes on the face's rim also lie on a face of a lower
    axis where the rim is shared with one; those take that face's value."""
    sp = spec_table()
    t = tables()
    k = f // 2
    ua, va = UV_AXES[k]
    checked = 0
    for i, j in itertools.product(range(NU), range(NV)):
        x = point_on_face(f, i / (NU - 1), j / (NV - 1))
        # node coordinates are not exact binary fractions: compare at rounding level
        if (x[ua] in (LO[ua], HI[ua]) and ua < k) or (x[va] in (LO[va], HI[va]) and va < k):
            assert oracle.g(sp, x) == pytest.approx(expected(x), rel=1e-12, abs=1e-12)
            continue
        assert oracle.g(sp, x) == pytest.approx(float(t[f, j, i]), rel=1e-12, abs=1e-12)
        checked += 1
    assert checked >= (NU - 2) * (NV - 2)


def test_edge_point_takes_the_lowest_axis_face():
    """A point on two faces: face_of picks the lowest axis (x before y before
    z), and the values of the two faces differ there, so the rule is seen."""
    sp = spec_table()
    rng = np.random.default_rng(7)
    for _ in range(20):
        x = [rng.uniform(LO[0], HI[0]), rng.uniform(LO[1], HI[1]), rng.uniform(LO[2], HI[2])]
        x[0] = HI[0]                           # on +x ...
        x[2] = LO[2]                           # ... and on -z
        got = oracle.g(sp, x)
        assert got == pytest.approx(expected_on_face(1, x), rel=1e-12, abs=1e-12)
        assert abs(expected_on_face(1, x) - expected_on_face(4, x)) > 1.0
        y = list(x)
        y[0] = 0.3                             # only on -z now
        assert oracle.g(sp, y) == pytest.approx(expected_on_face(4, y), rel=1e-12, abs=1e-12)
    corner = [LO[0], HI[1], HI[2]]             # -x, +y, +z: the x face wins
    assert oracle.g(sp, corner) == pytest.approx(expected_on_face(0, corner), rel=1e-12)


def test_table_off_the_boundary_is_nan():
    assert np.isnan(oracle.g(spec_table(), [0.1, 0.2, 0.3]))


def test_swapped_axes_would_be_seen():
    """Guard of the pin itself: the functions used above distinguish the u and
    v axes and the faces (a reading with u and v exchanged, or from the
    opposite face, differs by more than 1 somewhere on every face)."""
    rng = np.random.default_rng(3)
    for f in range(6):
        k = f // 2
        ua, va = UV_AXES[k]
        worst_swap, worst_face = 0.0, 0.0
        for s, t in rng.uniform(0, 1, size=(20, 2)):
            x = point_on_face(f, s, t)
            y = point_on_face(f, t, s)
            worst_swap = max(worst_swap, abs(expected_on_face(f, x) - expected_on_face(f, y)))
            worst_face = max(worst_face, abs(expected_on_face(f, x) - expected_on_face(f ^ 1, x)))
        assert worst_swap > 1.0 and worst_face > 1.0


# --- voxel density -------------------------------------------------------------

NX, NY, NZ = 4, 3, 2
ORG = (-1.5, 2.0, -0.25)
SP = (0.5, 0.75, 1.25)                     # binary fractions: cell faces are exact


def grid():
    g = np.empty((NZ, NY, NX), dtype=np.float32)
    for iz, iy, ix in itertools.product(range(NZ), range(NY), range(NX)):
        g[iz, iy, ix] = 1 + ix + 10 * iy + 100 * iz
    return g


def spec_voxel():
    return oracle.Spec(lo=(-10.0,) * 3, hi=(10.0,) * 3, rho_kind=oracle.RHO_VOXEL, grid=grid(), origin=ORG,
                       spacing=SP)


def cell_value(ix, iy, iz):
    return float(1 + ix + 10 * iy + 100 * iz)


def test_voxel_cell_interiors_x_fastest():
    sp = spec_voxel()
    for iz, iy, ix in itertools.product(range(NZ), range(NY), range(NX)):
        x = [ORG[0] + (ix + 0.5) * SP[0], ORG[1] + (iy + 0.5) * SP[1], ORG[2] + (iz + 0.5) * SP[2]]
        assert oracle.rho(sp, x) == cell_value(ix, iy, iz)


def test_voxel_cells_are_half_open():
    """A point exactly on a cell's lower face belongs to that cell; on its
    upper face, to the next cell; the grid's upper face is outside (0)."""
    sp = spec_voxel()
    n = (NX, NY, NZ)
    for axis in range(3):
        for i in range(n[axis] + 1):
            idx = [1 if n[a] > 1 else 0 for a in range(3)]
            idx[axis] = i
            x = [ORG[a] + (idx[a] + 0.5) * SP[a] for a in range(3)]
            x[axis] = ORG[axis] + i * SP[axis]            # exactly on the face between cells i-1 and i
            want = cell_value(*idx) if i < n[axis] else 0.0
            assert oracle.rho(sp, x) == want, (axis, i)
            x[axis] -= SP[axis] / 1024                     # just below (exactly): cell i - 1 (or outside)
            idx[axis] = i - 1
            want = cell_value(*idx) if i >= 1 else 0.0
            assert oracle.rho(sp, x) == want, (axis, i, "below")


def test_voxel_outside_the_grid_is_zero():
    sp = spec_voxel()
    inside = [ORG[a] + 0.5 * SP[a] for a in range(3)]
    assert oracle.rho(sp, inside) == cell_value(0, 0, 0)
    ext = (NX, NY, NZ)
    for axis in range(3):
        for v in (ORG[axis] - 1e-9, ORG[axis] - 3.0, ORG[axis] + ext[axis] * SP[axis] + 1e-9, 9.0):
            x = list(inside)
            x[axis] = v
            assert oracle.rho(sp, x) == 0.0
