"""Pins of the oracle's closed forms (CPU only).

The prism potential (Nagy's corner function, the analytic solution the paper
compares its walks against, Sec. 1 and Sec. 4.2) and the homogeneous sphere
are pinned by properties the mathematics fixes, not by retyping them:
far field -> point mass, additivity under subdivision, the finite-difference
Laplacian (= 4 pi G rho inside, 0 outside), dPhi/dz against the g_z closed
form, continuity, and symmetry.
"""
import numpy as np
import pytest

import oracle

G = 6.6743e-11


def fd_laplacian(f, x, h):
    x = np.asarray(x, float)
    s = -6 * f(x)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        s += f(x + e) + f(x - e)
    return s / h**2


def fd_dz(f, x, h):
    x = np.asarray(x, float)
    e = np.array([0.0, 0.0, h])
    return (f(x + e) - f(x - e)) / (2 * h)


LO, HI = (-100.0, -80.0, -250.0), (100.0, 120.0, -150.0)


def test_prism_far_field_point_mass():
    """Monopole + quadrupole of a uniform a x b x c box: Q_kk = M (3 a_k^2 -
    sum a^2) / 12, off-diagonal 0; the next term is O((L/r)^4) ~ 1e-8 here."""
    M = 500.0 * 200 * 200 * 100
    sides = np.array([HI[k] - LO[k] for k in range(3)])
    Q = M * (3 * sides**2 - np.sum(sides**2)) / 12.0
    c = np.array([(LO[k] + HI[k]) / 2 for k in range(3)])
    for d in ([20000.0, 0, 0], [0, 0, 20000.0], [12000.0, -9000.0, 11000.0]):
        x = c + np.array(d)
        dx = x - c
        r = np.linalg.norm(dx)
        want = -G * M / r - G / (2 * r**5) * np.sum(Q * dx**2)
        phi = oracle.prism_phi(G, 500.0, LO, HI, x)
        assert abs(phi - want) < 2e-8 * abs(want)
        gz = oracle.prism_gz(G, 500.0, LO, HI, x)
        qd = np.sum(Q * dx**2)
        want_gz = G * M * dx[2] / r**3 - G * Q[2] * dx[2] / r**5 + 2.5 * G * qd * dx[2] / r**7
        assert abs(gz - want_gz) < 2e-8 * G * M / r**2
    # a cube has no quadrupole: the point mass alone to O((L/r)^4)
    lo, hi = (-50.0, -50.0, -50.0), (50.0, 50.0, 50.0)
    for x in ([5000.0, 0, 0], [3000.0, 3000.0, -3000.0]):
        r = np.linalg.norm(x)
        assert abs(oracle.prism_phi(G, 500.0, lo, hi, x) + G * 500.0 * 1e6 / r) < 1e-8 * G * 5e8 / r


@pytest.mark.parametrize("x", [(0.0, 0.0, 0.0), (150.0, -30.0, -200.0), (5.0, 7.0, -190.0),
                               (100.0, 120.0, -150.0), (-300.0, 400.0, 50.0)])
def test_prism_additivity(x):
    whole = oracle.prism_phi(G, 500.0, LO, HI, x)
    mid = [(a + b) / 2 for a, b in zip(LO, HI)]
    parts = 0.0
    for i in range(2):
        for j in range(2):
            for k in range(2):
                lo = (LO[0] if i == 0 else mid[0], LO[1] if j == 0 else mid[1], LO[2] if k == 0 else mid[2])
                hi = (mid[0] if i == 0 else HI[0], mid[1] if j == 0 else HI[1], mid[2] if k == 0 else HI[2])
                parts += oracle.prism_phi(G, 500.0, lo, hi, x)
    assert abs(parts - whole) <= 1e-11 * abs(whole)


@pytest.mark.parametrize("x,inside", [((0.0, 10.0, -200.0), True), ((60.0, -50.0, -170.0), True),
                                      ((0.0, 0.0, 0.0), False), ((300.0, 0.0, -200.0), False),
                                      ((0.0, 0.0, -400.0), False)])
def test_prism_laplacian(x, inside):
    f = lambda y: oracle.prism_phi(G, 500.0, LO, HI, y)
    lap = fd_laplacian(f, x, 0.5)
    want = 4 * np.pi * G * 500.0 if inside else 0.0
    assert abs(lap - want) < 2e-4 * 4 * np.pi * G * 500.0


@pytest.mark.parametrize("x", [(0.0, 0.0, 0.0), (0.0, 0.0, 50.0), (-200.0, 100.0, 0.0), (30.0, 20.0, -200.0),
                               (100.0, 0.0, 0.0), (100.0, 120.0, -100.0), (0.0, 300.0, -250.0)])
def test_prism_gz_matches_fd(x):
    """Includes points above source edges and on the planes of faces, where the
    corner function has removable singularities (Sec. 4.2)."""
    f = lambda y: oracle.prism_phi(G, 500.0, LO, HI, y)
    fd = fd_dz(f, x, 0.01)
    gz = oracle.prism_gz(G, 500.0, LO, HI, x)
    assert abs(gz - fd) < 1e-6 * abs(gz) + 1e-16


def test_prism_symmetry_and_sign():
    lo, hi = (-100.0, -100.0, -250.0), (100.0, 100.0, -150.0)
    a = oracle.prism_phi(G, 500.0, lo, hi, (37.0, 11.0, 0.0))
    b = oracle.prism_phi(G, 500.0, lo, hi, (-37.0, 11.0, 0.0))
    c = oracle.prism_phi(G, 500.0, lo, hi, (11.0, 37.0, 0.0))
    assert a < 0
    assert abs(a - b) < 1e-13 * abs(a) and abs(a - c) < 1e-13 * abs(a)
    # above the body g_z = dPhi/dz > 0 (z up), below it < 0
    assert oracle.prism_gz(G, 500.0, lo, hi, (0, 0, 0)) > 0
    assert oracle.prism_gz(G, 500.0, lo, hi, (0, 0, -400)) < 0


def test_sphere_closed_form():
    c, a = (0.0, 0.0, 0.0), 0.25
    M = 4 / 3 * np.pi * a**3
    f = lambda y: oracle.sphere_phi(1.0, 1.0, c, a, y)
    # worked values quoted for the sphere workload: z = 0.3 on the axis
    assert abs(f((0, 0, 0.3)) - (-M / 0.3)) < 1e-15
    assert abs(oracle.sphere_gz(1.0, 1.0, c, a, (0, 0, 0.3)) - M / 0.09) < 1e-14
    # continuity at r = a, Laplacian 4 pi inside / 0 outside, g_z = dPhi/dz
    assert abs(f((0, 0, a * (1 - 1e-12))) - f((0, 0, a))) < 1e-10
    assert abs(fd_laplacian(f, (0.05, 0.02, -0.1), 1e-3) - 4 * np.pi) < 1e-4
    assert abs(fd_laplacian(f, (0.5, 0.2, -0.1), 1e-3)) < 1e-4
    for x in [(0.0, 0.0, 0.3), (0.1, 0.05, -0.12), (0.2, -0.3, 0.4)]:
        assert abs(oracle.sphere_gz(1.0, 1.0, c, a, x) - fd_dz(f, x, 1e-5)) < 1e-7


def test_sphere_equals_many_small_prisms_far_away():
    """A sphere and a cube of the same mass agree in the far field."""
    a = 10.0
    M = 4 / 3 * np.pi * a**3 * 500.0
    L = (4 / 3 * np.pi) ** (1 / 3) * a
    x = (0.0, 0.0, 5000.0)
    ps = oracle.sphere_phi(G, 500.0, (0, 0, 0), a, x)
    pp = oracle.prism_phi(G, 500.0, (-L / 2,) * 3, (L / 2,) * 3, x)
    assert abs(ps - pp) < 1e-8 * abs(ps)
    assert abs(ps + G * M / 5000.0) < 1e-12 * abs(ps)
