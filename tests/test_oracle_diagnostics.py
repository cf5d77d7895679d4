"""Pins of the oracle's diagnostic functions (area, volume, elastic energy).

These are the checkers of the GPU diagnostics (Sec. 5.1 area / volume
conservation, the energy of the force connections of Sec. 4.1), so each is
tied to something the mathematics fixes independently of its own formula:
closed-form areas and volumes of polygons and polyhedra, invariance under
translation, the sign flip under reversed orientation, the exact scaling of
volume by the determinant of a linear map, the O(nu^-2) convergence of a
geodesic sphere's volume to 4/3 pi R^3, and -- for the energy -- that its
gradient is minus the connection force of Step 2a (itself pinned against the
literal fiber form in test_oracle_pins.py).
"""
import numpy as np
import pytest

import oracle as O
from paper_1305_3976_gb300 import inputs as I


# ---------------------------------------------------------------------------
# 2D area from the directed edges of closed fibers


def _polygon(n, R, center):
    t = 2 * np.pi * np.arange(n) / n + 0.3
    X = np.stack([center[0] + R * np.cos(t), center[1] + R * np.sin(t)], axis=1)
    e = np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1).astype(np.int32)
    return X, e


@pytest.mark.parametrize("n", [3, 4, 7, 64, 1000])
def test_area_regular_polygon_closed_form(n):
    R = 0.37
    X, e = _polygon(n, R, (0.41, 0.63))
    exact = 0.5 * n * R * R * np.sin(2 * np.pi / n)
    assert O.area_2d(X, e) == pytest.approx(exact, rel=1e-13)
    # reversed orientation flips the sign; a translation changes nothing
    assert O.area_2d(X, e[:, ::-1].copy()) == pytest.approx(-exact, rel=1e-13)
    assert O.area_2d(X + np.array([3.0, -7.5]), e) == pytest.approx(exact, rel=1e-12)


def test_area_unit_square_and_ellipse_polygon():
    sq = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    e = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32)
    assert O.area_2d(sq, e) == 1.0
    # the Sec. 5.1 ellipse sampled at equal parameter steps is the affine image
    # diag(r1, r2) of a regular polygon: area r1 r2 (ns/2) sin(2 pi/ns)
    ns, r1, r2 = 256, 0.2, 0.25
    X = I.ellipse_points(ns, r1, r2)
    edges, _, _ = I.closed_fiber_connections(ns, 1.0)
    assert O.area_2d(X, edges) == pytest.approx(r1 * r2 * 0.5 * ns * np.sin(2 * np.pi / ns), rel=1e-13)


def test_area_sums_over_several_loops():
    X1, e1 = _polygon(12, 0.1, (0.25, 0.25))
    X2, e2 = _polygon(20, 0.15, (0.7, 0.6))
    X = np.concatenate([X1, X2])
    e = np.concatenate([e1, e2 + 12])
    a = 0.5 * 12 * 0.01 * np.sin(2 * np.pi / 12) + 0.5 * 20 * 0.0225 * np.sin(2 * np.pi / 20)
    assert O.area_2d(X, e) == pytest.approx(a, rel=1e-13)


# ---------------------------------------------------------------------------
# 3D volume from oriented triangles


def _outward(V, T):
    """Orient the triangles of a convex polyhedron away from its centroid."""
    T = T.copy()
    c = V.mean(axis=0)
    A, B, C = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(B - A, C - A), (A + B + C) / 3 - c) < 0
    T[flip] = T[flip][:, ::-1]
    return T


def _cube():
    V = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], dtype=np.float64)
    quads = [(0, 1, 3, 2), (4, 5, 7, 6), (0, 1, 5, 4), (2, 3, 7, 6), (0, 2, 6, 4), (1, 3, 7, 5)]
    T = np.array([t for a, b, c, d in quads for t in ((a, b, c), (a, c, d))], dtype=np.int32)
    return V, _outward(V, T)


def test_volume_unit_cube_box_and_translation():
    V, T = _cube()
    assert O.volume_3d(V, T) == pytest.approx(1.0, abs=1e-15)
    assert O.volume_3d(V, T[:, ::-1].copy()) == pytest.approx(-1.0, abs=1e-15)
    # a box of sides a, b, c anywhere in space
    s = np.array([0.3, 1.7, 0.45])
    assert O.volume_3d(V * s + np.array([5.0, -2.0, 11.0]), T) == pytest.approx(np.prod(s), rel=1e-12)


def test_volume_tetrahedron_is_determinant_over_six():
    rng = np.random.default_rng(3)
    for _ in range(5):
        P = rng.normal(size=(4, 3))
        T = _outward(P, np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]], np.int32))
        exact = abs(np.linalg.det(P[1:] - P[0])) / 6.0
        assert O.volume_3d(P, T) == pytest.approx(exact, rel=1e-12)


def test_volume_scales_with_the_determinant_of_a_linear_map():
    # ellipsoidal membranes are linear images of the geodesic sphere: the
    # enclosed volume scales exactly by det(M)
    V, T, _ = I.icosphere(6)
    v0 = O.volume_3d(V, T)
    M = np.array([[0.2, 0.03, 0.0], [0.0, 0.25, -0.04], [0.01, 0.0, 0.3]])
    assert O.volume_3d(V @ M.T + 0.5, T) == pytest.approx(np.linalg.det(M) * v0, rel=1e-12)


def test_geodesic_sphere_volume_converges_at_second_order():
    R = 0.3
    err = []
    for nu in (4, 8, 16):
        V, T, _ = I.icosphere(nu)
        err.append(4.0 / 3.0 * np.pi * R ** 3 - O.volume_3d(R * V + 0.5, T))
    assert all(e > 0 for e in err)                      # inscribed: always below the sphere
    assert 3.6 < err[0] / err[1] < 4.4 and 3.6 < err[1] / err[2] < 4.4, err
    assert err[2] < 5e-3 * 4.0 / 3.0 * np.pi * R ** 3


# ---------------------------------------------------------------------------
# elastic energy of the force connections


def test_energy_of_one_connection():
    X = np.array([[0.1, 0.2, 0.3], [0.4, 0.6, 0.3]])            # distance 0.5
    e = np.array([[0, 1]], np.int32)
    assert O.elastic_energy(X, e, np.array([3.0]), np.array([0.2])) == pytest.approx(0.5 * 3.0 * 0.09, rel=1e-15)
    assert O.elastic_energy(X, e, np.array([3.0])) == pytest.approx(0.5 * 3.0 * 0.25, rel=1e-15)


@pytest.mark.parametrize("dim,L", [(2, 0.0), (2, 0.5), (3, 0.0), (3, 0.5)])
def test_energy_gradient_is_minus_the_connection_force(dim, L):
    # G_a = -dE/dX_a for the connection force of Step 2a (Sec. 4.1, Fig. 3)
    rng = np.random.default_rng(10 + dim)
    if dim == 2:
        X = I.ellipse_points(40, 0.2, 0.27)
        e, k, r = I.closed_fiber_connections(40, 1.3, L)
    else:
        X, e, k, r, _ = I.ellipsoid_membrane(3, (0.2, 0.25, 0.3), (0.5, 0.5, 0.5))
        k = k * rng.uniform(0.5, 2.0, size=k.shape)
        r = r + L * 0.02
    X = X + rng.normal(scale=2e-3, size=X.shape)
    G = O.force_edges(X, e, k, r)
    step = 1e-6
    grad = np.zeros_like(X)
    for a in range(X.shape[0]):
        for c in range(dim):
            Xp, Xm = X.copy(), X.copy()
            Xp[a, c] += step
            Xm[a, c] -= step
            grad[a, c] = (O.elastic_energy(Xp, e, k, r) - O.elastic_energy(Xm, e, k, r)) / (2 * step)
    assert np.max(np.abs(grad + G)) < 1e-6 * np.max(np.abs(G)), np.max(np.abs(grad + G))
