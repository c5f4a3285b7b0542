"""Pins of the oracle's hexahedron quadrature (Section 3.1: trilinear hexes
integrated by 2x2x2 Gauss; Section 4.1: consistent mass) on distorted
elements, through the divergence theorem instead of a volume quadrature.

For a trilinear hex the faces are bilinear patches.  The volume and the first
moment of the solid follow from surface integrals over those patches:
    V = 1/3 sum_faces int x . (x_u x x_v) du dv,
    int x_i dV = sum_faces int (x_i^2 / 2) (x_u x x_v)_i du dv,
with polynomial integrands of degree <= 3 per variable, integrated exactly
here by 3-point Gauss-Legendre (a rule the oracle does not use).  The
consistent mass must reproduce both: sum_ab m_ab = rho V and
sum_ab m_ab X_b = rho int x dV (the shape functions sum to one and
interpolate x).  On undistorted cubes det J is constant, so a wrong Gauss
point, weight or Jacobian orientation can hide; jittered hexes expose it.
"""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O

# local corner order a = dx + 2 dy + 4 dz; each face as (fixed axis, side)
FACES = [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)]


def _corner(d):
    return d[0] + 2 * d[1] + 4 * d[2]


def _face_patch(Xe, axis, side):
    """Bilinear patch x(u, v) of one face, with (u, v) the two other axes in
    cyclic order, and the sign that makes x_u x x_v point outward."""
    a1, a2 = (axis + 1) % 3, (axis + 2) % 3
    P = np.zeros((2, 2, 3))
    for i in (0, 1):
        for j in (0, 1):
            d = [0, 0, 0]
            d[axis], d[a1], d[a2] = side, i, j
            P[i, j] = Xe[_corner(d)]
    return P, (1.0 if side == 1 else -1.0)


def _surface_integrals(Xe):
    g, w = np.polynomial.legendre.leggauss(3)
    t = 0.5 * (g + 1.0)          # points on [0, 1]
    wt = 0.5 * w
    V = 0.0
    mom = np.zeros(3)
    for axis, side in FACES:
        P, sgn = _face_patch(Xe, axis, side)
        for ui, wu in zip(t, wt):
            for vi, wv in zip(t, wt):
                x = ((1 - ui) * (1 - vi) * P[0, 0] + ui * (1 - vi) * P[1, 0]
                     + (1 - ui) * vi * P[0, 1] + ui * vi * P[1, 1])
                xu = (1 - vi) * (P[1, 0] - P[0, 0]) + vi * (P[1, 1] - P[0, 1])
                xv = (1 - ui) * (P[0, 1] - P[0, 0]) + ui * (P[1, 1] - P[1, 0])
                n = sgn * np.cross(xu, xv)
                V += wu * wv * np.dot(x, n) / 3.0
                mom += wu * wv * 0.5 * x * x * n
    return V, mom


@pytest.mark.parametrize("jitter,seed", [(0.0, 1), (0.2, 1), (0.3, 9)])
def test_hex_consistent_mass_volume_and_first_moment(jitter, seed):
    mesh = fi.hex_beam(2, 2, 3, jitter=jitter, seed=seed)
    rho = 1000.0
    m = O.element_mass(O.HEX8, mesh.X, mesh.conn, rho)          # [E, 8, 8] scalars
    for e in range(mesh.conn.shape[0]):
        Xe = mesh.X[mesh.conn[e]]
        V, mom = _surface_integrals(Xe)
        assert V > 0
        me = m[e]
        np.testing.assert_allclose(me.sum(), rho * V, rtol=1e-12)
        np.testing.assert_allclose(me.sum(axis=0) @ Xe, rho * mom, rtol=1e-11,
                                   atol=1e-12 * rho * V * np.abs(Xe).max())


def test_surface_route_is_exact_on_a_box():
    """The check itself on a box of known volume and centroid."""
    Xe = np.array([[dx * 2.0, dy * 3.0, dz * 5.0] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)])
    V, mom = _surface_integrals(Xe)
    assert abs(V - 30.0) < 1e-12
    np.testing.assert_allclose(mom, 30.0 * np.array([1.0, 1.5, 2.5]), rtol=1e-13)
