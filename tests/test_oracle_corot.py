"""Pins of the oracle's co-rotational elements (Section 3.1, Eq. "eqmodel":
K0 = int B^T D B dV rotated per element by the polar decomposition of the
deformation gradient).

  * at rest the stiffness is the textbook linear-elastic one, equal to the
    St Venant-Kirchhoff tangent at rest (itself pinned against Voigt B^T D B);
  * a rigid motion gives zero force and the rotated rest stiffness;
  * frame indifference at a deformed state: f(Qx + c) = Q f(x),
    K(Qx + c) = Qb K(x) Qb^T;
  * the rotation is a proper rotation with R^T F symmetric positive definite;
  * small displacements: f = K0 u to second order;
  * K is symmetric.
"""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O

PRM = (3.4e3, 3.1e4, 0.0)


def _mesh(kind):
    return fi.tet_beam(2, 2, 3) if kind == "tet" else fi.hex_beam(2, 2, 3, jitter=0.1, seed=3)


def _rot(seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return Q * np.sign(np.linalg.det(Q))


def _deformed(mesh, amp=0.1, seed=0):
    rng = np.random.default_rng(seed)
    return mesh.X + amp * 0.01 * rng.standard_normal(mesh.X.shape)


@pytest.mark.parametrize("kind", ["tet", "hex"])
def test_rest_stiffness_is_linear_elasticity(kind):
    mesh = _mesh(kind)
    q = O.Quadrature(mesh.elem_type, mesh.X, mesh.conn)
    Kc = O.element_tangent(q, mesh.X, O.COROTATIONAL, PRM)
    Ks = O.element_tangent(q, mesh.X, O.SVK, PRM)
    np.testing.assert_allclose(Kc, Ks, rtol=1e-12, atol=1e-12 * np.abs(Ks).max())
    assert np.abs(O.element_force(q, mesh.X, O.COROTATIONAL, PRM)).max() <= 1e-12 * np.abs(Ks).max()


@pytest.mark.parametrize("kind", ["tet", "hex"])
def test_rigid_motion(kind):
    mesh = _mesh(kind)
    q = O.Quadrature(mesh.elem_type, mesh.X, mesh.conn)
    Q = _rot(1)
    x = mesh.X @ Q.T + np.array([0.3, -0.2, 0.1])
    K0 = O.element_tangent(q, mesh.X, O.COROTATIONAL, PRM)
    f = O.element_force(q, x, O.COROTATIONAL, PRM)
    assert np.abs(f).max() <= 1e-11 * np.abs(K0).max() * 0.01
    Qb = np.kron(np.eye(q.npe), Q)
    np.testing.assert_allclose(O.element_tangent(q, x, O.COROTATIONAL, PRM), Qb @ K0 @ Qb.T,
                               rtol=1e-11, atol=1e-11 * np.abs(K0).max())


@pytest.mark.parametrize("kind", ["tet", "hex"])
def test_frame_indifference(kind):
    mesh = _mesh(kind)
    q = O.Quadrature(mesh.elem_type, mesh.X, mesh.conn)
    x = _deformed(mesh, amp=0.2)
    Q, c = _rot(2), np.array([1.0, 2.0, -0.5])
    f, K = O.element_force(q, x, O.COROTATIONAL, PRM), O.element_tangent(q, x, O.COROTATIONAL, PRM)
    f2 = O.element_force(q, x @ Q.T + c, O.COROTATIONAL, PRM)
    K2 = O.element_tangent(q, x @ Q.T + c, O.COROTATIONAL, PRM)
    Qb = np.kron(np.eye(q.npe), Q)
    np.testing.assert_allclose(f2, np.einsum("mn,en->em", Qb, f), rtol=1e-10, atol=1e-10 * np.abs(f).max())
    np.testing.assert_allclose(K2, Qb @ K @ Qb.T, rtol=1e-10, atol=1e-10 * np.abs(K).max())
    np.testing.assert_allclose(K, np.swapaxes(K, 1, 2), rtol=0, atol=1e-12 * np.abs(K).max())


@pytest.mark.parametrize("kind", ["tet", "hex"])
def test_polar_rotation(kind):
    mesh = _mesh(kind)
    q = O.Quadrature(mesh.elem_type, mesh.X, mesh.conn)
    x = _deformed(mesh, amp=0.1, seed=4)
    assert np.linalg.det(q.deformation_gradient(x)).min() > 0
    R = O.corot_rotation(q, x)
    I = np.broadcast_to(np.eye(3), R.shape)
    np.testing.assert_allclose(R @ np.swapaxes(R, 1, 2), I, atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-13)
    F = q.deformation_gradient(x)
    Fb = np.einsum("eq,eqiJ->eiJ", q.w, F) / q.w.sum(axis=1)[:, None, None]
    S = np.swapaxes(R, 1, 2) @ Fb
    np.testing.assert_allclose(S, np.swapaxes(S, 1, 2), atol=1e-13 * np.abs(S).max())
    assert np.linalg.eigvalsh(0.5 * (S + np.swapaxes(S, 1, 2))).min() > 0


@pytest.mark.parametrize("kind", ["tet", "hex"])
def test_small_displacement_is_linear_elasticity(kind):
    mesh = _mesh(kind)
    q = O.Quadrature(mesh.elem_type, mesh.X, mesh.conn)
    K0 = O.element_tangent(q, mesh.X, O.COROTATIONAL, PRM)
    rng = np.random.default_rng(7)
    du = rng.standard_normal(mesh.X.shape) * 0.01
    errs = []
    for eps in (1e-3, 1e-4):
        x = mesh.X + eps * du
        ue = (x - mesh.X)[q.conn].reshape(q.conn.shape[0], -1)
        f = O.element_force(q, x, O.COROTATIONAL, PRM)
        errs.append(np.abs(f - np.einsum("emn,en->em", K0, ue)).max() / np.abs(f).max())
    # |f - K0 u| = O(eps^2) while |f| = O(eps): the relative gap falls like eps
    assert errs[1] < errs[0] * 0.2
