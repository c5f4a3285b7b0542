"""Pins of the oracle's contact step (Section "Lagrangian multipliers",
Eq. "KKT": free motion, compliance W = H A^{-1} H^T, projected Gauss-Seidel,
motion correction), against what the mathematics fixes:

  * the projected Gauss-Seidel solution equals the LCP solution found by
    brute-force enumeration of active sets (the LCP with a symmetric
    positive-definite W has exactly one solution);
  * the corrected motion satisfies the KKT system: A a - H^T lambda = b,
    lambda >= 0, end-of-step gap g = n . x - c >= 0, lambda . g = 0;
  * a single active contact lands its node exactly on the plane;
  * contacts far from the body give lambda = 0 and the free step exactly;
  * W is symmetric positive definite.
"""
import itertools

import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O


def _lcp_brute(W, r):
    m = W.shape[0]
    for k in range(m + 1):
        for S in itertools.combinations(range(m), k):
            S = list(S)
            lam = np.zeros(m)
            if S:
                lam[S] = np.linalg.solve(W[np.ix_(S, S)], r[S])
            w = W @ lam - r
            if lam.min() >= -1e-12 and w.min() >= -1e-10 * max(1.0, np.abs(r).max()):
                return lam
    raise AssertionError("no LCP solution found")


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_pgs_equals_brute_force_lcp(seed):
    rng = np.random.default_rng(seed)
    m = 7
    G = rng.standard_normal((m, m))
    W = G @ G.T + 0.5 * np.eye(m)
    r = rng.standard_normal(m)
    lam = O.pgs(W, r, 5000, 1e-15)
    ref = _lcp_brute(W, r)
    np.testing.assert_allclose(lam, ref, atol=1e-10 * max(1.0, np.abs(ref).max()))
    assert (lam > 0).any() and (lam == 0).any()


def _drop(model_id=O.NEOHOOKE):
    mesh = fi.tet_beam(2, 2, 6)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, model_id, (3.4e3, 3.1e4, 0.0),
                1000.0, 0.01, 0.1, 0.01)
    q = mesh.X.reshape(-1).copy()
    v = np.zeros_like(q)
    v.reshape(-1, 3)[:, 2] = -0.5 * mesh.X[:, 0] / mesh.X[:, 0].max()  # the free end moving down
    v[m.fixed_dofs] = 0.0
    p = fi.body_force(mesh, 1000.0, (0.0, 0.0, -9.81)).reshape(-1)
    bottom = np.nonzero((mesh.X[:, 2] == 0.0) & (mesh.X[:, 0] > 0.0))[0].astype(np.int32)
    return mesh, m, q, v, p, bottom


def test_kkt_and_complementarity():
    mesh, m, q, v, p, nodes = _drop()
    normals = np.tile([0.0, 0.0, 1.0], (len(nodes), 1))
    offsets = np.full(len(nodes), -0.002)   # a floor 2 mm below the beam's bottom face
    q1, v1, a, lam, W = m.contact_step(q, v, p, nodes, normals, offsets)
    _, _, a_free = m.step(q, v, p)
    gap_free = (q + 0.01 * (v + 0.01 * a_free)).reshape(-1, 3)[nodes, 2] - offsets
    assert gap_free.min() < 0                                 # the free motion penetrates
    A, b = m.system(q, v, p)
    H = m.contact_jacobian(nodes, normals)
    np.testing.assert_allclose(A @ a - H.T @ lam, b, atol=1e-9 * np.abs(b).max())
    gap = q1.reshape(-1, 3)[nodes, 2] - offsets
    assert lam.min() >= 0.0
    assert gap.min() >= -1e-12
    assert np.abs(lam * gap).max() <= 1e-9 * np.abs(lam).max() * 0.002
    assert (lam > 0).sum() >= 1 and (lam == 0).sum() >= 1


def test_single_contact_lands_on_the_plane():
    mesh, m, q, v, p, nodes = _drop()
    tip = nodes[np.argmax(mesh.X[nodes, 0])]
    q1, v1, a, lam, W = m.contact_step(q, v, p, [tip], [[0.0, 0.0, 1.0]], [-0.002])
    assert lam[0] > 0
    assert abs(q1[3 * tip + 2] - (-0.002)) <= 1e-12
    # closed form of the one-constraint LCP
    _, _, a_free = m.step(q, v, p)
    delta = (-0.002 - (q + 0.01 * v)[3 * tip + 2]) / 1e-4
    np.testing.assert_allclose(lam[0], (delta - a_free[3 * tip + 2]) / W[0, 0], rtol=1e-12)


def test_distant_contacts_change_nothing():
    mesh, m, q, v, p, nodes = _drop()
    normals = np.tile([0.0, 0.0, 1.0], (len(nodes), 1))
    q1, v1, a, lam, W = m.contact_step(q, v, p, nodes, normals, np.full(len(nodes), -1.0))
    qf, vf, af = m.step(q, v, p)
    assert np.all(lam == 0.0)
    np.testing.assert_array_equal(a, af)
    np.testing.assert_array_equal(q1, qf)


def test_compliance_is_spd():
    mesh, m, q, v, p, nodes = _drop()
    normals = np.tile([0.0, 0.0, 1.0], (len(nodes), 1))
    _, _, _, _, W = m.contact_step(q, v, p, nodes, normals, np.full(len(nodes), -0.002))
    np.testing.assert_allclose(W, W.T, rtol=1e-10, atol=1e-14 * np.abs(W).max())
    assert np.linalg.eigvalsh(0.5 * (W + W.T)).min() > 0
