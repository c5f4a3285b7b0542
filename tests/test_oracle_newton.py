"""Pins of the oracle's multi-iteration Newton step (the backward-Euler step
solved beyond the paper's single linearisation).

  * one iteration is the paper's step (Eqs. "dynamic equation1"/"dynamic
    equation2");
  * without stiffness damping (beta = 0) the iteration is Newton's method on
    the nonlinear step residual, so the corrections converge quadratically
    and the residual, evaluated independently from the definition
    M a + f(q') + (alpha M + beta K(q')) v' - p, vanishes;
  * with stiffness damping the Jacobian leaves out the derivative of K in the
    damping term: the corrections still contract and the residual vanishes;
  * an unconstrained body in free fall reproduces the closed form.
"""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O


def _loaded_beam(beta, h=0.01, g_scale=5.0):
    mesh = fi.tet_beam(2, 2, 6)
    mu, lam = fi.lame_from_young(1e4, 0.3)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, O.NEOHOOKE, (mu, lam, 0.0),
                1000.0, h, 0.1, beta)
    p = fi.body_force(mesh, 1000.0, (0.0, 0.0, -9.81 * g_scale)).reshape(-1)
    p[m.fixed_dofs] = 0.0
    q = mesh.X.reshape(-1).copy()
    return m, q, np.zeros_like(q), p


def test_one_newton_iteration_is_the_paper_step():
    m, q, v, p = _loaded_beam(0.01)
    v = 0.05 * np.random.default_rng(0).standard_normal(q.size)
    v[m.fixed_dofs] = 0.0
    q1, v1, a1 = m.step(q, v, p)
    qn, vn, an, corr = m.newton_step(q, v, p, 1)
    assert corr == []
    np.testing.assert_array_equal(an, a1)
    np.testing.assert_array_equal(qn, q1)


def test_newton_converges_quadratically_without_stiffness_damping():
    m, q, v, p = _loaded_beam(0.0)
    _, _, a1 = m.step(q, v, p)
    qn, vn, an, corr = m.newton_step(q, v, p, 6)
    # the linearised step leaves a residual; Newton removes it
    r1 = np.linalg.norm(m.newton_residual(q, v, p, a1))
    rn = np.linalg.norm(m.newton_residual(q, v, p, an))
    assert r1 > 1e-2 * np.linalg.norm(p)
    assert rn <= 1e-12 * np.linalg.norm(p)
    # order of convergence log(e2/e1) / log(e1/e0) ~ 2 while above rounding
    big = [c for c in corr if c > 1e-9]
    assert len(big) >= 3
    for e0, e1, e2 in zip(big[:-2], big[1:-1], big[2:]):
        assert np.log(e2 / e1) / np.log(e1 / e0) >= 1.6
    # and the displacement changed materially (the nonlinearity matters here)
    assert np.linalg.norm(an - a1) > 1e-3 * np.linalg.norm(an)


def test_newton_with_stiffness_damping_contracts_to_the_solution():
    m, q, v, p = _loaded_beam(0.01)
    qn, vn, an, corr = m.newton_step(q, v, p, 12)
    rn = np.linalg.norm(m.newton_residual(q, v, p, an))
    assert rn <= 1e-9 * np.linalg.norm(p)
    assert corr[-1] <= 1e-6 * corr[0]


@pytest.mark.parametrize("iters", [2, 4])
def test_newton_free_fall_closed_form(iters):
    """Rigid translation keeps K v = 0, so every correction is zero and the
    step keeps a = (g - alpha v)/(1 + h alpha)."""
    mesh = fi.tet_beam(2, 2, 3)
    h, al = 0.01, 0.1
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, np.zeros(0, np.int64), O.NEOHOOKE,
                (3.4e3, 3.1e4, 0), 1000.0, h, al, 0.01)
    p = fi.body_force(mesh, 1000.0, (0, 0, -9.81)).reshape(-1)
    q = mesh.X.reshape(-1).copy()
    v = np.zeros_like(q)
    g = -9.81
    for t in range(1, 4):
        q, v, a, corr = m.newton_step(q, v, p, iters)
        vt = g / al * (1 - (1 + h * al) ** (-t))
        np.testing.assert_allclose(v.reshape(-1, 3)[:, 2], vt, rtol=1e-9, atol=1e-12)
        assert max(corr) <= 1e-9
