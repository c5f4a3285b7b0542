"""Pins of the oracle's discrete adjoint (reading C-12): gradients of
L = 1/2 ||q_T - q*||^2 w.r.t. per-element energy scales and the external
forces p_t, against a complex-step derivative of the whole rollout (exact to
rounding) and against central finite differences (eps = 1e-6 relative)."""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O


def _problem(kind, law, T=3):
    mesh = fi.tet_beam(2, 2, 3) if kind == "tet" else fi.hex_beam(2, 2, 3, jitter=0.1, seed=5)
    base = {fi.SVK: np.array([*fi.lame_from_young(1.0, 0.45), 0.0]),
            fi.NEOHOOKE: np.array([*fi.lame_from_young(1.0, 0.4506), 0.0]),
            fi.MOONEY_RIVLIN: np.array([0.15, 0.05, 5.0])}[law]
    E = fi.lognormal_modulus(mesh.n_elems, seed=11)
    rng = np.random.default_rng(3)
    trac = fi.end_traction(mesh, (0.0, 0.0, 40.0)).reshape(-1)
    grav = fi.body_force(mesh, 1000.0, (0, 0, -9.81)).reshape(-1)
    loads = lambda t: grav + (1.0 + 0.3 * t) * trac  # noqa: E731

    def model(Evec):
        return O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, law,
                       Evec[:, None] * base[None, :], 1000.0, 0.01, 0.1, 0.01)

    q0 = mesh.X.reshape(-1).copy()
    v0 = np.zeros_like(q0)
    q_target = q0 + 1e-3 * rng.standard_normal(q0.size)
    return mesh, model, E, loads, q0, v0, q_target, T


def _loss(model, q0, v0, loads, T, q_target):
    qs, _, _ = O.rollout_with_history(model, q0, v0, loads, T)
    d = qs[T] - q_target
    return 0.5 * (d @ d)


@pytest.mark.parametrize("kind,law", [("tet", fi.SVK), ("hex", fi.NEOHOOKE), ("tet", fi.MOONEY_RIVLIN)])
def test_adjoint_vs_complex_step(kind, law):
    mesh, model, E, loads, q0, v0, qt, T = _problem(kind, law)
    L, s_bar, p_bar = O.adjoint_rollout(model(E), q0, v0, loads, T, qt)
    dLdE = s_bar / E
    rng = np.random.default_rng(13)
    d = rng.standard_normal(E.size)
    d /= np.linalg.norm(d)
    h = 1e-30
    Lc = _loss(model(E * (1.0 + 1j * h * d)), q0, v0, loads, T, qt)
    exact = Lc.imag / h
    np.testing.assert_allclose(dLdE @ (E * d), exact, rtol=1e-9)
    np.testing.assert_allclose(Lc.real, L, rtol=1e-12)
    # external forces at every step
    dp = rng.standard_normal(p_bar.shape)
    Lp = _loss(model(E), q0, v0, lambda t: loads(t) + 1j * h * dp[t], T, qt)
    np.testing.assert_allclose((p_bar * dp).sum(), Lp.imag / h, rtol=1e-9)


def test_adjoint_vs_central_fd():
    mesh, model, E, loads, q0, v0, qt, T = _problem("hex", fi.NEOHOOKE, T=4)
    _, s_bar, _ = O.adjoint_rollout(model(E), q0, v0, loads, T, qt)
    rng = np.random.default_rng(13)
    for _ in range(3):
        d = rng.standard_normal(E.size)
        d /= np.linalg.norm(d)
        eps = 1e-6
        fd = (_loss(model(E * (1 + eps * d)), q0, v0, loads, T, qt)
              - _loss(model(E * (1 - eps * d)), q0, v0, loads, T, qt)) / (2 * eps)
        assert abs(s_bar @ d - fd) <= 1e-5 * abs(fd)
