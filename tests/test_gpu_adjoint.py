"""GPU discrete adjoint (fe_adjoint, S10) against the oracle adjoint and
against central finite differences of the GPU rollout (reading C-13:
eps = 1e-6 relative, solves at tol 1e-13, so FD noise stays < 1e-5).
Tolerances: FP64 gradients <= 1e-8 relative to the oracle's (norm); mixed
path <= 1e-5 (FP32 tangent and dual-number pass; measured 1.6e-6)."""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O

pytestmark = pytest.mark.gpu


def _problem(kind, law, T=3):
    mesh = fi.tet_beam(2, 2, 5) if kind == "tet" else fi.hex_beam(2, 2, 5, jitter=0.1, seed=5)
    base = {fi.SVK: np.array([*fi.lame_from_young(1.0, 0.45), 0.0]),
            fi.NEOHOOKE: np.array([*fi.lame_from_young(1.0, 0.4506), 0.0]),
            fi.MOONEY_RIVLIN: np.array([0.15, 0.05, 5.0])}[law]
    E = fi.lognormal_modulus(mesh.n_elems, seed=11)
    trac = fi.end_traction(mesh, (0.0, 0.0, 40.0)).reshape(-1)
    grav = fi.body_force(mesh, 1000.0, (0, 0, -9.81)).reshape(-1)
    loads = np.stack([grav + (1.0 + 0.3 * t) * trac for t in range(T)])
    q0 = mesh.X.reshape(-1).copy()
    rng = np.random.default_rng(12)
    q_target = q0 + 1e-3 * rng.standard_normal(q0.size)
    return mesh, base, E, loads, q0, q_target


def _gpu_ctx(fe, mesh, law, base, E, precision=0, R=1, tol=1e-13):
    return fe.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, law, 1000.0,
                        E[:, None] * base[None, :], 0.01, 0.1, 0.01, precision=precision,
                        refactor_every=R, tol=tol, keep_checkpoints=1)


def _gpu_loss_and_grad(ctx, loads, q_target, grad=True):
    q = np.empty(ctx.n)
    v = np.empty(ctx.n)
    ctx.set_state(ctx_q0(ctx), np.zeros(ctx.n))
    ctx.clear_checkpoints()
    for t in range(loads.shape[0]):
        ctx.step(loads[t], q, v)
    d = q - q_target
    L = 0.5 * d @ d
    if not grad:
        return L, None, None
    ds, dp = ctx.adjoint(d)
    return L, ds, dp


def ctx_q0(ctx):
    return ctx._q0


@pytest.mark.parametrize("kind,law,R", [("tet", fi.SVK, 1), ("hex", fi.NEOHOOKE, 2),
                                        ("tet", fi.MOONEY_RIVLIN, 2)])
def test_adjoint_matches_oracle(gpu_lib, kind, law, R):
    mesh, base, E, loads, q0, qt = _problem(kind, law)
    ctx = _gpu_ctx(gpu_lib, mesh, law, base, E, R=R)
    ctx._q0 = q0
    L, ds, dp = _gpu_loss_and_grad(ctx, loads, qt)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, law, E[:, None] * base[None, :],
                1000.0, 0.01, 0.1, 0.01)
    Lo, so, po = O.adjoint_rollout(m, q0, np.zeros_like(q0), lambda t: loads[t], loads.shape[0], qt)
    assert abs(L - Lo) <= 1e-10 * abs(Lo)
    assert np.linalg.norm(ds - so) <= 1e-8 * np.linalg.norm(so)
    assert np.linalg.norm(dp - po) <= 1e-8 * np.linalg.norm(po)
    ctx.close()


def test_adjoint_vs_central_fd_on_gpu(gpu_lib):
    mesh, base, E, loads, q0, qt = _problem("hex", fi.NEOHOOKE, T=4)
    ctx = _gpu_ctx(gpu_lib, mesh, fi.NEOHOOKE, base, E, R=1)
    ctx._q0 = q0
    _, ds, _ = _gpu_loss_and_grad(ctx, loads, qt)
    rng = np.random.default_rng(13)
    for _ in range(4):
        d = rng.standard_normal(E.size)
        d /= np.linalg.norm(d)
        eps = 1e-6
        Ls = []
        for sgn in (1.0, -1.0):
            ctx.set_params((E * (1 + sgn * eps * d))[:, None] * base[None, :])
            Ls.append(_gpu_loss_and_grad(ctx, loads, qt, grad=False)[0])
        fd = (Ls[0] - Ls[1]) / (2 * eps)
        assert abs(ds @ d - fd) <= 1e-5 * abs(fd)
        ctx.set_params(E[:, None] * base[None, :])
    ctx.close()


def test_adjoint_mixed_precision(gpu_lib):
    mesh, base, E, loads, q0, qt = _problem("hex", fi.NEOHOOKE)
    ctx = _gpu_ctx(gpu_lib, mesh, fi.NEOHOOKE, base, E, precision=1, R=2, tol=1e-10)
    ctx._q0 = q0
    _, ds, dp = _gpu_loss_and_grad(ctx, loads, qt)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.NEOHOOKE,
                E[:, None] * base[None, :], 1000.0, 0.01, 0.1, 0.01)
    _, so, po = O.adjoint_rollout(m, q0, np.zeros_like(q0), lambda t: loads[t], loads.shape[0], qt)
    es, ep = np.linalg.norm(ds - so) / np.linalg.norm(so), np.linalg.norm(dp - po) / np.linalg.norm(po)
    print(f"mixed adjoint: dL/ds error {es:.2e}, dL/dp error {ep:.2e}")
    assert es <= 1e-5 and ep <= 1e-5
    ctx.close()


def test_autograd_function(gpu_lib):
    import torch
    from paper_2306_05893_gb300.autograd import rollout
    mesh, base, E, loads, q0, qt = _problem("tet", fi.SVK)
    ctx = _gpu_ctx(gpu_lib, mesh, fi.SVK, base, E, R=1)
    scale = torch.tensor(E, dtype=torch.float64, requires_grad=True)
    P = torch.tensor(loads, dtype=torch.float64, requires_grad=True)
    qT, vT = rollout(scale, P, ctx, base, q0, np.zeros_like(q0))
    loss = 0.5 * ((qT - torch.tensor(qt)) ** 2).sum()
    loss.backward()
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.SVK, E[:, None] * base[None, :],
                1000.0, 0.01, 0.1, 0.01)
    _, so, po = O.adjoint_rollout(m, q0, np.zeros_like(q0), lambda t: loads[t], loads.shape[0], qt)
    assert np.linalg.norm(scale.grad.numpy() - so) <= 1e-8 * np.linalg.norm(so)
    assert np.linalg.norm(P.grad.numpy() - po) <= 1e-8 * np.linalg.norm(po)
    ctx.close()


# ------------------------------------------ the adjoint workload (reading C-10)

def _modulus_beam(a, b, c, T):
    """The adjoint workload's beam: trilinear hexes jittered by +-10% of the
    spacing (seed 1), neo-Hookean with nu = lambda / (2 (lambda + mu)) of
    (3.4e3, 3.1e4) Pa, per-element Young's modulus log-normal (median 1e4,
    sigma 0.3, seed 11), the free end pulled by 50 Pa for T steps; the target
    positions come from the seed-12 modulus field."""
    mesh = fi.hex_beam(a, b, c, jitter=0.1, seed=1)
    nu = 3.1e4 / (2 * (3.1e4 + 3.4e3))
    base = np.array([*fi.lame_from_young(1.0, nu), 0.0])
    E = fi.lognormal_modulus(mesh.n_elems, seed=11)
    Et = fi.lognormal_modulus(mesh.n_elems, seed=12)
    trac = fi.end_traction(mesh, (50.0, 0.0, 0.0)).reshape(-1)
    return mesh, base, E, Et, np.tile(trac, (T, 1))


def _fd_check(gpu_lib, mesh, base, E, Et, loads, n_dirs, seed=13, eps=1e-6):
    """Adjoint dL/ds . d against central differences of the GPU rollout,
    L(E (1 + eps d)), d ~ N(0, I) normalised (reading C-13: FP64, exact
    factor every step, solves to 1e-13)."""
    q0 = mesh.X.reshape(-1).copy()
    ctx = _gpu_ctx(gpu_lib, mesh, fi.NEOHOOKE, base, Et, R=1)
    ctx._q0 = q0
    qt = np.empty(ctx.n)
    ctx.set_state(q0, np.zeros_like(q0))
    for t in range(loads.shape[0]):
        ctx.step(loads[t], qt, None)
    ctx.set_params(E[:, None] * base[None, :])
    _, ds, _ = _gpu_loss_and_grad(ctx, loads, qt)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(n_dirs):
        d = rng.standard_normal(E.size)
        d /= np.linalg.norm(d)
        Ls = []
        for sgn in (1.0, -1.0):
            ctx.set_params((E * (1 + sgn * eps * d))[:, None] * base[None, :])
            Ls.append(_gpu_loss_and_grad(ctx, loads, qt, grad=False)[0])
        fd = (Ls[0] - Ls[1]) / (2 * eps)
        rel = abs(ds @ d - fd) / abs(fd)
        worst = max(worst, rel)
        assert rel <= 1e-5, (rel, ds @ d, fd)
    ctx.close()
    return ds, qt, worst


def test_adjoint_workload_small_beam_16_directions(gpu_lib):
    """The 4 x 4 x 16 hex beam (1,275 DOF) over T = 20 steps: 16 central
    difference directions, and the oracle's adjoint of the same loss."""
    mesh, base, E, Et, loads = _modulus_beam(4, 4, 16, 20)
    ds, qt, worst = _fd_check(gpu_lib, mesh, base, E, Et, loads, 16)
    q0 = mesh.X.reshape(-1).copy()
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.NEOHOOKE,
                E[:, None] * base[None, :], 1000.0, 0.01, 0.1, 0.01)
    _, so, _ = O.adjoint_rollout(m, q0, np.zeros_like(q0), lambda t: loads[t], loads.shape[0], qt)
    assert np.linalg.norm(ds - so) <= 1e-8 * np.linalg.norm(so)
    print(f"16 directions: worst |adjoint - FD| / |FD| = {worst:.2e}")


def test_adjoint_workload_full_beam_2_directions(gpu_lib):
    """The 20 x 20 x 80 hex beam (107,163 DOF, the adjoint workload's own
    mesh) over T = 20 steps: 2 central-difference directions.  A normalised
    direction spreads over 32,000 elements (about 6e-3 each), so eps = 1e-6
    would move the positions by ~1e-11 m, where the rounding of coordinates
    of ~1 m (1e-16 m) already leaves ~1e-4 of FD noise; eps = 1e-4 keeps the
    perturbation per element below 1e-6 and the truncation error O(eps^2)."""
    mesh, base, E, Et, loads = _modulus_beam(20, 20, 80, 20)
    _, _, worst = _fd_check(gpu_lib, mesh, base, E, Et, loads, 2, eps=1e-4)
    print(f"107k DOF, 2 directions: worst |adjoint - FD| / |FD| = {worst:.2e}")
