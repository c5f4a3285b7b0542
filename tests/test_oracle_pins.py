"""Pins of the FP64 oracle against facts fixed by mathematics and the paper.

Each test targets a plausible mistake (a dropped term, a wrong sign or index,
a transposed operand) that would otherwise hide in the oracle:
  * stress/tangent = exact derivatives of the energy (complex step);
  * element force/tangent = exact derivatives of the element energy;
  * symmetry, rigid-body null modes, frame indifference;
  * the linear patch test (interior forces vanish, face forces = traction);
  * the small-strain limit = textbook linear elasticity (Voigt D from E, nu);
  * closed-form consistent mass;
  * CSR pattern and C = the library routine scipy coo->csr, and the hand
    example of tests/golden/pattern_one_tet.json (Section 4.2, Section 5.1);
  * the direct solve against a dense solve, residual <= 1e-14;
  * the whole step against closed-form free fall and against backward Euler
    of the linearised ODE (Eqs. "newton's law", "implicit integration",
    "dynamic equation1"/"dynamic equation2").
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg  # noqa: F401

import fe_inputs as fi
from oracle import fe_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LAW_PARAMS = {O.SVK: (3.4e3, 3.1e4, 0.0), O.NEOHOOKE: (3.4e3, 3.1e4, 0.0),
              O.MOONEY_RIVLIN: (1.5e3, 5e2, 5e4)}


def _rand_F(n, scale=0.2, seed=0):
    rng = np.random.default_rng(seed)
    F = np.eye(3) + scale * rng.standard_normal((n, 3, 3))
    return F[np.linalg.det(F) > 0.3]


def _cstep(fun, x, dx, h=1e-30):
    return fun(x + 1j * h * dx).imag / h


# ------------------------------------------------------------ material laws

@pytest.mark.parametrize("law", [O.SVK, O.NEOHOOKE, O.MOONEY_RIVLIN])
def test_pk1_is_energy_derivative(law):
    psi, pk1, _ = O.LAWS[law]
    p = LAW_PARAMS[law]
    F = _rand_F(20)
    P = pk1(F, *p)
    for k in range(3):
        for L in range(3):
            dF = np.zeros((3, 3))
            dF[k, L] = 1.0
            d = _cstep(lambda G: psi(G, *p), F, dF)
            np.testing.assert_allclose(P[:, k, L], d, rtol=1e-12, atol=1e-12 * np.abs(P).max())


@pytest.mark.parametrize("law", [O.SVK, O.NEOHOOKE, O.MOONEY_RIVLIN])
def test_tangent_is_pk1_derivative(law):
    _, pk1, tan = O.LAWS[law]
    p = LAW_PARAMS[law]
    F = _rand_F(20, seed=1)
    CC = tan(F, *p)
    for k in range(3):
        for L in range(3):
            dF = np.zeros((3, 3))
            dF[k, L] = 1.0
            d = _cstep(lambda G: pk1(G, *p), F, dF)
            np.testing.assert_allclose(CC[:, :, :, k, L], d, rtol=1e-12,
                                       atol=1e-12 * np.abs(CC).max())


@pytest.mark.parametrize("law", [O.SVK, O.NEOHOOKE, O.MOONEY_RIVLIN])
def test_stress_free_reference(law):
    _, pk1, _ = O.LAWS[law]
    P = pk1(np.eye(3)[None], *LAW_PARAMS[law])
    assert np.abs(P).max() < 1e-10


# ------------------------------------------------------------------- meshes

def _small_model(kind, law, jitter=0.1, deform=0.05, seed=3):
    if kind == "tet":
        mesh = fi.tet_beam(2, 2, 3)
    else:
        mesh = fi.hex_beam(2, 2, 3, jitter=jitter, seed=seed)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, law, LAW_PARAMS[law],
                1000.0, 0.01, 0.1, 0.01)
    rng = np.random.default_rng(seed)
    q = mesh.X.reshape(-1) + deform * 0.01 * rng.standard_normal(mesh.X.size)
    return mesh, m, q


CASES = [(k, law) for k in ("tet", "hex") for law in (O.SVK, O.NEOHOOKE, O.MOONEY_RIVLIN)]


@pytest.mark.parametrize("kind,law", CASES)
def test_force_is_energy_gradient(kind, law):
    mesh, m, q = _small_model(kind, law)
    f = m.internal_force(q)
    rng = np.random.default_rng(5)
    for _ in range(3):
        w = rng.standard_normal(q.size)
        d_cs = _cstep(m.energy, q, w)
        np.testing.assert_allclose(f @ w, d_cs, rtol=1e-11, atol=1e-11 * np.abs(f).sum())
        eps = 1e-6
        d_fd = (m.energy(q + eps * w) - m.energy(q - eps * w)) / (2 * eps)
        assert abs(f @ w - d_fd) <= 1e-5 * (abs(f @ w) + 1e-3 * np.abs(f).sum())


@pytest.mark.parametrize("kind,law", CASES)
def test_tangent_is_force_jacobian(kind, law):
    mesh, m, q = _small_model(kind, law)
    K = m.stiffness(q).toarray()
    rng = np.random.default_rng(6)
    for _ in range(3):
        w = rng.standard_normal(q.size)
        d_cs = _cstep(m.internal_force, q, w)
        np.testing.assert_allclose(K @ w, d_cs, rtol=1e-10, atol=1e-11 * np.abs(K).max())
        eps = 1e-6 * np.abs(q).max()
        d_fd = (m.internal_force(q + eps * w) - m.internal_force(q - eps * w)) / (2 * eps)
        assert np.linalg.norm(K @ w - d_fd) <= 1e-6 * np.linalg.norm(K @ w)


@pytest.mark.parametrize("kind,law", CASES)
def test_tangent_symmetric(kind, law):
    _, m, q = _small_model(kind, law)
    Ke = m.element_tangent(q)
    asym = np.abs(Ke - np.swapaxes(Ke, 1, 2)).max()
    assert asym <= 1e-14 * np.abs(Ke).max()


def _rigid_modes(x):
    x = x.reshape(-1, 3)
    modes = []
    for d in range(3):
        t = np.zeros_like(x)
        t[:, d] = 1.0
        modes.append(t.reshape(-1))
    for d in range(3):
        w = np.zeros(3)
        w[d] = 1.0
        modes.append(np.cross(w[None, :], x).reshape(-1))
    return modes


@pytest.mark.parametrize("kind,law", CASES)
def test_rigid_body_null_modes_at_rest(kind, law):
    mesh, m, _ = _small_model(kind, law)
    q0 = mesh.X.reshape(-1)
    K = m.stiffness(q0).toarray()
    nK = np.abs(K).max()
    for r in _rigid_modes(q0):
        assert np.linalg.norm(K @ r) <= 1e-12 * nK * np.linalg.norm(r) * math.sqrt(K.shape[0])
    # and the rest state is stress free
    assert np.abs(m.internal_force(q0)).max() <= 1e-12 * nK * 0.01


@pytest.mark.parametrize("kind,law", CASES)
def test_frame_indifference_deformed(kind, law):
    mesh, m, q = _small_model(kind, law, deform=0.1)
    K = m.stiffness(q).toarray()
    f = m.internal_force(q)
    modes = _rigid_modes(q)
    nK = np.abs(K).max()
    for t in modes[:3]:                        # translations stay null
        assert np.linalg.norm(K @ t) <= 1e-11 * nK * np.linalg.norm(t)
    for d in range(3):                         # K (w x q) = w x f
        w = np.zeros(3)
        w[d] = 1.0
        lhs = K @ modes[3 + d]
        rhs = np.cross(w[None, :], f.reshape(-1, 3)).reshape(-1)
        np.testing.assert_allclose(lhs, rhs, atol=1e-10 * nK * np.abs(q).max())
    assert np.abs(f.reshape(-1, 3).sum(axis=0)).max() <= 1e-11 * np.abs(f).max()


@pytest.mark.parametrize("kind,law", CASES)
def test_linear_patch(kind, law):
    """Affine map q = G X + c: every element has F = G; interior nodal forces
    vanish and nodes inside the x = L face carry int N_a dA * P(G) e_x."""
    # a jittered hex mesh has curved faces, whose area vector is not the
    # rest-area times e_x: the face check uses the planar grid, the interior
    # check runs on both
    for jit in ((0.0,) if kind == "tet" else (0.1, 0.0)):
        _patch_case(kind, law, jit)


def _patch_case(kind, law, jit):
    mesh = fi.tet_beam(3, 3, 4) if kind == "tet" else fi.hex_beam(3, 3, 4, jitter=jit, seed=9)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, law, LAW_PARAMS[law],
                1000.0, 0.01, 0.1, 0.01)
    G = np.array([[1.05, 0.02, -0.03], [0.01, 0.97, 0.04], [-0.02, 0.03, 1.02]])
    x = mesh.X @ G.T + np.array([0.1, -0.2, 0.3])
    F = m.quad.deformation_gradient(x)
    assert np.abs(F - G).max() < 1e-12
    f = m.internal_force(x.reshape(-1)).reshape(-1, 3)
    ijk = np.stack(np.unravel_index(np.arange(mesh.n_nodes),
                                    (mesh.nz + 1, mesh.ny + 1, mesh.nx + 1)), axis=1)[:, ::-1]
    i, j, k = ijk[:, 0], ijk[:, 1], ijk[:, 2]
    interior = (i > 0) & (i < mesh.nx) & (j > 0) & (j < mesh.ny) & (k > 0) & (k < mesh.nz)
    scale = np.abs(f).max()
    assert np.abs(f[interior]).max() <= 1e-11 * scale
    if jit > 0:
        return
    P = O.LAWS[law][1](G[None], *LAW_PARAMS[law])[0]
    face = (i == mesh.nx) & (j > 0) & (j < mesh.ny) & (k > 0) & (k < mesh.nz)
    expect = fi.end_traction(mesh, P[:, 0])
    np.testing.assert_allclose(f[face], expect[face], rtol=1e-10, atol=1e-12 * scale)


def _voigt_D(lam, mu):
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] = lam + 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    return D


def _voigt_D_young(E, nu):
    c = E / ((1 + nu) * (1 - 2 * nu))
    D = np.zeros((6, 6))
    D[:3, :3] = c * nu
    D[np.arange(3), np.arange(3)] = c * (1 - nu)
    D[np.arange(3, 6), np.arange(3, 6)] = c * (1 - 2 * nu) / 2
    return D


def _B(gradN):
    """Strain-displacement 6 x 3npe (engineering shear, order xx yy zz yz xz xy)."""
    npe = gradN.shape[0]
    B = np.zeros((6, 3 * npe))
    for a in range(npe):
        gx, gy, gz = gradN[a]
        B[0, 3 * a] = gx
        B[1, 3 * a + 1] = gy
        B[2, 3 * a + 2] = gz
        B[3, 3 * a + 1], B[3, 3 * a + 2] = gz, gy
        B[4, 3 * a], B[4, 3 * a + 2] = gz, gx
        B[5, 3 * a], B[5, 3 * a + 1] = gy, gx
    return B


@pytest.mark.parametrize("kind,law", CASES)
def test_small_strain_limit(kind, law):
    mesh, _, _ = _small_model(kind, law)
    if law == O.MOONEY_RIVLIN:
        c10, c01, kap = LAW_PARAMS[law]
        mu = 2 * (c10 + c01)
        D = _voigt_D(kap - 2 * mu / 3, mu)
        params = LAW_PARAMS[law]
    else:
        E, nu = 1e4, 0.45
        D = _voigt_D_young(E, nu)
        params = (*fi.lame_from_young(E, nu), 0.0)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, law, params,
                1000.0, 0.01, 0.1, 0.01)
    Ke = m.element_tangent(mesh.X.reshape(-1))
    for e in range(0, mesh.n_elems, max(1, mesh.n_elems // 7)):
        Kl = np.zeros_like(Ke[e])
        for qp in range(m.quad.w.shape[1]):
            B = _B(m.quad.gradN[e, qp])
            Kl += m.quad.w[e, qp] * B.T @ D @ B
        np.testing.assert_allclose(Ke[e], Kl, rtol=1e-12, atol=1e-12 * np.abs(Kl).max())


def test_tet_mass_closed_form_and_gravity_input():
    mesh = fi.tet_beam(2, 2, 3)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, O.SVK, (1, 1, 0),
                1000.0, 0.01, 0.1, 0.01)
    V = 0.01 ** 3 / 6
    np.testing.assert_allclose(m.m_e[0], 1000 * V / 20 * (np.ones((4, 4)) + np.eye(4)), rtol=1e-13)
    np.testing.assert_allclose(m.M.sum(), 3 * 1000 * 0.02 * 0.02 * 0.03, rtol=1e-13)
    g = np.tile([0.0, 0.0, -9.81], mesh.n_nodes)
    np.testing.assert_allclose(m.M @ g, fi.body_force(mesh, 1000.0, (0, 0, -9.81)).reshape(-1),
                               rtol=1e-12, atol=1e-15)


def test_hex_mass_cube_tensor_product():
    mesh = fi.hex_beam(1, 1, 1)
    m_e = O.element_mass(O.HEX8, mesh.X, mesh.conn, 1000.0)[0]
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]]) * 0.01 / 6.0      # 1D consistent mass, length s
    expect = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            expect[a, b] = 1000.0 * np.prod([m1[(a >> r) & 1, (b >> r) & 1] for r in range(3)])
    np.testing.assert_allclose(m_e, expect, rtol=1e-13)
    hx = fi.hex_beam(2, 2, 3, jitter=0.1)
    mm = O.Model(hx.elem_type, hx.X, hx.conn, hx.fixed_nodes, O.SVK, (1, 1, 0), 1000.0, .01, .1, .01)
    g = np.tile([0.0, 0.0, -9.81], hx.n_nodes)
    np.testing.assert_allclose(mm.M @ g, fi.body_force(hx, 1000.0, (0, 0, -9.81)).reshape(-1),
                               rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------- pattern and C

@pytest.mark.parametrize("kind", ["tet", "hex"])
def test_pattern_matches_library_coo_to_csr(kind):
    mesh = fi.tet_beam(2, 3, 4) if kind == "tet" else fi.hex_beam(2, 3, 4)
    n = 3 * mesh.n_nodes
    fixed = (3 * mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)
    rowptr, colind, C = O.csr_pattern(n, mesh.conn, fixed)
    row, col = O.triplet_dofs(mesh.conn)
    isfix = np.zeros(n, bool)
    isfix[fixed] = True
    keep = ~(isfix[row] | isfix[col])
    r = np.concatenate([row[keep], fixed])
    c = np.concatenate([col[keep], fixed])
    S = sp.coo_matrix((np.ones(r.size), (r, c)), shape=(n, n)).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    np.testing.assert_array_equal(rowptr, S.indptr)
    np.testing.assert_array_equal(colind, S.indices)
    # C sends each kept triplet to the slot holding its own (row, col)
    slot_row = np.repeat(np.arange(n), np.diff(rowptr))
    assert np.all(C[~keep] == -1)
    assert np.all(slot_row[C[keep]] == row[keep])
    assert np.all(colind[C[keep]] == col[keep])


def test_pattern_golden_one_tet():
    g = json.load(open(os.path.join(GOLDEN, "pattern_one_tet.json")))
    conn = np.array(g["conn"], dtype=np.int32)
    rowptr, colind, C = O.csr_pattern(12, conn, np.array(g["fixed_dofs"]))
    assert rowptr.tolist() == g["rowptr"]
    assert colind.tolist() == g["colind"]
    for t, s in g["C_samples"]:
        assert C[t] == s
    assert int((C >= 0).sum()) == g["n_mapped"]


# -------------------------------------------------------------- the solve

def test_direct_solve_dense_brute_force():
    wl = fi.workload("tet4x4x16-svk-fp64")
    m = O.Model.from_workload(wl)
    q = wl.mesh.X.reshape(-1).copy()
    v = np.zeros_like(q)
    A, b = m.system(q, v, wl.p(0).reshape(-1))
    a = O.direct_solve(A, b)
    # normwise backward error at FP64 rounding level
    bwd = np.linalg.norm(A @ a - b) / (sp.linalg.norm(A) * np.linalg.norm(a) + np.linalg.norm(b))
    assert bwd <= 1e-15
    a2 = np.linalg.solve(A.toarray(), b)
    np.testing.assert_allclose(a, a2, rtol=1e-10, atol=1e-13 * np.abs(a2).max())
    import scipy.sparse.linalg as spla
    a3 = spla.splu(A.tocsc()).solve(b)
    np.testing.assert_allclose(a, a3, rtol=1e-10, atol=1e-13 * np.abs(a2).max())
    # the constrained DOFs stay at rest
    assert np.all(a[m.fixed_dofs] == 0.0)


@pytest.mark.parametrize("kind", ["tet", "hex"])
def test_free_fall_closed_form(kind):
    """Unconstrained body at rest under uniform gravity: stays stress free and
    a = (g - alpha v)/(1 + h alpha) exactly, so v_t = g/alpha (1 - (1+h alpha)^-t)."""
    mesh = fi.tet_beam(2, 2, 3) if kind == "tet" else fi.hex_beam(2, 2, 3, jitter=0.1)
    h, al = 0.01, 0.1
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, np.zeros(0, np.int64), O.NEOHOOKE,
                (3.4e3, 3.1e4, 0), 1000.0, h, al, 0.01)
    p = fi.body_force(mesh, 1000.0, (0, 0, -9.81)).reshape(-1)
    q = mesh.X.reshape(-1).copy()
    v = np.zeros_like(q)
    T = 6
    qs, vs = O.rollout(m, q, v, lambda t: p, T)
    g = -9.81
    for t in range(T + 1):
        vt = g / al * (1 - (1 + h * al) ** (-t))
        np.testing.assert_allclose(vs[t].reshape(-1, 3)[:, 2], vt, rtol=1e-9, atol=1e-12)
        assert np.abs(vs[t].reshape(-1, 3)[:, :2]).max() < 1e-12
        dz = sum(h * (g / al * (1 - (1 + h * al) ** (-s))) for s in range(1, t + 1))
        np.testing.assert_allclose(qs[t].reshape(-1, 3)[:, 2] - mesh.X[:, 2], dz,
                                   rtol=1e-9, atol=1e-13)


def test_step_is_backward_euler_of_linearised_ode():
    """Tiny displacements: one step equals backward Euler of
    M a + (alpha M + beta K0) v + K0 (q - X) = p with the textbook K0."""
    mesh = fi.tet_beam(2, 2, 4)
    E, nu, h, al, be = 1e4, 0.45, 0.01, 0.1, 0.01
    mu, lam = fi.lame_from_young(E, nu)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, O.SVK, (mu, lam, 0),
                1000.0, h, al, be)
    n = 3 * mesh.n_nodes
    K0 = np.zeros((n, n))
    D = _voigt_D_young(E, nu)
    for e in range(mesh.n_elems):
        B = _B(m.quad.gradN[e, 0])
        dofs = (3 * mesh.conn[e][:, None] + np.arange(3)).reshape(-1)
        K0[np.ix_(dofs, dofs)] += m.quad.w[e, 0] * B.T @ D @ B
    M = m.M.toarray()
    rng = np.random.default_rng(2)
    U, V, Pp = (rng.standard_normal(n) for _ in range(3))
    free = np.setdiff1d(np.arange(n), m.fixed_dofs)
    errs = []
    for eps in (1e-8, 1e-9):
        u0, v0, p = eps * U, eps * V, eps * 1e-3 * Pp
        u0[m.fixed_dofs] = 0
        v0[m.fixed_dofs] = 0
        q0 = mesh.X.reshape(-1) + u0
        q1, v1, a1 = m.step(q0, v0, p)
        Aff = (M + h * (al * M + be * K0) + h * h * K0)[np.ix_(free, free)]
        rhs = (p - K0 @ u0 - (al * M + be * K0) @ v0 - h * K0 @ v0)[free]
        a_lin = np.zeros(n)
        a_lin[free] = np.linalg.solve(Aff, rhs)
        errs.append(np.linalg.norm(a1 - a_lin) / np.linalg.norm(a_lin))
    # the gap is the O(eps) geometric/material nonlinearity: it must shrink
    # linearly with the amplitude (a wrong sign or factor would leave O(1))
    assert errs[1] <= 2e-5
    assert 5.0 < errs[0] / errs[1] < 20.0
    np.testing.assert_allclose(v1, v0 + h * a1, rtol=0, atol=1e-20)
    np.testing.assert_allclose(q1, q0 + h * v1, rtol=0, atol=1e-18)


def test_equilibrium_is_stationary():
    """p = f(q), v = 0: b = 0 so the step leaves the state unchanged (sign of f vs p)."""
    mesh, m, q = _small_model("hex", O.NEOHOOKE, deform=0.1)
    q = q.copy()
    q[m.fixed_dofs] = mesh.X.reshape(-1)[m.fixed_dofs]
    p = m.internal_force(q)
    q1, v1, a1 = m.step(q, np.zeros_like(q), p)
    assert np.abs(a1).max() < 1e-9 * np.abs(p).max() / m.M.diagonal().max()


def test_cg_solve_reaches_the_direct_solution():
    """The Jacobi CG of the oracle (cg_solve) against the dense solve on an
    SPD system of a small beam: the returned residual meets the tolerance
    and the solution agrees with numpy's dense solve within the tolerance
    times the condition number's reach."""
    wl = fi.workload("tet-mr", a=2, b=2, c=6)
    m = O.Model.from_workload(wl)
    q = wl.mesh.X.reshape(-1).copy()
    A, b = m.system(q, np.zeros_like(q), wl.p(0).reshape(-1))
    x, its = O.cg_solve(A.tocsr(), b, 1e-13)
    assert its > 1
    assert np.linalg.norm(b - A @ x) <= 1e-13 * np.linalg.norm(b)
    xd = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    x0, its0 = O.cg_solve(A.tocsr(), np.zeros_like(b), 1e-13)
    assert its0 == 0 and not x0.any()


def test_cg_step_matches_direct_step():
    """step_cg at tol 1e-13 and step (direct solve) give the same positions
    after three steps of the loaded Mooney-Rivlin beam, to 1e-10 of the
    displacement."""
    wl = fi.workload("tet-mr", a=2, b=2, c=6)
    m = O.Model.from_workload(wl)
    q = q2 = wl.mesh.X.reshape(-1).copy()
    v = v2 = np.zeros_like(q)
    for t in range(3):
        p = wl.p(t).reshape(-1)
        q, v, _ = m.step(q, v, p)
        q2, v2, _, _ = m.step_cg(q2, v2, p, 1e-13)
    X = wl.mesh.X.reshape(-1)
    assert np.linalg.norm(q2 - q) <= 1e-10 * np.linalg.norm(q - X)
