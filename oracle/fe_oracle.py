"""FP64 CPU oracle of the implicit FE time step (TEST INFRASTRUCTURE ONLY).

Only tests, the package's smoke check and the benchmark's CPU-baseline leg may
import this module.  The product path (the CUDA library and its binding) never
calls it, and it shares no code with that path: the only common input is the
seeded workload generator ``fe_inputs``.

What it computes, in the paper's order (arXiv 2306.05893, Section 3):
  * element internal force f_e = dW_e/dx and exact tangent K_e = df_e/dx for
    P1 tets (one point) and trilinear hexes (2x2x2 Gauss), for St Venant-
    Kirchhoff, compressible neo-Hookean and decoupled Mooney-Rivlin energies
    written with the invariants I1 = tr C, I2 = ((tr C)^2 - tr C^2)/2 and
    J = det F of Section 3.1;
  * consistent mass M;
  * triplet assembly by plain summation, then the projective constraints of
    Section 5.1 (fixed rows and columns cleared, 1 on the diagonal);
  * A = (1 + h alpha) M + h (beta + h) K (Eq. "dynamic equation2") and
    b = p - f - (alpha M + (beta + h) K) v (Eq. "dynamic equation1" with the
    Rayleigh damping B = alpha M + beta K);
  * a direct sparse solve of A a = b, then backward Euler
    v+ = v + h a, q+ = q + h v+ (Eq. "implicit integration"); for meshes
    whose direct factor is too large for the host, the same step with a
    Jacobi-preconditioned CG solve to a stated residual (cg_solve);
  * the CSR pattern and the triplet -> slot map C (Section 4.2), built here by
    sorting unique (row, col) keys, i.e. independently of the double transpose;
  * frictionless contact against rigid planes by Lagrange multipliers
    (Section "Lagrangian multipliers"): free motion, compliance
    W = H A^{-1} H^T by one direct solve per constraint, projected
    Gauss-Seidel, motion correction.

Everything is numpy float64 (complex128 where a complex-step derivative is
taken), vectorised over elements only: no blocking, fusion or reordering.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

SVK, NEOHOOKE, MOONEY_RIVLIN, COROTATIONAL = 0, 1, 2, 3
TET4, HEX8 = 0, 1

_I3 = np.eye(3)


# ============================================================ material laws
# Each law gives the energy density psi(F), the first Piola-Kirchhoff stress
# P = dpsi/dF and the tangent CC[i,J,k,L] = dP_iJ / dF_kL.  Arrays broadcast
# over leading axes; p0, p1, p2 are the law's three parameters:
#   SVK, neo-Hookean: (mu, lambda, unused); Mooney-Rivlin: (C10, C01, kappa).

def _ex(p, F):
    return np.asarray(p)[..., None, None]


def _ex4(p):
    return np.asarray(p)[..., None, None, None, None]


def _tr(A):
    return np.einsum("...ii->...", A)


def svk_psi(F, mu, lam, _=None):
    """Saint Venant-Kirchhoff energy density mu tr(E^2) + lambda/2 (tr E)^2 (Section 3.1 names the
    law; textbook form)."""
    E = 0.5 * (np.swapaxes(F, -1, -2) @ F - _I3)
    trE = _tr(E)
    return mu * _tr(E @ E) + 0.5 * lam * trE * trE


def svk_pk1(F, mu, lam, _=None):
    """P = F S with S = 2 mu E + lambda tr(E) I: the derivative of svk_psi (Section 3.1)."""
    E = 0.5 * (np.swapaxes(F, -1, -2) @ F - _I3)
    S = 2.0 * _ex(mu, F) * E + _ex(lam, F) * _tr(E)[..., None, None] * _I3
    return F @ S


def svk_tangent(F, mu, lam, _=None):
    """CC = dP/dF of the Saint Venant-Kirchhoff law, exact, no projection (Section 3.1)."""
    E = 0.5 * (np.swapaxes(F, -1, -2) @ F - _I3)
    S = 2.0 * _ex(mu, F) * E + _ex(lam, F) * _tr(E)[..., None, None] * _I3
    B = F @ np.swapaxes(F, -1, -2)
    CC = np.einsum("ik,...LJ->...iJkL", _I3, S)
    CC = CC + _ex4(mu) * (np.einsum("...iL,...kJ->...iJkL", F, F)
                          + np.einsum("...ik,JL->...iJkL", B, _I3))
    CC = CC + _ex4(lam) * np.einsum("...iJ,...kL->...iJkL", F, F)
    return CC


def nh_psi(F, mu, lam, _=None):
    """Compressible neo-Hookean energy mu/2 (I1 - 3) - mu ln J + lambda/2 (ln J)^2 with the
    invariants of Section 3.1 (Bonet-Wood form)."""
    J = np.linalg.det(F)
    lnJ = np.log(J)
    I1 = _tr(np.swapaxes(F, -1, -2) @ F)
    return 0.5 * mu * (I1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ


def nh_pk1(F, mu, lam, _=None):
    """P = mu (F - F^-T) + lambda ln J F^-T: the derivative of nh_psi (Section 3.1)."""
    G = np.swapaxes(np.linalg.inv(F), -1, -2)
    lnJ = np.log(np.linalg.det(F))
    return _ex(mu, F) * (F - G) + (_ex(lam, F) * lnJ[..., None, None]) * G


def nh_tangent(F, mu, lam, _=None):
    """CC = dP/dF of the neo-Hookean law, exact, no projection (Section 3.1)."""
    G = np.swapaxes(np.linalg.inv(F), -1, -2)
    lnJ = np.log(np.linalg.det(F))
    CC = _ex4(mu) * np.einsum("ik,JL->iJkL", _I3, _I3)
    CC = CC + (_ex4(mu) - _ex4(lam) * lnJ[..., None, None, None, None]) * np.einsum(
        "...iL,...kJ->...iJkL", G, G)
    CC = CC + _ex4(lam) * np.einsum("...iJ,...kL->...iJkL", G, G)
    return CC


def _mr_parts(F):
    C = np.swapaxes(F, -1, -2) @ F
    I1 = _tr(C)
    I2 = 0.5 * (I1 * I1 - _tr(C @ C))
    J = np.linalg.det(F)
    G = np.swapaxes(np.linalg.inv(F), -1, -2)
    return C, I1, I2, J, G


def mr_psi(F, c10, c01, kappa):
    """Decoupled Mooney-Rivlin energy C10 (J^-2/3 I1 - 3) + C01 (J^-4/3 I2 - 3) + kappa/2 (J - 1)^2
    with the invariants I1, I2, J of Section 3.1."""
    _, I1, I2, J, _ = _mr_parts(F)
    return (c10 * (J ** (-2.0 / 3.0) * I1 - 3.0) + c01 * (J ** (-4.0 / 3.0) * I2 - 3.0)
            + 0.5 * kappa * (J - 1.0) ** 2)


def mr_pk1(F, c10, c01, kappa):
    """P = dpsi/dF of the decoupled Mooney-Rivlin law (Section 3.1), term by term."""
    C, I1, I2, J, G = _mr_parts(F)
    x = lambda s: s[..., None, None]  # noqa: E731
    J23, J43 = J ** (-2.0 / 3.0), J ** (-4.0 / 3.0)
    H = x(I1) * F - F @ C
    P = _ex(c10, F) * x(J23) * (2.0 * F - (2.0 / 3.0) * x(I1) * G)
    P = P + _ex(c01, F) * x(J43) * (2.0 * H - (4.0 / 3.0) * x(I2) * G)
    P = P + _ex(kappa, F) * x((J - 1.0) * J) * G
    return P


def mr_tangent(F, c10, c01, kappa):
    """CC = dP/dF of the decoupled Mooney-Rivlin law, exact, no projection (Section 3.1)."""
    C, I1, I2, J, G = _mr_parts(F)
    B = F @ np.swapaxes(F, -1, -2)
    x2 = lambda s: s[..., None, None]  # noqa: E731
    x4 = lambda s: s[..., None, None, None, None]  # noqa: E731
    J23, J43 = J ** (-2.0 / 3.0), J ** (-4.0 / 3.0)
    H = x2(I1) * F - F @ C
    dd = np.einsum("ik,JL->iJkL", _I3, _I3)
    o = lambda a, b: np.einsum("...iJ,...kL->...iJkL", a, b)  # noqa: E731  a_iJ b_kL
    x_ = lambda a, b: np.einsum("...iL,...kJ->...iJkL", a, b)  # noqa: E731  a_iL b_kJ
    t1 = (-(2.0 / 3.0) * o(2.0 * F - (2.0 / 3.0) * x2(I1) * G, G) + 2.0 * dd
          - (4.0 / 3.0) * o(G, F) + (2.0 / 3.0) * x4(I1) * x_(G, G))
    d_fc = (np.einsum("ik,...LJ->...iJkL", _I3, C) + x_(F, F)
            + np.einsum("...ik,JL->...iJkL", B, _I3))
    t2 = (-(4.0 / 3.0) * o(2.0 * H - (4.0 / 3.0) * x2(I2) * G, G)
          + 2.0 * (2.0 * o(F, F) + x4(I1) * dd - d_fc)
          - (8.0 / 3.0) * o(G, H) + (4.0 / 3.0) * x4(I2) * x_(G, G))
    t3 = x4((2.0 * J - 1.0) * J) * o(G, G) - x4(J * J - J) * x_(G, G)
    return _ex4(c10) * x4(J23) * t1 + _ex4(c01) * x4(J43) * t2 + _ex4(kappa) * t3


LAWS = {
    SVK: (svk_psi, svk_pk1, svk_tangent),
    NEOHOOKE: (nh_psi, nh_pk1, nh_tangent),
    MOONEY_RIVLIN: (mr_psi, mr_pk1, mr_tangent),
}


# ======================================================== element geometry

def _hex_corners():
    return np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1]
                     for a in range(8)], dtype=np.float64)


def hex_shape(xi):
    """Trilinear shape functions N[8] and derivatives dN[8, 3] at xi on [-1,1]^3,
    local node a at corner (2dx-1, 2dy-1, 2dz-1) with a = dx + 2dy + 4dz.
    Section 3.1: trilinear hexahedra.
    """
    c = _hex_corners()
    f = 1.0 + c * np.asarray(xi)[None, :]
    N = np.prod(f, axis=1) / 8.0
    dN = np.empty((8, 3))
    for r in range(3):
        o = [s for s in range(3) if s != r]
        dN[:, r] = c[:, r] * f[:, o[0]] * f[:, o[1]] / 8.0
    return N, dN


def hex_gauss_points():
    """2x2x2 Gauss points +-1/sqrt(3) (weight 1) in the local corner order.  Section 3.1: hexahedra
    integrated by 2x2x2 Gauss."""
    return _hex_corners() / math.sqrt(3.0)


class Quadrature:
    """Rest-state data: gradN [E, Q, npe, 3] (w.r.t. rest coordinates X) and
    weights w [E, Q] (volume for a tet; detJ0 for a hex Gauss point).
    Section 3.1: element kernels on P1 tets and trilinear hexes.
    """

    def __init__(self, elem_type, X, conn):
        self.elem_type = elem_type
        self.conn = np.asarray(conn)
        Xe = np.asarray(X)[self.conn]                       # [E, npe, 3]
        self.Xe = Xe
        if elem_type == TET4:
            Dm = np.swapaxes(Xe[:, 1:] - Xe[:, [0]], 1, 2)  # columns X_a - X_0
            Gm = np.linalg.inv(Dm)                           # row a-1 = grad N_a
            g = np.concatenate([-Gm.sum(axis=1, keepdims=True), Gm], axis=1)
            self.gradN = g[:, None]                          # [E, 1, 4, 3]
            self.w = (np.linalg.det(Dm) / 6.0)[:, None]
        else:
            gps = hex_gauss_points()
            grads, ws = [], []
            for q in range(8):
                _, dN = hex_shape(gps[q])
                J0 = np.einsum("eai,ar->eir", Xe, dN)         # dX_i / dxi_r
                J0inv = np.linalg.inv(J0)
                grads.append(np.einsum("ar,erJ->eaJ", dN, J0inv))
                ws.append(np.linalg.det(J0))
            self.gradN = np.stack(grads, axis=1)             # [E, 8, 8, 3]
            self.w = np.stack(ws, axis=1)                    # [E, 8]

    @property
    def npe(self):
        """Nodes per element (4 for P1 tets, 8 for trilinear hexes; Section 3.1)."""
        return self.conn.shape[1]

    def deformation_gradient(self, x):
        """F[e, q] = sum_a x_a (outer) gradN_a.  Section 3.1."""
        xe = np.asarray(x)[self.conn]                        # [E, npe, 3]
        return np.einsum("eai,eqaJ->eqiJ", xe, self.gradN)


def _params(params, E):
    p = np.asarray(params)
    p = p.astype(np.result_type(p.dtype, np.float64))  # complex parameters stay complex
    if p.ndim == 1:
        p = np.broadcast_to(p, (E, 3))
    return p[:, 0][:, None], p[:, 1][:, None], p[:, 2][:, None]   # [E, 1] each


# ============================================ co-rotational linear elements
# Section 3.1, Eq. "eqmodel": the rest stiffness K0_e = int B^T D B dV (B the
# strain-displacement matrix, D the isotropic stress-strain matrix from
# (mu, lambda)), rotated per element: with R_e the rotation of the polar
# decomposition of the element's deformation gradient (for a hex, of its
# volume average over the Gauss points),
#   f_e = Rb K0_e (Rb^T x_e - X_e),   K_e = Rb K0_e Rb^T,   Rb = diag(R_e, ..).
# The tangent leaves out the derivative of R_e (the usual co-rotational
# stiffness), so there is no element energy.

def voigt_B(gradN):
    """[..., npe, 3] -> [..., 6, 3 npe]; strain order xx, yy, zz, xy, yz, zx
    with engineering shears.
    Eq. "eqmodel": the linear-elastic K_0 of the co-rotational model.
    """
    npe = gradN.shape[-2]
    B = np.zeros(gradN.shape[:-2] + (6, 3 * npe))
    for a in range(npe):
        gx, gy, gz = gradN[..., a, 0], gradN[..., a, 1], gradN[..., a, 2]
        c = 3 * a
        B[..., 0, c] = gx
        B[..., 1, c + 1] = gy
        B[..., 2, c + 2] = gz
        B[..., 3, c], B[..., 3, c + 1] = gy, gx
        B[..., 4, c + 1], B[..., 4, c + 2] = gz, gy
        B[..., 5, c], B[..., 5, c + 2] = gz, gx
    return B


def voigt_D(mu, lam):
    """[E, 1] parameters -> [E, 6, 6] isotropic stress-strain matrix.  Eq. "eqmodel" (isotropic
    linear elasticity)."""
    mu, lam = np.asarray(mu).reshape(-1), np.asarray(lam).reshape(-1)
    D = np.zeros((mu.shape[0], 6, 6), dtype=np.result_type(mu, lam))
    D[:, :3, :3] = lam[:, None, None]
    for k in range(3):
        D[:, k, k] += 2.0 * mu
        D[:, 3 + k, 3 + k] = mu
    return D


def corot_rotation(quad, x):
    """R_e [E, 3, 3] = the rotation of the polar decomposition F = R S of the
    element's (volume-averaged) deformation gradient, by SVD.
    Eq. "eqmodel": the element rotation of the co-rotational model.
    """
    F = quad.deformation_gradient(x)
    Fb = np.einsum("eq,eqiJ->eiJ", quad.w, F) / quad.w.sum(axis=1)[:, None, None]
    U, _, Vt = np.linalg.svd(Fb)
    d = np.sign(np.linalg.det(U @ Vt))
    U = U.copy()
    U[:, :, 2] *= d[:, None]  # a proper rotation (det = +1)
    return U @ Vt


def corot_K0(quad, params):
    """Rest stiffness K0_e = sum_q w_q B^T D B of linear elasticity, the K_0 of the co-rotational
    model (Eq. "eqmodel")."""
    mu, lam, _ = _params(params, quad.conn.shape[0])
    B = voigt_B(quad.gradN)                                   # [E, Q, 6, 3npe]
    D = voigt_D(mu, lam)
    return np.einsum("eq,eqsm,est,eqtn->emn", quad.w, B, D, B, optimize=True)


def _block_rotation(R, npe):
    E = R.shape[0]
    Rb = np.zeros((E, 3 * npe, 3 * npe), dtype=R.dtype)
    for a in range(npe):
        Rb[:, 3 * a:3 * a + 3, 3 * a:3 * a + 3] = R
    return Rb


def corot_force(quad, x, params):
    """f_e = R (K0 (R^T x - X)) of the co-rotational model (Eq. "eqmodel"), R from corot_rotation."""
    R = corot_rotation(quad, x)
    Rb = _block_rotation(R, quad.npe)
    xe = np.asarray(x)[quad.conn].reshape(R.shape[0], -1)
    u_loc = np.einsum("emn,em->en", Rb, xe) - quad.Xe.reshape(R.shape[0], -1)   # Rb^T x - X
    return np.einsum("emn,enk,ek->em", Rb, corot_K0(quad, params), u_loc)


def corot_tangent(quad, x, params):
    """K_e = R K0 R^T: the co-rotational tangent with the rotation held fixed (Eq. "eqmodel")."""
    Rb = _block_rotation(corot_rotation(quad, x), quad.npe)
    return np.einsum("emn,enk,elk->eml", Rb, corot_K0(quad, params), Rb)


def element_energy(quad, x, model, params):
    """W_e = sum_q w_q psi(F_q)  -> [E].  Section 3.1: the elastic energy whose gradient is the
    internal force."""
    psi = LAWS[model][0]
    F = quad.deformation_gradient(x)
    a, b, c = _params(params, F.shape[0])
    return np.einsum("eq,eq->e", quad.w, psi(F, a, b, c))


def element_force(quad, x, model, params):
    """f_e[3a+i] = sum_q w_q sum_J P_iJ gradN_aJ  (internal force dW_e/dx).  Section 3.1; Eq.
    "newton's law" uses f."""
    if model == COROTATIONAL:
        return corot_force(quad, x, params)
    P = LAWS[model][1](quad.deformation_gradient(x), *_params(params, quad.conn.shape[0]))
    f = np.einsum("eq,eqiJ,eqaJ->eai", quad.w, P, quad.gradN)
    return f.reshape(f.shape[0], -1)


def element_tangent(quad, x, model, params):
    """K_e[3a+i, 3b+k] = sum_q w_q sum_JL CC_iJkL gradN_aJ gradN_bL.  Section 3.1: K = df/dq, the K
    of Eq. "dynamic equation2"."""
    if model == COROTATIONAL:
        return corot_tangent(quad, x, params)
    CC = LAWS[model][2](quad.deformation_gradient(x), *_params(params, quad.conn.shape[0]))
    K = np.einsum("eq,eqiJkL,eqaJ,eqbL->eaibk", quad.w, CC, quad.gradN, quad.gradN,
                  optimize=True)
    E, n = K.shape[0], K.shape[1] * 3
    return K.reshape(E, n, n)


def element_mass(elem_type, X, conn, rho):
    """Consistent mass scalars m_e[a, b] = rho int N_a N_b dV (times I3 per block).  Section 4.1:
    per-element mass, assembled like K."""
    X = np.asarray(X)
    if elem_type == TET4:
        Xe = X[conn]
        Dm = np.swapaxes(Xe[:, 1:] - Xe[:, [0]], 1, 2)
        V = np.linalg.det(Dm) / 6.0
        base = (np.ones((4, 4)) + np.eye(4)) / 20.0
        return rho * V[:, None, None] * base[None]
    Xe = X[conn]
    m = np.zeros((conn.shape[0], 8, 8))
    for xi in hex_gauss_points():
        N, dN = hex_shape(xi)
        detJ = np.linalg.det(np.einsum("eai,ar->eir", Xe, dN))
        m += rho * detJ[:, None, None] * np.outer(N, N)[None]
    return m


# ================================================= triplets, pattern and C

def triplet_dofs(conn):
    """(row, col) DOF of every triplet in the fill order
    t = ((e*npe + a)*npe + b)*9 + 3i + k, value K_e[3a+i, 3b+k].
    Section 4.2: the triplet stream of the element matrices.
    """
    conn = np.asarray(conn, dtype=np.int64)
    E, npe = conn.shape
    a = np.arange(npe)
    i = np.arange(3)
    # shapes [E, a, b, i, k]
    row = 3 * conn[:, :, None, None, None] + i[None, None, None, :, None]
    col = 3 * conn[:, None, :, None, None] + i[None, None, None, None, :]
    row = np.broadcast_to(row, (E, npe, npe, 3, 3)).reshape(-1)
    col = np.broadcast_to(col, (E, npe, npe, 3, 3)).reshape(-1)
    del a
    return row, col


def element_values_fill_order(Ke):
    """K_e [E, 3npe, 3npe] with index (3a+i, 3b+k) -> fill-order values [E*npe*npe*9].  Section
    4.2: values in the triplet stream's filling order."""
    E, n, _ = Ke.shape
    npe = n // 3
    return Ke.reshape(E, npe, 3, npe, 3).transpose(0, 1, 3, 2, 4).reshape(-1)


def csr_pattern(n_dof, conn, fixed_dofs):
    """CSR pattern of the projected matrix and the map C (triplet -> slot, or -1).

    Rows and columns ascending, duplicates merged, fixed rows hold only their
    diagonal, fixed columns are removed (Section 5.1); C[t] = -1 whenever the
    triplet's row or column DOF is fixed.  Built by sorting unique keys."""
    row, col = triplet_dofs(conn)
    fixed = np.zeros(n_dof, dtype=bool)
    fixed[np.asarray(fixed_dofs, dtype=np.int64)] = True
    keep = ~(fixed[row] | fixed[col])
    keys = row[keep] * n_dof + col[keep]
    fd = np.nonzero(fixed)[0].astype(np.int64)
    uniq = np.unique(np.concatenate([keys, fd * n_dof + fd]))
    r = uniq // n_dof
    colind = (uniq % n_dof).astype(np.int32)
    rowptr = np.zeros(n_dof + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    C = np.full(row.shape[0], -1, dtype=np.int64)
    C[keep] = np.searchsorted(uniq, keys)
    return rowptr, colind, C.astype(np.int32)


def triplets_to_csr(n, rows, cols, vals, prev=None):
    """Compressed matrix of a caller's triplet stream (Section 4.2 "Collect
    data" and "Build matrix pattern").  Returns (keep, rowptr, colind, C,
    values): keep is True when the (row, col) stream equals the previous one
    `prev` = (rows, cols) element by element and in length (the filling-order
    test of Algorithm "add"), the pattern has rows and columns ascending with
    duplicates merged, C maps triplet t to its slot, and every slot's value is
    the sum of its triplets in ascending t order.  Built by sorting unique
    keys, not by the double transpose."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    keep = prev is not None and len(prev[0]) == len(rows) and bool(
        np.array_equal(prev[0], rows) and np.array_equal(prev[1], cols))
    keys = rows * n + cols
    uniq, C = np.unique(keys, return_inverse=True)
    colind = (uniq % n).astype(np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, uniq // n + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    values = np.zeros(uniq.shape[0], dtype=np.float64)
    np.add.at(values, C, np.asarray(vals, dtype=np.float64))  # in ascending t per slot
    return keep, rowptr, colind, C.astype(np.int32), values


def assemble(n_dof, conn, values_fill_order):
    """Unconstrained global matrix: plain sum of every triplet (COO -> CSR).
    Section 4.2 ("Collect data"): duplicates summed."""
    row, col = triplet_dofs(conn)
    return sp.coo_matrix((values_fill_order, (row, col)), shape=(n_dof, n_dof)).tocsr()


def mass_fill_order(m_scalar):
    """Mass scalars m[e, a, b] -> fill-order triplet values (block m_ab * I3).  Section 4.1."""
    E, npe, _ = m_scalar.shape
    blk = m_scalar[:, :, :, None, None] * _I3[None, None, None]
    return blk.reshape(-1)


def project(Afull, fixed_dofs):
    """Projective constraints: clear fixed rows and columns, 1 on the diagonal.  Section 5.1."""
    n = Afull.shape[0]
    keep = np.ones(n)
    keep[np.asarray(fixed_dofs, dtype=np.int64)] = 0.0
    D = sp.diags(keep)
    fixd = sp.diags(1.0 - keep)
    return (D @ Afull @ D + fixd).tocsr()


def values_in_pattern(Aproj, rowptr, colind):
    """Values of a sparse matrix read at every slot of a CSR pattern.  Section 4.2: a matrix read
    on the compressed pattern."""
    n = rowptr.shape[0] - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    return np.asarray(Aproj[rows, colind]).reshape(-1)


# ================================================================ the model

class Model:
    """A mesh + material + time-integration parameters; state-independent data.  Section 3 (the
    step), Section 4 (assembly), Section 5.1 (constraints)."""

    def __init__(self, elem_type, X, conn, fixed_nodes, model, params, rho, h, alpha, beta):
        self.elem_type = elem_type
        self.X = np.asarray(X, dtype=np.float64)
        self.conn = np.asarray(conn, dtype=np.int64)
        self.n_dof = 3 * self.X.shape[0]
        fn = np.asarray(fixed_nodes, dtype=np.int64)
        self.fixed_dofs = (3 * fn[:, None] + np.arange(3)[None, :]).reshape(-1)
        self.model = model
        self.params = np.asarray(params)
        self.params = self.params.astype(np.result_type(self.params.dtype, np.float64))
        self.rho, self.h, self.alpha, self.beta = rho, h, alpha, beta
        self.quad = Quadrature(elem_type, self.X, self.conn)
        self.m_e = element_mass(elem_type, self.X, self.conn, rho)
        self.M = assemble(self.n_dof, self.conn, mass_fill_order(self.m_e))

    @classmethod
    def from_workload(cls, wl, params=None):
        """The model of a seeded workload: mesh, law, h and the Rayleigh alpha, beta of
        Eq. "dynamic equation1"."""
        m = wl.mesh
        return cls(m.elem_type, m.X, m.conn, m.fixed_nodes, wl.model,
                   wl.params if params is None else params, wl.rho, wl.h, wl.alpha, wl.beta)

    # -- per element
    def energy(self, q):
        """Total elastic energy at positions q (Section 3.1)."""
        return element_energy(self.quad, q.reshape(-1, 3), self.model, self.params).sum()

    def element_force(self, q):
        """Per-element internal forces f_e at q (Section 3.1)."""
        return element_force(self.quad, q.reshape(-1, 3), self.model, self.params)

    def element_tangent(self, q):
        """Per-element tangents K_e = df_e/dq at q (Section 3.1)."""
        return element_tangent(self.quad, q.reshape(-1, 3), self.model, self.params)

    # -- assembled
    def internal_force(self, q):
        """Assembled f(q) (Section 4.2 summation of the element forces)."""
        fe = self.element_force(q)
        f = np.zeros(self.n_dof, dtype=fe.dtype)
        dofs = (3 * self.conn[:, :, None] + np.arange(3)[None, None, :]).reshape(fe.shape[0], -1)
        np.add.at(f, dofs.reshape(-1), fe.reshape(-1))
        return f

    def stiffness(self, q):
        """Assembled K(q), unprojected (Section 4.2)."""
        return assemble(self.n_dof, self.conn, element_values_fill_order(self.element_tangent(q)))

    def system(self, q, v, p):
        """Projected A and b of one step (Eq. "dynamic equation2"; C-1 reading of b)."""
        h, al, be = self.h, self.alpha, self.beta
        f = self.internal_force(q)
        K = self.stiffness(q)
        A = (1.0 + h * al) * self.M + h * (be + h) * K
        b = p - f - (al * (self.M @ v) + (be + h) * (K @ v))
        b[self.fixed_dofs] = 0.0
        return project(A, self.fixed_dofs), b

    def step(self, q, v, p):
        """One backward-Euler step with one Newton iteration; direct solve.  Eqs. "dynamic
        equation2" and "implicit integration"."""
        A, b = self.system(q, v, p)
        a = direct_solve(A, b)
        v1 = v + self.h * a
        q1 = q + self.h * v1
        return q1, v1, a

    def step_cg(self, q, v, p, tol):
        """The same step as step() with the linear system solved by Jacobi
        CG to ||b - A a|| <= tol ||b|| (cg_solve) instead of the direct
        solve: the CPU analogue of fast assembly + CG, and, at tol 1e-13, a
        reference for meshes whose direct factor is too large for the host.
        Returns q+, v+, a and the CG iterations."""
        A, b = self.system(q, v, p)
        a, its = cg_solve(A.tocsr(), b, tol)
        v_next = v + self.h * a
        return q + self.h * v_next, v_next, a, its

    def newton_residual(self, q, v, p, a):
        """Nonlinear backward-Euler residual of one step at the acceleration a:
        R(a) = M a + f(q') + (alpha M + beta K(q')) v' - p with v' = v + h a,
        q' = q + h v' (Eqs. "newton's law" and "implicit integration", the
        Rayleigh damping taken at the end-of-step configuration), zero on the
        fixed DOFs."""
        h, al, be = self.h, self.alpha, self.beta
        v1 = v + h * a
        q1 = q + h * v1
        R = self.M @ a + self.internal_force(q1) + al * (self.M @ v1) + be * (self.stiffness(q1) @ v1) - p
        R[self.fixed_dofs] = 0.0
        return R

    def newton_step(self, q, v, p, iters):
        """Backward Euler by `iters` Newton iterations on newton_residual.
        Iteration 1 is the paper's linearised step (step()); iteration k > 1
        solves A(q_k) delta = -R(a_k) with the same matrix form
        A = (1 + h alpha) M + h (beta + h) K(q_k) at q_k = q + h v + h^2 a_k
        (the derivative of K in the damping term is not taken) and sets
        a_{k+1} = a_k + delta.  Returns q+, v+, a and the norms of the
        corrections.
        Eqs. "newton's law" and "implicit integration".
        """
        h = self.h
        _, _, a = self.step(q, v, p)
        corr = []
        for _ in range(1, iters):
            qk = q + h * v + h * h * a
            K = self.stiffness(qk)
            A = project((1.0 + h * self.alpha) * self.M + h * (self.beta + h) * K, self.fixed_dofs)
            delta = direct_solve(A, -self.newton_residual(q, v, p, a))
            a = a + delta
            corr.append(float(np.linalg.norm(delta)))
        v1 = v + h * a
        return q + h * v1, v1, a, corr

    def pattern(self):
        """CSR pattern and map C of this mesh (Section 4.2, Section 5.1)."""
        return csr_pattern(self.n_dof, self.conn, self.fixed_dofs)

    def contact_jacobian(self, nodes, normals):
        """H (m x n_dof): row i is the unit normal n_i on the three DOFs of
        node i (Section "Lagrangian multipliers", Eq. "KKT": the linearised
        constraint equations of a deformable object against a rigid one)."""
        m = len(nodes)
        rows = np.repeat(np.arange(m), 3)
        cols = (3 * np.asarray(nodes)[:, None] + np.arange(3)).reshape(-1)
        return sp.csr_matrix((np.asarray(normals, float).reshape(-1), (rows, cols)), shape=(m, self.n_dof))

    def contact_step(self, q, v, p, nodes, normals, offsets, sweeps=200, tol=1e-12):
        """One step with frictionless contacts against rigid planes
        n_i . x >= c_i (x the node's end-of-step position), in the paper's
        three stages (Section "Lagrangian multipliers"):
          * free motion: A a_free = b (the step without contacts);
          * constraint resolution: compliance W = H A^{-1} H^T and the LCP
            lambda >= 0, w = W lambda - (delta - H a_free) >= 0,
            lambda . w = 0, solved by projected Gauss-Seidel; here
            x_end = q + h v + h^2 a, so the constraint on the unknown a is
            H a >= delta with delta_i = (c_i - n_i . (q + h v)_node) / h^2;
          * motion correction: a = a_free + A^{-1} H^T lambda.
        Returns q+, v+, a, lambda and W."""
        A, b = self.system(q, v, p)
        a_free = direct_solve(A, b)
        H = self.contact_jacobian(nodes, normals)
        Z = np.column_stack([direct_solve(A, H.getrow(i).toarray().ravel()) for i in range(H.shape[0])]) \
            if H.shape[0] else np.zeros((self.n_dof, 0))
        W = H @ Z
        h = self.h
        x_pred = (q + h * v).reshape(-1, 3)[np.asarray(nodes)]
        delta = (np.asarray(offsets, float) - np.einsum("ij,ij->i", np.asarray(normals, float), x_pred)) / (h * h)
        lam = pgs(W, delta - H @ a_free, sweeps, tol)
        a = a_free + Z @ lam
        v1 = v + h * a
        return q + h * v1, v1, a, lam, W


def pgs(W, r, sweeps, tol):
    """Projected Gauss-Seidel for the LCP lambda >= 0, W lambda - r >= 0,
    lambda . (W lambda - r) = 0 (the constraint-resolution step of Section
    "Lagrangian multipliers"): constraints in index order, each set to the
    non-negative value that zeroes its own residual given the others; stops
    when a sweep changes no lambda by more than tol * max |lambda|.  A
    constraint with W_ii <= 0 (a node that cannot move) keeps lambda = 0."""
    m = W.shape[0]
    lam = np.zeros(m)
    for _ in range(sweeps):
        dmax = 0.0
        for i in range(m):
            if W[i, i] <= 0.0:
                continue
            new = max(0.0, lam[i] + (r[i] - W[i] @ lam) / W[i, i])
            dmax = max(dmax, abs(new - lam[i]))
            lam[i] = new
        if dmax <= tol * max(1e-300, np.abs(lam).max()):
            break
    return lam


def direct_solve(A, b):
    """Sparse direct solve (SuperLU with a symmetric fill-reducing order).  The exact solve that
    the lagged LDL^T preconditioner of Section 3.3 approximates."""
    if A.shape[0] <= 3000:
        return np.linalg.solve(A.toarray(), b)
    lu = spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A")
    return lu.solve(b)


def cg_solve(A, b, tol, maxiter=100000):
    """Conjugate gradients (Hestenes-Stiefel) with the Jacobi preconditioner
    diag(A)^-1 on the SPD system A x = b from x = 0, stopped once the true
    residual satisfies ||b - A x||_2 <= tol ||b||_2: the stopping test the
    paper's CG uses on the assembled system (Section 6.2, "System
    solution"), here without the LDL^T preconditioner.  Returns (x, iterations).
    Each iteration is one sparse product and a few vector updates.  In FP64
    the true residual levels off (near 4e-13 of ||b|| on the 348,843-DOF
    beam): a tolerance below that level raises instead of looping."""
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0
    dinv = 1.0 / A.diagonal()
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = r @ z
    misses = 0
    for k in range(1, maxiter + 1):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        if np.linalg.norm(r) <= tol * bn:
            r = b - A @ x                     # the recursion's residual drifts: confirm with the true one
            if np.linalg.norm(r) <= tol * bn:
                return x, k
            misses += 1
            if misses > 20:
                raise RuntimeError("cg_solve: the true residual stays above tol (below FP64's reach)")
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    raise RuntimeError("cg_solve: no convergence")


def rollout(model, q0, v0, loads, n_steps):
    """q_t, v_t for t = 0..n_steps (loads(t) -> p_t as a [n_dof] vector).  Eq. "implicit
    integration" iterated."""
    qs, vs = [q0.copy()], [v0.copy()]
    q, v = q0.copy(), v0.copy()
    for t in range(n_steps):
        q, v, _ = model.step(q, v, loads(t))
        qs.append(q)
        vs.append(v)
    return np.array(qs), np.array(vs)


# ================================================================ adjoint
# Discrete adjoint of the rollout (reading C-12 of the reconstruction notes):
# step residual R(a; q, v, s, p) = A(q, s) a - b(q, v, s, p) with every
# element's energy scaled by s_e (Young's modulus E_e = s_e * E_ref at fixed
# nu, or the three Mooney-Rivlin constants together).  Backwards:
#   a_bar = h v_bar_{t+1} + h^2 q_bar_{t+1};   A_t lambda = a_bar
#   q_bar_t = q_bar_{t+1} - (c_K dK[lambda] a + (beta+h) dK[lambda] v + K lambda)
#   v_bar_t = v_bar_{t+1} + h q_bar_{t+1} - (alpha M + (beta+h) K) lambda
#   s_bar_e -= lambda_e . (c_K K_e a_e + f_e + (beta+h) K_e v_e)
#   p_bar_t = lambda
# dK[lambda] u is the directional derivative of the element tangents along
# lambda, taken here by a complex step of the analytic tangent.

def _gather_elem(conn, x):
    xe = np.asarray(x).reshape(-1, 3)[conn]
    return xe.reshape(conn.shape[0], -1)


def _scatter_elem(n_dof, conn, ve):
    out = np.zeros(n_dof, dtype=ve.dtype)
    dofs = (3 * conn[:, :, None] + np.arange(3)[None, None, :]).reshape(conn.shape[0], -1)
    np.add.at(out, dofs.reshape(-1), ve.reshape(-1))
    return out


def rollout_with_history(model, q0, v0, loads, T):
    """rollout keeping every (q_t, v_t, a_t): the checkpoints of the discrete adjoint (Eq.
    "implicit integration" iterated; the adjoint is not in the paper)."""
    qs, vs, accs = [q0.copy()], [v0.copy()], []
    q, v = q0.copy(), v0.copy()
    for t in range(T):
        q, v, a = model.step(q, v, loads(t))
        qs.append(q)
        vs.append(v)
        accs.append(a)
    return qs, vs, accs


def adjoint_rollout(model, q0, v0, loads, T, q_target, v_bar_T=None):
    """Loss L = 1/2 ||q_T - q_target||^2 and its gradients:
    returns (L, dL/ds [E] for the per-element energy scales, dL/dp [T, n]).
    Not in the paper: the discrete adjoint of the step of Eq. "dynamic equation2".
    """
    h, al, be = model.h, model.alpha, model.beta
    cK = h * (be + h)
    qs, vs, accs = rollout_with_history(model, q0, v0, loads, T)
    diff = qs[T] - q_target
    loss = 0.5 * float(diff @ diff)
    q_bar = diff.copy()
    v_bar = np.zeros_like(q_bar) if v_bar_T is None else np.asarray(v_bar_T, dtype=np.float64).copy()
    s_bar = np.zeros(model.conn.shape[0])
    p_bar = np.zeros((T, model.n_dof))
    conn = model.conn
    for t in range(T - 1, -1, -1):
        q, v, a = qs[t], vs[t], accs[t]
        A, _ = model.system(q, v, loads(t))
        a_bar = h * v_bar + h * h * q_bar
        a_bar[model.fixed_dofs] = 0.0
        lam = direct_solve(A, a_bar)
        lam[model.fixed_dofs] = 0.0
        Ke = model.element_tangent(q)
        fe = model.element_force(q)
        ae, ve, le = _gather_elem(conn, a), _gather_elem(conn, v), _gather_elem(conn, lam)
        u = cK * ae + (be + h) * ve
        eps = 1e-30
        Kc = element_tangent(model.quad, (q + 1j * eps * lam).reshape(-1, 3), model.model, model.params)
        dKu = np.einsum("eij,ej->ei", Kc.imag / eps, u)
        Kl = np.einsum("eij,ej->ei", Ke, le)
        gq = _scatter_elem(model.n_dof, conn, dKu + Kl)
        Klam = _scatter_elem(model.n_dof, conn, Kl)
        gv = al * (model.M @ lam) + (be + h) * Klam
        s_bar -= np.einsum("ei,ei->e", le, cK * np.einsum("eij,ej->ei", Ke, ae) + fe
                           + (be + h) * np.einsum("eij,ej->ei", Ke, ve))
        p_bar[t] = lam
        q_bar, v_bar = q_bar - gq, v_bar + h * q_bar - gv
    return loss, s_bar, p_bar
