"""Parity at the full size of the 350k-DOF beam (tet30x30x120, 348,843 DOF,
648,000 tets, Mooney-Rivlin, mixed precision, factor of A_s taken every R = 5
steps and first used k = 5 steps later, binary16 copy of the apply
operators: the launch configuration that bench.py times).

The oracle cannot solve this system in seconds, so it is compared on outputs it
computes one by one, from the elements that touch a seeded sample of nodes
(clamped, interior and free-end nodes):
  * CSR rows of the pattern, bit-exact, and every scatter-map entry of the
    sampled elements (slot of the right (row, column), -1 exactly when a DOF
    is fixed);
  * the element kernel's force and tangent of sampled elements (Section 3.1);
  * rows of the assembled A and b (Eqs. "dynamic equation1/2") at the sampled
    nodes, whose rows are complete in the sub-mesh;
  * over eleven steps (the first factorisation, then the lagged one launched
    at step 5 on the side stream and first used at step 10),
    the rows of A and b at each step's own state, and the step's acceleration
    a = (v_{t+1} - v_t)/h put into the oracle's own FP64 equations at the
    sampled rows.
Properties that hold at any size cover the rest of each step: a solves the
library's assembled system to the requested tolerance, q_{t+1} = q_t + h
v_{t+1}, and the clamped face stays at rest.  Last, the FP64 exact factor of
the same mesh at rest inverts A to 1e-9 (Section 3.3's preconditioner with
no lag).

Tolerances: element and assembly values 2e-5 of the largest sampled entry (FP32
element math, as in the small-mesh parity tests), b during the steps 2e-5 of the
largest |A||a| + |b| row term; the oracle-equation residual
1e-4 of |A||a| + |b| over the sampled rows (the FP32 tangent perturbs A by
~1e-7 relative, the solve is driven to 1e-8 by FP64 refinement; a wrong term or
sign leaves O(1); terms as small as the Rayleigh mass damping are the FP64
small-mesh tests' business, at 1e-12); the library-system residual 1e-6 of |b|
(PCG stops at 1e-8).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import fe_inputs as fi
from oracle import fe_oracle as O

pytestmark = pytest.mark.gpu

WORKLOAD = "tet30x30x120-mr"
STEPS = 11
LAG = 5         # bench.py's default factor_lag for this workload (k = R)


# ------------------------------------------------------------------ samples

def sample_nodes(mesh, k, seed):
    rng = np.random.default_rng(seed)
    n_nodes = mesh.X.shape[0]
    pick = rng.choice(n_nodes, size=min(k, n_nodes), replace=False)
    extra = np.concatenate([np.asarray(mesh.fixed_nodes[:5]), [0, n_nodes - 1]])
    return np.unique(np.concatenate([pick, extra]).astype(np.int64))


def node_dofs(nodes):
    return (3 * np.asarray(nodes, dtype=np.int64)[:, None] + np.arange(3)).reshape(-1)


def elements_touching(conn, nodes):
    return np.nonzero(np.isin(conn, nodes).any(axis=1))[0]


def sub_model(wl, elems):
    m = wl.mesh
    params = wl.params if np.ndim(wl.params) == 1 else np.asarray(wl.params)[elems]
    return O.Model(m.elem_type, m.X, m.conn[elems], m.fixed_nodes, wl.model, params, wl.rho, wl.h,
                   wl.alpha, wl.beta)


def deformed_state(mesh, seed):
    rng = np.random.default_rng(seed)
    q = mesh.X.reshape(-1) + 5e-4 * rng.standard_normal(mesh.X.size)
    fixed = node_dofs(mesh.fixed_nodes)
    q[fixed] = mesh.X.reshape(-1)[fixed]
    v = 0.01 * rng.standard_normal(mesh.X.size)
    v[fixed] = 0.0
    p = 0.1 * rng.standard_normal(mesh.X.size)
    return q, v, p


def row_slots(rowptr, rows):
    lens = np.asarray(rowptr[rows + 1], dtype=np.int64) - np.asarray(rowptr[rows], dtype=np.int64)
    slots = np.concatenate([np.arange(rowptr[i], rowptr[i + 1], dtype=np.int64) for i in rows])
    return slots, np.repeat(rows, lens)


# ------------------------------------------------------------------- checks

def check_pattern_and_scatter_map(wl, ctx, n_nodes=400, seed=1):
    mesh = wl.mesh
    nodes = sample_nodes(mesh, n_nodes, seed)
    elems = elements_touching(mesh.conn, nodes)
    fixed = node_dofs(mesh.fixed_nodes)
    rp, ci, C_sub = O.csr_pattern(ctx.n, mesh.conn[elems], fixed)
    rowptr = np.asarray(ctx.rowptr, dtype=np.int64)
    colind = np.asarray(ctx.colind)
    for i in node_dofs(nodes):
        np.testing.assert_array_equal(colind[rowptr[i]:rowptr[i + 1]], ci[rp[i]:rp[i + 1]])
    # scatter map of the sampled elements: global triplet ids, fill order
    npe = mesh.conn.shape[1]
    per = 9 * npe * npe
    t_glob = (elems[:, None] * per + np.arange(per)[None, :]).reshape(-1)
    Cg = np.asarray(ctx.C)[t_glob].astype(np.int64)
    row, col = O.triplet_dofs(mesh.conn[elems])
    dropped = C_sub < 0
    assert np.array_equal(Cg < 0, dropped)
    s, r, c = Cg[~dropped], row[~dropped], col[~dropped]
    assert np.all(rowptr[r] <= s) and np.all(s < rowptr[r + 1])
    assert np.array_equal(colind[s].astype(np.int64), c)
    return len(nodes), len(elems)


def check_element_kernel(wl, ctx, n_elems=3000, seed=2, tol=2e-5):
    mesh = wl.mesh
    q, _, _ = deformed_state(mesh, seed)
    f, K = ctx.element_eval(q)
    rng = np.random.default_rng(seed)
    E = mesh.conn.shape[0]
    elems = np.unique(np.concatenate([rng.choice(E, size=min(n_elems, E), replace=False), [0, E - 1]]))
    m = sub_model(wl, elems)
    fo = m.element_force(q)
    Ko = O.element_values_fill_order(m.element_tangent(q)).reshape(len(elems), -1)
    Kg = np.asarray(K).reshape(E, -1)[elems]
    assert np.abs(np.asarray(f)[elems] - fo).max() <= 1e-12 * np.abs(fo).max()   # FP64 forces
    assert np.abs(Kg - Ko).max() <= tol * np.abs(Ko).max()
    return len(elems)


def compare_rows(ctx, A, b, Ao, bo, rows, tol, b_scale=None):
    """Rows of the library's A and b against the oracle's.  b is measured against
    b_scale when given (the size of the equation's terms): at rest b is the
    small dead load alone, while the FP32 element force leaves noise of the
    order of the stiffness times the rounding of F."""
    slots, srow = row_slots(np.asarray(ctx.rowptr, dtype=np.int64), rows)
    Av = np.asarray(Ao[srow, np.asarray(ctx.colind)[slots]]).reshape(-1)
    assert np.abs(A[slots] - Av).max() <= tol * np.abs(Av).max()
    bs = np.abs(bo[rows]).max() if b_scale is None else b_scale
    assert np.abs(b[rows] - bo[rows]).max() <= tol * bs


def check_assembly_rows(wl, ctx, n_nodes=400, seed=3, tol=2e-5):
    mesh = wl.mesh
    q, v, p = deformed_state(mesh, seed)
    ctx.set_state(q, v)
    A, b = ctx.assemble(p)
    nodes = sample_nodes(mesh, n_nodes, seed)
    rows = node_dofs(nodes)
    m = sub_model(wl, elements_touching(mesh.conn, nodes))
    Ao, bo = m.system(q, v, p)
    compare_rows(ctx, A, b, Ao, bo, rows, tol)
    return len(rows)


def check_steps(wl, ctx, steps=STEPS, n_nodes=200, seed=4, tol_oracle=1e-4, tol_lib=1e-6, tol_rows=2e-5):
    mesh = wl.mesh
    n = ctx.n
    X = mesh.X.reshape(-1)
    q, v = X.copy(), np.zeros(n)
    ctx.set_state(q, v)
    nodes = sample_nodes(mesh, n_nodes, seed)
    rows = node_dofs(nodes)
    m = sub_model(wl, elements_touching(mesh.conn, nodes))
    fixed = node_dofs(mesh.fixed_nodes)
    worst = 0.0
    for t in range(steps):
        p = wl.p(t).reshape(-1)
        A, b = ctx.assemble(p)  # the library's own system at (q_t, v_t)
        q1, v1 = np.empty(n), np.empty(n)
        ctx.step(p, q1, v1)
        a = (v1 - v) / wl.h
        S = sp.csr_matrix((A, np.asarray(ctx.colind), np.asarray(ctx.rowptr)), shape=(n, n))
        assert np.linalg.norm(S @ a - b) <= tol_lib * np.linalg.norm(b)
        Ao, bo = m.system(q, v, p)
        scale = (abs(Ao) @ np.abs(a) + np.abs(bo))[rows]
        compare_rows(ctx, A, b, Ao, bo, rows, tol_rows, b_scale=scale.max())  # the step's own state
        r = (Ao @ a - bo)[rows]
        rel = np.linalg.norm(r) / np.linalg.norm(scale)
        worst = max(worst, rel)
        assert rel <= tol_oracle
        np.testing.assert_allclose(q1, q + wl.h * v1, rtol=0, atol=1e-15 * max(1.0, np.abs(q1).max()))
        assert np.all(v1[fixed] == 0.0) and np.all(q1[fixed] == X[fixed])
        q, v = q1, v1
    assert np.abs(q - X).max() > 0.0  # the beam moved
    return worst


def check_exact_factor(wl, ctx, seed=5, tol=1e-9):
    """FP64 factor of A at rest, applied once: z = A^{-1} r up to rounding.
    On this mesh 13 fronts have more than 4,096 update rows, so the assembly
    reads their row maps from global memory; a wrong extend-add anywhere
    leaves an O(1) residual."""
    A, _ = ctx.assemble()
    ctx.factor_now()
    rng = np.random.default_rng(seed)
    r = rng.standard_normal(ctx.n)
    fixed = node_dofs(wl.mesh.fixed_nodes)
    r[fixed] = 0.0
    z = ctx.apply_preconditioner(r)
    S = sp.csr_matrix((A, np.asarray(ctx.colind), np.asarray(ctx.rowptr)), shape=(ctx.n, ctx.n))
    res = np.linalg.norm(S @ z - r) / np.linalg.norm(r)
    assert res <= tol
    assert np.all(z[fixed] == 0.0)
    return res


# -------------------------------------------------------------------- tests

@pytest.fixture(scope="module")
def full(gpu_lib):
    wl = fi.workload(WORKLOAD)
    ctx = gpu_lib.FEContext.from_workload(wl, precond_fp16=1, factor_lag=LAG)
    yield wl, ctx
    ctx.close()


def test_fullsize_steps_solve_the_oracle_equations_at_sampled_rows(full):
    check_steps(*full)


def test_fullsize_pattern_and_scatter_map_sampled(full):
    check_pattern_and_scatter_map(*full)


def test_fullsize_element_kernel_sampled(full):
    check_element_kernel(*full)


def test_fullsize_assembly_sampled_rows(full):
    check_assembly_rows(*full)


def test_fullsize_exact_factor_inverts_A(gpu_lib):
    wl = fi.workload(WORKLOAD)
    ctx = gpu_lib.FEContext.from_workload(wl, precision=0, refactor_every=1)
    try:
        check_exact_factor(wl, ctx)
    finally:
        ctx.close()


# ------------------------------------------ positions after N steps at full size

def _golden():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tet30x30x120_mr_rollout.json")
    with open(path) as f:
        return json.load(f)


# Measured errors (displacement-relative, sampled DOFs) are printed; the bounds
# hold them with a margin.  FP64 and the mixed path with FP64 tangents solve
# the FP64 system to 1e-8 each step (measured 5.4e-12 and 3.8e-11 of the
# displacement after 10 steps); the default mixed path's FP32 tangents perturb
# A by their rounding, which the nearly incompressible Mooney-Rivlin law
# (kappa / mu ~ 12) amplifies (measured 2.3e-5).
@pytest.mark.parametrize("precision,k64,tol", [(0, 0, 1e-9), (1, 0, 5e-5), (1, 1, 1e-9)])
def test_fullsize_positions_after_ten_steps_match_the_oracle(gpu_lib, precision, k64, tol):
    """q and v after 10 steps from rest in the bench's launch configuration
    (R = 5, k = 5; binary16 apply operators in the mixed path) against the
    FP64 oracle's rollout (each step's system solved to 1e-12 by the
    oracle's CG; tests/golden/make_fullsize_reference.py), at every 97th
    node and the whole free end."""
    g = _golden()
    wl = fi.workload(WORKLOAD)
    ctx = gpu_lib.FEContext.from_workload(wl, precision=precision, element_fp64=k64,
                                          precond_fp16=1 if precision else 0, factor_lag=LAG)
    q, v = np.empty(ctx.n), np.empty(ctx.n)
    try:
        for t in range(g["steps"]):
            info = ctx.step(wl.p(t).reshape(-1), q, v)
            assert info.rel_residual <= wl.tol
    finally:
        ctx.close()
    S = np.asarray(g["dofs"])
    X = wl.mesh.X.reshape(-1)[S]
    qo, vo = np.asarray(g["q"]), np.asarray(g["v"])
    eq = np.linalg.norm(q[S] - qo) / np.linalg.norm(qo - X)
    ev = np.linalg.norm(v[S] - vo) / np.linalg.norm(vo)
    print(f"precision={precision} element_fp64={k64}: position error {eq:.3e}, velocity error {ev:.3e}")
    assert eq <= tol and ev <= 10 * tol, (eq, ev)
