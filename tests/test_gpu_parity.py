"""GPU parity: every stage of the CUDA path against the FP64 oracle, through
the C ABI, on seeded meshes that span several tiles and ragged tails.

Tolerances (relative to the largest entry of the oracle quantity):
  FP64 path: element outputs and assembled A, b <= 1e-12 (same sums, other
  rounding order); positions after N steps <= 1e-8 of the displacement.
  Mixed path (FP64-accurate element forces, assembly sums and residual in
  double-float, FP32 element tangents, FP32 inner solve and factor): forces
  <= 1e-12, tangents
  <= 2e-5 (FP32 rounding of the contraction), A and b <= MIX_SYS (the FP32
  tangents' rounding, about 6e-8 of each entry, summed); positions after N
  steps <= MIX_POS of the displacement.  With element_fp64 the tangents, A
  and b are the FP64 path's (<= 1e-12) and positions follow the oracle to
  1e-8 like the FP64 path: only the preconditioner is FP32, and the FP64
  refinement drives the residual of the FP64 system to the tolerance.
"""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O

pytestmark = pytest.mark.gpu

MIX_SYS = 2e-6
MIX_POS = 1e-5

LAWS = {fi.SVK: (3.4e3, 3.1e4, 0.0), fi.NEOHOOKE: (3.4e3, 3.1e4, 0.0),
        fi.MOONEY_RIVLIN: (1.5e3, 5e2, 5e4), fi.COROTATIONAL: (3.4e3, 3.1e4, 0.0)}


def _mesh(kind):
    return fi.tet_beam(3, 4, 9) if kind == "tet" else fi.hex_beam(3, 3, 7, jitter=0.1, seed=4)


def _state(mesh, amp=0.05, seed=0):
    rng = np.random.default_rng(seed)
    q = mesh.X.reshape(-1) + amp * 0.01 * rng.standard_normal(mesh.X.size)
    fixed = (3 * mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)
    q[fixed] = mesh.X.reshape(-1)[fixed]
    v = 0.01 * rng.standard_normal(mesh.X.size)
    v[fixed] = 0.0
    p = 0.1 * rng.standard_normal(mesh.X.size)
    return q, v, p


def _ctx(fe, mesh, law, precision, **kw):
    return fe.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, law, 1000.0, LAWS[law],
                        0.01, 0.1, 0.01, precision=precision, **kw)


@pytest.mark.parametrize("kind", ["tet", "hex"])
@pytest.mark.parametrize("law", [fi.SVK, fi.NEOHOOKE, fi.MOONEY_RIVLIN, fi.COROTATIONAL])
@pytest.mark.parametrize("precision,k64", [(0, 0), (1, 0), (1, 1)])
def test_element_kernel(gpu_lib, kind, law, precision, k64):
    mesh = _mesh(kind)
    q, _, _ = _state(mesh)
    ctx = _ctx(gpu_lib, mesh, law, precision, element_fp64=k64)
    f, K = ctx.element_eval(q)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, law, LAWS[law], 1000., .01, .1, .01)
    fo = m.element_force(q)
    Ko = O.element_values_fill_order(m.element_tangent(q))
    ferr = np.abs(f - fo).max() / np.abs(fo).max()
    kerr = np.abs(K - Ko).max() / np.abs(Ko).max()
    assert ferr <= 1e-12, ferr  # forces in FP64, or double-float (about 2^-46 per operation) when mixed
    assert kerr <= (1e-12 if precision == 0 or k64 else 2e-5), kerr
    ctx.close()


@pytest.mark.parametrize("kind,law", [("tet", fi.SVK), ("tet", fi.MOONEY_RIVLIN), ("hex", fi.NEOHOOKE),
                                      ("tet", fi.COROTATIONAL), ("hex", fi.COROTATIONAL)])
@pytest.mark.parametrize("precision,k64", [(0, 0), (1, 0), (1, 1)])
def test_assembly(gpu_lib, kind, law, precision, k64):
    mesh = _mesh(kind)
    q, v, p = _state(mesh, seed=1)
    ctx = _ctx(gpu_lib, mesh, law, precision, element_fp64=k64)
    ctx.set_state(q, v)
    A, b = ctx.assemble(p)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, law, LAWS[law], 1000., .01, .1, .01)
    Ao, bo = m.system(q, v, p)
    Av = O.values_in_pattern(Ao, ctx.rowptr, ctx.colind)
    tol = 1e-12 if precision == 0 or k64 else MIX_SYS
    aerr = np.abs(A - Av).max() / np.abs(Av).max()
    berr = np.abs(b - bo).max() / np.abs(bo).max()
    assert aerr <= tol, aerr
    assert berr <= tol, berr
    ctx.close()


@pytest.mark.parametrize("kind,leaf", [("tet", 64), ("tet", 8), ("hex", 16), ("hex", 4)])
def test_exact_factor_inverts_A(gpu_lib, kind, leaf):
    """FP64 LDL^T of the current A applied level by level is A^{-1}."""
    mesh = _mesh(kind)
    q, v, p = _state(mesh, amp=0.01, seed=2)     # A is SPD at this state
    ctx = _ctx(gpu_lib, mesh, fi.NEOHOOKE, 0, nd_leaf_nodes=leaf)
    ctx.set_state(q, v)
    A, _ = ctx.assemble(p)
    ctx.factor_now()
    rng = np.random.default_rng(3)
    r = rng.standard_normal(ctx.n)
    fixed = (3 * mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)
    r[fixed] = 0.0
    z = ctx.apply_preconditioner(r)
    import scipy.sparse as sp
    S = sp.csr_matrix((A, ctx.colind, ctx.rowptr), shape=(ctx.n, ctx.n))
    zo = O.direct_solve(S, r)
    assert np.linalg.norm(z - zo) <= 1e-9 * np.linalg.norm(zo)
    assert np.all(z[fixed] == 0.0)
    ctx.close()


@pytest.mark.parametrize("kind,law", [("tet", fi.MOONEY_RIVLIN), ("hex", fi.NEOHOOKE)])
def test_mixed_refinement_residual_is_the_fp64_residual(gpu_lib, kind, law):
    """The mixed path refines until its double-float residual b - A2 x2 (A
    and the iterate as float pairs) is below tol; recomputed in FP64 on the
    host from the same system (fe_assemble returns A2 summed to FP64, b is
    FP64) and the step's acceleration (from rest, a = v+ / h), the residual
    meets the tolerance too and agrees with the reported one to 1e-3 of
    the tolerance (the pairs carry ~48 bits: their rounding is far below)."""
    import scipy.sparse as sp
    mesh = _mesh(kind)
    q, _, p = _state(mesh, amp=0.01, seed=5)
    v = np.zeros_like(q)
    ctx = _ctx(gpu_lib, mesh, law, 1)
    ctx.set_state(q, v)
    A, b = ctx.assemble(p)
    qo, vo = np.empty_like(q), np.empty_like(q)
    info = ctx.step(p, qo, vo)
    a = vo / 0.01
    S = sp.csr_matrix((A, ctx.colind, ctx.rowptr), shape=(ctx.n, ctx.n))
    rel = np.linalg.norm(b - S @ a) / np.linalg.norm(b)
    print(f"{kind}: reported {info.rel_residual:.3e}, FP64 recomputed {rel:.3e}, {info.refinements} sweeps")
    assert info.refinements >= 2
    assert rel <= 1e-8
    assert abs(rel - info.rel_residual) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("bf16,tol", [(0, 1e-3), (1, 5e-2)])
def test_mixed_factor_is_a_close_preconditioner(gpu_lib, bf16, tol):
    """The FP32 factor of A (3xTF32 updates, or BF16 operands in the
    superpanels' deferred updates) applied to a random vector: P^{-1} r
    solves A z = r up to the factor's rounding."""
    mesh = _mesh("tet")
    q, v, p = _state(mesh, amp=0.01, seed=5)
    ctx = _ctx(gpu_lib, mesh, fi.MOONEY_RIVLIN, 1, update_bf16=bf16)
    ctx.set_state(q, v)
    A, _ = ctx.assemble(p)
    ctx.factor_now()
    r = np.random.default_rng(4).standard_normal(ctx.n)
    r[(3 * mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)] = 0.0
    z = ctx.apply_preconditioner(r)
    import scipy.sparse as sp
    S = sp.csr_matrix((A, ctx.colind, ctx.rowptr), shape=(ctx.n, ctx.n))
    res = np.linalg.norm(S @ z - r) / np.linalg.norm(r)
    print(f"mixed factor bf16={bf16}: relative residual {res:.2e}")
    assert res <= tol
    ctx.close()


@pytest.mark.parametrize("tf32,fp16,bf16,res_tol,sol_tol", [(0, 0, 0, 1e-4, 1e-3), (1, 0, 0, 3e-2, 3e-1),
                                                          (0, 1, 0, 3e-2, 3e-1), (0, 0, 1, 3e-2, 2e-2),
                                                          (0, 1, 1, 3e-2, 2e-2)])
@pytest.mark.parametrize("kind", ["tet", "hex"])
def test_mixed_factor_with_superpanels(gpu_lib, kind, tf32, fp16, bf16, res_tol, sol_tol):
    """FP32 factor of fronts wider than one superpanel (512 pivots, applied
    to the rest of the front once per superpanel; inside it, 128-pivot
    sub-blocks applied to the rest of the superpanel once per sub-block)
    with ragged tails: the preconditioned vector agrees with the FP64 direct
    solve to FP32 accuracy; a missed or doubled update would leave an O(1)
    error."""
    mesh = fi.tet_beam(14, 14, 40) if kind == "tet" else fi.hex_beam(13, 13, 30, jitter=0.1, seed=4)
    q, v, p = _state(mesh, amp=0.01, seed=6)
    ctx = _ctx(gpu_lib, mesh, fi.NEOHOOKE, 1, factor_tf32=tf32, precond_fp16=fp16, update_bf16=bf16)
    npiv = ctx.ordering()["npiv"]
    assert npiv.max() > 512 and np.any(npiv % 64 != 0)
    ctx.set_state(q, v)
    A, _ = ctx.assemble(p)
    ctx.factor_now()
    r = np.random.default_rng(8).standard_normal(ctx.n)
    fixed = (3 * mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)
    r[fixed] = 0.0
    z = ctx.apply_preconditioner(r)
    # a second factorisation of the same matrix reuses every scratch buffer
    # of the first (the BF16 copies hold the previous superpanels' values)
    # and must reproduce it bit for bit
    ctx.factor_now()
    np.testing.assert_array_equal(ctx.apply_preconditioner(r), z)
    import scipy.sparse as sp
    S = sp.csr_matrix((A, ctx.colind, ctx.rowptr), shape=(ctx.n, ctx.n))
    zo = O.direct_solve(S, r)
    res = np.linalg.norm(S @ z - r) / np.linalg.norm(r)
    sol = np.linalg.norm(z - zo) / np.linalg.norm(zo)
    print(f"superpanels {kind} tf32={tf32} fp16={fp16} bf16={bf16}: residual {res:.2e}, solution {sol:.2e}")
    assert res <= res_tol
    assert sol <= sol_tol
    assert np.all(z[fixed] == 0.0)
    ctx.close()


@pytest.mark.parametrize("kind", ["tet", "hex"])
@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, MIX_POS)])
def test_rollout_corotational(gpu_lib, kind, precision, tol):
    """Co-rotational beams sagging under gravity (large rotations, small
    strains) follow the oracle's rollout."""
    mesh = fi.tet_beam(3, 3, 10) if kind == "tet" else fi.hex_beam(3, 3, 10, jitter=0.1, seed=4)
    mu, lam = fi.lame_from_young(1e4, 0.3)
    grav = fi.body_force(mesh, 1000.0, (0.0, 0.0, -9.81)).reshape(-1)
    ctx = gpu_lib.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.COROTATIONAL, 1000.0,
                            (mu, lam, 0.0), 0.01, 0.1, 0.01, precision=precision, tol=1e-10, refactor_every=3)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, O.COROTATIONAL, (mu, lam, 0.0),
                1000.0, 0.01, 0.1, 0.01)
    q = mesh.X.reshape(-1).copy()
    v = np.zeros_like(q)
    qg, vg = np.empty_like(q), np.empty_like(q)
    for t in range(8):
        ctx.step(grav, qg, vg)
        q, v, _ = m.step(q, v, grav)
    disp = np.abs(q - mesh.X.reshape(-1)).max()
    assert disp > 1e-3
    assert np.abs(qg - q).max() <= tol * disp
    ctx.close()


def test_corotational_refuses_checkpoints(gpu_lib):
    mesh = fi.tet_beam(2, 2, 3)
    with pytest.raises(gpu_lib.FEError):
        gpu_lib.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.COROTATIONAL, 1000.0,
                          LAWS[fi.COROTATIONAL], 0.01, 0.1, 0.01, keep_checkpoints=1)


def test_fp16_copy_is_a_symmetric_close_preconditioner(gpu_lib):
    """The binary16 copy of Y changes M^{-1} = Y^T D^{-1} Y only by the
    entries' rounding: it stays symmetric (both sweeps read the same stored
    entries) and positive, and close to the FP32 copy's result."""
    mesh = _mesh("tet")
    q, v, p = _state(mesh, amp=0.01, seed=5)
    zs = {}
    for fp16 in (0, 1):
        # (3xTF32 updates: the binary16 copy's effect alone)
        ctx = _ctx(gpu_lib, mesh, fi.MOONEY_RIVLIN, 1, precond_fp16=fp16, update_bf16=0)
        ctx.set_state(q, v)
        A, _ = ctx.assemble(p)
        ctx.factor_now()
        rng = np.random.default_rng(4)
        fixed = (3 * mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)
        r, s = rng.standard_normal(ctx.n), rng.standard_normal(ctx.n)
        r[fixed] = s[fixed] = 0.0
        zr, zs_ = ctx.apply_preconditioner(r), ctx.apply_preconditioner(s)
        zs[fp16] = zr
        scale = np.linalg.norm(r) * np.linalg.norm(zs_)
        assert abs(r @ zs_ - s @ zr) <= 1e-5 * scale
        assert r @ zr > 0 and s @ zs_ > 0
        import scipy.sparse as sp
        S = sp.csr_matrix((A, ctx.colind, ctx.rowptr), shape=(ctx.n, ctx.n))
        assert np.linalg.norm(S @ zr - r) <= (1e-3 if fp16 == 0 else 1e-2) * np.linalg.norm(r)
        ctx.close()
    assert np.linalg.norm(zs[1] - zs[0]) <= 1e-2 * np.linalg.norm(zs[0])


@pytest.mark.parametrize("kind", ["tet", "hex"])
def test_rollout_with_fp16_preconditioner(gpu_lib, kind):
    """The binary16 Y coarsens only the preconditioner: the FP64-refined
    rollout follows the oracle to the mixed tolerance."""
    wl = fi.workload("tet-mr", a=3, b=3, c=10) if kind == "tet" else fi.workload("hex-nh", a=3, b=3, c=10)
    qg, vg, q, v, infos = _rollout_pair(gpu_lib, wl, 6, precision=1, precond_fp16=1)
    disp = np.abs(q - wl.mesh.X.reshape(-1)).max()
    assert np.abs(qg - q).max() <= MIX_POS * disp
    assert all(i.rel_residual <= wl.tol for i in infos)


def test_rollout_with_tf32_factor(gpu_lib):
    """Plain TF32 products in the factor coarsen only the preconditioner: the
    FP64-refined rollout still follows the oracle to the mixed tolerance."""
    wl = fi.workload("tet-mr", a=3, b=3, c=10)
    qg, vg, q, v, infos = _rollout_pair(gpu_lib, wl, 6, precision=1, factor_tf32=1)
    disp = np.abs(q - wl.mesh.X.reshape(-1)).max()
    assert np.abs(qg - q).max() <= MIX_POS * disp
    assert all(i.rel_residual <= wl.tol for i in infos)


@pytest.mark.parametrize("precision", [0, 1])
def test_indefinite_matrix_is_reported(gpu_lib, precision):
    """A random 5%-of-spacing jitter makes the neo-Hookean tangent indefinite
    (the oracle's A has a negative eigenvalue there): the factor reports a
    non-positive pivot as FE_ERR_BREAKDOWN (reading C-6)."""
    mesh = _mesh("tet")
    q, v, p = _state(mesh, amp=0.05, seed=2)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.NEOHOOKE,
                LAWS[fi.NEOHOOKE], 1000., .01, .1, .01)
    Ao, _ = m.system(q, v, p)
    assert np.linalg.eigvalsh(Ao.toarray()).min() < 0
    ctx = _ctx(gpu_lib, mesh, fi.NEOHOOKE, precision)
    ctx.set_state(q, v)
    ctx.assemble(p)
    with pytest.raises(gpu_lib.FEError) as ei:
        ctx.factor_now()
    assert ei.value.status == 6
    ctx.close()


def _rollout_pair(fe, wl, steps, **kw):
    ctx = fe.FEContext.from_workload(wl, **kw)
    om = O.Model.from_workload(wl)
    q = wl.mesh.X.reshape(-1).copy()
    v = np.zeros_like(q)
    qg = np.empty_like(q)
    vg = np.empty_like(q)
    infos = []
    for t in range(steps):
        p = wl.p(t).reshape(-1)
        infos.append(ctx.step(p, qg, vg))
        q, v, _ = om.step(q, v, p)
    ctx.close()
    return qg, vg, q, v, infos


def test_rollout_tet_svk_fp64_exact_factor(gpu_lib):
    """The small FP64 tet beam, 10 steps, exact LDL^T every step (R = 1)."""
    wl = fi.workload("tet4x4x16-svk-fp64")
    qg, vg, qo, vo, infos = _rollout_pair(gpu_lib, wl, 10)
    X = wl.mesh.X.reshape(-1)
    assert np.linalg.norm(qg - qo) <= 1e-8 * np.linalg.norm(qo - X)
    assert np.linalg.norm(vg - vo) <= 1e-8 * np.linalg.norm(vo)
    assert all(i.iters <= 2 for i in infos), [i.iters for i in infos]
    assert all(i.rel_residual <= 1e-10 for i in infos)


@pytest.mark.parametrize("precision,k64,tol", [(0, 0, 1e-8), (1, 0, MIX_POS), (1, 1, 1e-8)])
def test_rollout_tet_mr_lagged(gpu_lib, precision, k64, tol):
    """Mooney-Rivlin tet beam with gravity + end traction, lagged factor R = 5."""
    wl = fi.workload("tet-mr", a=4, b=4, c=12)
    wl.precision = precision
    qg, vg, qo, vo, infos = _rollout_pair(gpu_lib, wl, 8, element_fp64=k64)
    X = wl.mesh.X.reshape(-1)
    err = np.linalg.norm(qg - qo) / np.linalg.norm(qo - X)
    assert err <= tol, err
    assert all(i.rel_residual <= 1e-8 for i in infos)
    ages = [i.factor_age for i in infos]
    assert ages[:7] == [0, 1, 2, 3, 4, 5, 1], ages


@pytest.mark.parametrize("precision,k64,tol", [(0, 0, 1e-8), (1, 0, MIX_POS), (1, 1, 1e-8)])
def test_rollout_hex_nh(gpu_lib, precision, k64, tol):
    wl = fi.workload("hex-nh", a=3, b=3, c=10)
    wl.precision = precision
    qg, vg, qo, vo, infos = _rollout_pair(gpu_lib, wl, 6, element_fp64=k64)
    X = wl.mesh.X.reshape(-1)
    err = np.linalg.norm(qg - qo) / np.linalg.norm(qo - X)
    assert err <= tol, err


def test_zero_load_stays_at_rest(gpu_lib):
    wl = fi.workload("tet4x4x16-svk-fp64")
    ctx = gpu_lib.FEContext.from_workload(wl)
    q = np.empty(ctx.n)
    v = np.empty(ctx.n)
    info = ctx.step(np.zeros(ctx.n), q, v)
    assert np.all(q == wl.mesh.X.reshape(-1)) and np.all(v == 0.0)
    assert info.iters == 0
    ctx.close()


def test_unconstrained_free_fall_closed_form(gpu_lib):
    mesh0 = fi.tet_beam(2, 2, 5)
    mesh = fi.TetBeam(2, 2, 5, mesh0.X, mesh0.conn, np.zeros(0, np.int32))
    h, al = 0.01, 0.1
    ctx = gpu_lib.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.NEOHOOKE, 1000.0,
                            (3.4e3, 3.1e4, 0.0), h, al, 0.01)
    p = fi.body_force(mesh, 1000.0, (0, 0, -9.81)).reshape(-1)
    q = np.empty(ctx.n)
    v = np.empty(ctx.n)
    for t in range(1, 5):
        ctx.step(p, q, v)
        vt = -9.81 / al * (1 - (1 + h * al) ** (-t))
        np.testing.assert_allclose(v.reshape(-1, 3)[:, 2], vt, rtol=1e-9)
    ctx.close()


def test_inverted_element_is_reported(gpu_lib):
    mesh = fi.tet_beam(2, 2, 3)
    ctx = gpu_lib.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.NEOHOOKE, 1000.0,
                            (3.4e3, 3.1e4, 0.0), 0.01, 0.1, 0.01)
    q = mesh.X.reshape(-1).copy()
    far = mesh.n_nodes - 1
    q[3 * far:3 * far + 3] = mesh.X[0] - 0.05      # pull a corner node through its tets
    ctx.set_state(q, None)
    with pytest.raises(gpu_lib.FEError) as ei:
        ctx.step(np.zeros(ctx.n))
    assert ei.value.status == 7
    ctx.close()


def test_iteration_cap_is_reported(gpu_lib):
    wl = fi.workload("tet-mr", a=3, b=3, c=8)
    ctx = gpu_lib.FEContext.from_workload(wl, precision=0, max_iters=1, refactor_every=100, tol=1e-14)
    q = np.empty(ctx.n)
    with pytest.raises(gpu_lib.FEError) as ei:
        for t in range(0, 4):                     # the factor of A_0 is reused (R = 100)
            ctx.step(wl.p(t).reshape(-1) * (1.0 + 50.0 * t), q, None)
    assert ei.value.status == 5
    ctx.close()
