"""GPU parity of the contact step (fe_set_contacts; Section "Lagrangian
multipliers": free motion, compliance W = H P^{-1} H^T with the step's
preconditioner, projected Gauss-Seidel, motion correction) against the
oracle's contact_step, with the exact factor of the current matrix
(refactor_every = 1, so P = A up to rounding)."""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O

pytestmark = pytest.mark.gpu


def _setup(fe, precision, **kw):
    mesh = fi.tet_beam(2, 2, 6)
    ctx = fe.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.NEOHOOKE, 1000.0,
                       (3.4e3, 3.1e4, 0.0), 0.01, 0.1, 0.01, precision=precision, refactor_every=1,
                       tol=1e-12 if precision == 0 else 1e-10, **kw)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, O.NEOHOOKE, (3.4e3, 3.1e4, 0.0),
                1000.0, 0.01, 0.1, 0.01)
    q = mesh.X.reshape(-1).copy()
    v = np.zeros_like(q)
    v.reshape(-1, 3)[:, 2] = -0.5 * mesh.X[:, 0] / mesh.X[:, 0].max()
    v[m.fixed_dofs] = 0.0
    p = fi.body_force(mesh, 1000.0, (0.0, 0.0, -9.81)).reshape(-1)
    nodes = np.nonzero((mesh.X[:, 2] == 0.0) & (mesh.X[:, 0] > 0.0))[0].astype(np.int32)
    return mesh, ctx, m, q, v, p, nodes


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-4)])
def test_contact_rollout_matches_oracle(gpu_lib, precision, tol):
    mesh, ctx, m, q, v, p, nodes = _setup(gpu_lib, precision)
    normals = np.tile([0.0, 0.0, 1.0], (len(nodes), 1))
    offsets = np.full(len(nodes), -0.002)
    ctx.set_state(q, v)
    ctx.set_contacts(nodes, normals, offsets)
    qg, vg = np.empty_like(q), np.empty_like(q)
    active = 0
    worst = [0.0, 0.0]
    for t in range(5):
        ctx.step(p, qg, vg)
        lam_g = ctx.contact_forces()
        q, v, _, lam, _ = m.contact_step(q, v, p, nodes, normals, offsets)
        active = max(active, int((lam > 0).sum()))
        scale = max(np.abs(lam).max(), 1e-30)
        worst[0] = max(worst[0], np.abs(lam_g - lam).max() / scale)
        assert np.abs(lam_g - lam).max() <= tol * scale, (t, np.abs(lam_g - lam).max(), scale)
        disp = np.abs(q - mesh.X.reshape(-1)).max()
        worst[1] = max(worst[1], np.abs(qg - q).max() / disp)
        assert np.abs(qg - q).max() <= tol * disp
        if precision == 0:
            gap = qg.reshape(-1, 3)[nodes, 2] - offsets
            assert gap.min() >= -1e-9 * 0.002
            assert lam_g.min() >= 0.0
    assert active >= 1
    print(f"contact precision={precision}: worst multiplier error {worst[0]:.2e}, position error {worst[1]:.2e}")
    ctx.close()


def test_distant_contacts_leave_the_step_unchanged(gpu_lib):
    mesh, ctx, m, q, v, p, nodes = _setup(gpu_lib, 0, spmv_variant=4)
    ctx2 = gpu_lib.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.NEOHOOKE, 1000.0,
                             (3.4e3, 3.1e4, 0.0), 0.01, 0.1, 0.01, precision=0, refactor_every=1, tol=1e-12,
                             spmv_variant=4)
    for c in (ctx, ctx2):
        c.set_state(q, v)
    ctx.set_contacts(nodes, np.tile([0.0, 0.0, 1.0], (len(nodes), 1)), np.full(len(nodes), -1.0))
    qa, qb = np.empty_like(q), np.empty_like(q)
    ctx.step(p, qa, None)
    ctx2.step(p, qb, None)
    assert np.all(ctx.contact_forces() == 0.0)
    np.testing.assert_array_equal(qa, qb)
    # removing the contacts
    ctx.set_contacts(np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros(0))
    ctx.step(p, qa, None)
    ctx2.step(p, qb, None)
    np.testing.assert_array_equal(qa, qb)
    ctx.close()
    ctx2.close()


def test_contact_arguments_are_checked(gpu_lib):
    mesh, ctx, m, q, v, p, nodes = _setup(gpu_lib, 0)
    with pytest.raises(gpu_lib.FEError) as ei:
        ctx.set_contacts([mesh.n_nodes], [[0.0, 0.0, 1.0]], [0.0])
    assert ei.value.status == 1
    with pytest.raises(gpu_lib.FEError):
        ctx.set_contacts([nodes[0]], [[0.0, 0.0, 0.0]], [0.0])
    ctx.close()
    _, ctx_ck, *_ = _setup(gpu_lib, 0, keep_checkpoints=1)
    with pytest.raises(gpu_lib.FEError):
        ctx_ck.set_contacts([nodes[0]], [[0.0, 0.0, 1.0]], [0.0])
    ctx_ck.close()
