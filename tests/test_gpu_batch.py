"""Batched stepping (S11) on the GPU against per-member oracle rollouts: each
member of a batch of uneven beams (SVK and neo-Hookean) must follow its own
FP64 oracle trajectory (FP64 <= 1e-8, mixed <= 1e-5 of the displacement) and
report its own PCG iterations and residual, with the solve host-driven or
as one graph whose loops end on the device (use_graph), bit-identical."""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O

pytestmark = pytest.mark.gpu


def _small_members():
    rng = np.random.default_rng(3)
    out = []
    for k, (m, L) in enumerate([(2, 4), (3, 5), (2, 7), (3, 3), (2, 5)]):
        mesh = fi.tet_beam(m, m, L)
        model = fi.SVK if k % 2 == 0 else fi.NEOHOOKE
        mu, lam = fi.lame_from_young(float(rng.uniform(5e3, 5e4)), float(rng.uniform(0.3, 0.45)))
        load = fi.body_force(mesh, 1000.0, (0, 0, -9.81)) * (1.0 + k)
        out.append(fi.BatchMember(mesh, model, np.array([float(mu), float(lam), 0.0]), load))
    return out


@pytest.mark.parametrize("use_graph", [0, 1])
@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-5)])
def test_batch_members_follow_their_oracles(gpu_lib, precision, tol, use_graph):
    mem = _small_members()
    b = gpu_lib.FEBatch([(m.mesh.elem_type, m.mesh.X, m.mesh.conn, m.mesh.fixed_nodes, m.model, m.params)
                         for m in mem], 0.01, 0.1, 0.01, 1000.0, precision=precision, refactor_every=2,
                        use_graph=use_graph)
    p = b.concat([m.load for m in mem])
    q = np.empty(b.n)
    v = np.empty(b.n)
    T = 4
    for _ in range(T):
        info = b.step(p, q, v)
    iters, res = b.stats()
    assert np.all(iters >= 1) and np.all(res <= 1e-8)
    assert info.iters == iters.max()
    qs = b.split(q)
    for k, m in enumerate(mem):
        om = O.Model(m.mesh.elem_type, m.mesh.X, m.mesh.conn, m.mesh.fixed_nodes, m.model, m.params,
                     1000.0, 0.01, 0.1, 0.01)
        qo, _ = O.rollout(om, m.mesh.X.reshape(-1).copy(), np.zeros(3 * m.mesh.n_nodes),
                          lambda t: m.load.reshape(-1), T)
        X = m.mesh.X.reshape(-1)
        err = np.linalg.norm(qs[k] - qo[T]) / np.linalg.norm(qo[T] - X)
        assert err <= tol, (k, err)
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_graph_equals_host_driven_solve(gpu_lib, precision):
    """The batched solve as one graph runs the host-driven solve's kernels in
    the same order: identical states after several steps."""
    mem = _small_members()
    out = []
    for use_graph in (0, 1):
        b = gpu_lib.FEBatch([(m.mesh.elem_type, m.mesh.X, m.mesh.conn, m.mesh.fixed_nodes, m.model, m.params)
                             for m in mem], 0.01, 0.1, 0.01, 1000.0, precision=precision, refactor_every=3,
                            use_graph=use_graph, spmv_variant=2)
        p = b.concat([m.load for m in mem])
        q, v = np.empty(b.n), np.empty(b.n)
        its = [b.step(p, q, v).iters for _ in range(5)]
        out.append((q.copy(), v.copy(), its, b.stats()[0].copy()))
        b.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
    np.testing.assert_array_equal(out[0][3], out[1][3])
