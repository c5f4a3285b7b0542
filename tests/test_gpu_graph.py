"""The solve and integration of a step as one CUDA graph (fe_options.use_graph):
the PCG iterations, and in the mixed path the FP64 refinement sweeps around
them, are WHILE conditional nodes whose condition a kernel sets from the
device scalars, so a step reads the device once, at its end.  The kernels
and their order are those of the host-driven solve, so a rollout is
bit-identical to it; the iteration cap and a dependency-wait timeout are
still reported, and a failed step leaves the state unchanged (the
integration inside the graph is skipped on the device)."""
import numpy as np
import pytest

import fe_inputs as fi

pytestmark = pytest.mark.gpu


def _rollout(fe, wl, steps, **kw):
    ctx = fe.FEContext.from_workload(wl, spmv_variant=4, **kw)
    q = np.empty(ctx.n)
    v = np.empty(ctx.n)
    its = []
    for t in range(steps):
        its.append(ctx.step(wl.p(t).reshape(-1), q, v).iters)
    ctx.close()
    return q, v, its


@pytest.mark.parametrize("name,precision", [("tet4x4x16-svk-fp64", 0), ("tet-mr", 1), ("hex-nh", 0)])
def test_graph_replay_is_bit_identical(gpu_lib, name, precision):
    wl = fi.workload(name) if name.startswith("tet4") else fi.workload(name, a=3, b=3, c=10)
    wl.precision = precision
    q0, v0, it0 = _rollout(gpu_lib, wl, 6, refactor_every=3)
    q1, v1, it1 = _rollout(gpu_lib, wl, 6, refactor_every=3, use_graph=1)
    assert it0 == it1
    np.testing.assert_array_equal(q0, q1)
    np.testing.assert_array_equal(v0, v1)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_reports_the_iteration_cap(gpu_lib, precision):
    wl = fi.workload("tet4x4x16-svk-fp64")
    ctx = gpu_lib.FEContext.from_workload(wl, precision=precision, max_iters=2, refactor_every=100, tol=1e-14,
                                          use_graph=1)
    with pytest.raises(gpu_lib.FEError) as ei:
        for t in range(0, 6):
            q0, v0 = ctx.get_state()
            ctx.step(wl.p(t).reshape(-1))
    assert ei.value.status == 5
    q1, v1 = ctx.get_state()
    assert np.array_equal(q0, q1) and np.array_equal(v0, v1)   # the failed step changed nothing
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_step_dependency_timeout(gpu_lib, precision):
    """A held front inside the graph's first application: the wait runs out
    (dep_wait_s = 20 ms), the step returns FE_ERR_TIMEOUT with the state
    unchanged, and the rollout then equals the host-driven one."""
    wl = fi.workload("tet-mr", a=3, b=3, c=10)
    wl.precision = precision
    q_ref, v_ref, _ = _rollout(gpu_lib, wl, 3, refactor_every=1)
    ctx = gpu_lib.FEContext.from_workload(wl, refactor_every=1, use_graph=1, dep_wait_s=0.02, spmv_variant=4)
    q = np.empty(ctx.n)
    ctx.step(wl.p(0).reshape(-1), q, None)
    order = ctx.ordering()
    root = [f for f in np.nonzero(order["parent"] < 0)[0] if np.any(order["parent"] == f)][0]
    ctx.hold_front(int(root))
    before = ctx.get_state()
    with pytest.raises(gpu_lib.FEError) as ei:
        ctx.step(wl.p(1).reshape(-1), q, None)
    assert ei.value.status == 8
    after = ctx.get_state()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    for t in (1, 2):
        ctx.step(wl.p(t).reshape(-1), q, None)
    np.testing.assert_array_equal(q, q_ref)
    ctx.close()
