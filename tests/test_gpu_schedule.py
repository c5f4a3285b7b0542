"""GPU: the schedule of the lagged factor and the bounded waits.

Eq. "asynchronous preconditioner" (Section 3.3) uses the factor of an earlier
matrix, available some steps after it was taken.  With refactor_every = R and
factor_lag = k the factor of A_s (s = 0 mod R) preconditions steps
s+k .. s+k+R-1 and steps 0 .. k+R-1 use the factor of A_0.  The lag changes
only the preconditioner: every step is still refined to the tolerance.

Failure detection without a GPU fault: the host deadline on a lagged factor
runs out because the factor of a large FP64 beam takes far longer than the
step that waits for it; a dependency wait of the preconditioner application
runs out because a test hook adds a pending child that nothing completes.
Both return FE_ERR_TIMEOUT with the state unchanged, and the context goes on
to give the same steps as an uninterrupted one.
"""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O

pytestmark = pytest.mark.gpu


def expected_age(t, R, k):
    """Steps since the matrix of the factor that preconditions step t."""
    if R == 1 or t < k + R:
        return t if R > 1 else 0
    s = ((t - k) // R) * R
    return t - s


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("lag", [1, 3, 5])
def test_factor_lag_schedule(gpu_lib, precision, lag):
    wl = fi.workload("tet-mr", a=4, b=4, c=12)
    R, steps = 5, 13
    ctx = gpu_lib.FEContext.from_workload(wl, precision=precision, refactor_every=R, factor_lag=lag)
    om = O.Model.from_workload(wl)
    q = wl.mesh.X.reshape(-1).copy()
    v = np.zeros_like(q)
    qg = np.empty_like(q)
    ages = []
    for t in range(steps):
        p = wl.p(t).reshape(-1)
        info = ctx.step(p, qg, None)
        ages.append(info.factor_age)
        assert info.rel_residual <= wl.tol
        q, v, _ = om.step(q, v, p)
    ctx.close()
    assert ages == [expected_age(t, R, lag) for t in range(steps)], ages
    X = wl.mesh.X.reshape(-1)
    err = np.linalg.norm(qg - q) / np.linalg.norm(q - X)
    assert err <= (1e-8 if precision == 0 else 1e-5), err


def test_expected_age_formula():
    # R = 5, k = 1: the factor of A_s preconditions steps s+1 .. s+5
    assert [expected_age(t, 5, 1) for t in range(12)] == [0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 1]
    assert [expected_age(t, 5, 5) for t in range(16)] == list(range(10)) + [5, 6, 7, 8, 9, 5]
    assert [expected_age(t, 1, 1) for t in range(4)] == [0, 0, 0, 0]


def _rollout(ctx, wl, t0, t1, q):
    for t in range(t0, t1):
        ctx.step(wl.p(t).reshape(-1), q, None)


def test_lagged_factor_deadline_runs_out_and_context_recovers(gpu_lib):
    """An FP64 factorisation of the 107,163-DOF tet beam takes far longer
    than the step that launched it: with a 1 microsecond deadline the first
    step that needs the lagged factor returns FE_ERR_TIMEOUT (the
    synchronous factor of step 0 is not held to it).  After the factor has
    finished the same step succeeds, and the rollout equals an
    uninterrupted one bit for bit."""
    import torch
    wl = fi.workload("tet-mr", a=20, b=20, c=80)
    kw = dict(precision=0, refactor_every=3, factor_lag=1, spmv_variant=4)
    ref = gpu_lib.FEContext.from_workload(wl, **kw)
    ctx = gpu_lib.FEContext.from_workload(wl, factor_timeout_s=1e-6, **kw)
    q_ref = np.empty(ref.n)
    q = np.empty(ctx.n)
    _rollout(ref, wl, 0, 6, q_ref)
    _rollout(ctx, wl, 0, 4, q)                    # step 3 launches the factor of A_3
    q_before, v_before = ctx.get_state()
    with pytest.raises(gpu_lib.FEError) as ei:
        ctx.step(wl.p(4).reshape(-1), q, None)    # step 4 needs it
    assert ei.value.status == 8 and "deadline" in str(ei.value)
    q_after, v_after = ctx.get_state()
    assert np.array_equal(q_after, q_before) and np.array_equal(v_after, v_before)
    torch.cuda.synchronize()                      # the factor completes on its stream
    _rollout(ctx, wl, 4, 6, q)
    assert np.array_equal(q, q_ref)
    ref.close()
    ctx.close()


def _root_front(ctx):
    order = ctx.ordering()
    roots = np.nonzero(order["parent"] < 0)[0]
    has_children = [f for f in roots if np.any(order["parent"] == f)]
    return int(has_children[0])


@pytest.mark.parametrize("precision", [0, 1])
def test_apply_dependency_wait_runs_out_and_context_recovers(gpu_lib, precision):
    """A root front held with one extra pending child: its forward tasks wait
    until dep_wait_s (20 ms) runs out, the application stops, the step
    returns FE_ERR_TIMEOUT with the state unchanged; the next calls run
    normally and equal an uninterrupted context's, bit for bit."""
    wl = fi.workload("tet-mr", a=3, b=4, c=9)
    kw = dict(precision=precision, refactor_every=1, dep_wait_s=0.02, spmv_variant=4)
    ref = gpu_lib.FEContext.from_workload(wl, **kw)
    ctx = gpu_lib.FEContext.from_workload(wl, **kw)
    q_ref, q = np.empty(ref.n), np.empty(ctx.n)
    _rollout(ref, wl, 0, 3, q_ref)
    _rollout(ctx, wl, 0, 1, q)
    q_before, v_before = ctx.get_state()
    ctx.hold_front(_root_front(ctx))
    with pytest.raises(gpu_lib.FEError) as ei:
        ctx.step(wl.p(1).reshape(-1), q, None)
    assert ei.value.status == 8 and "dependency wait" in str(ei.value)
    q_after, v_after = ctx.get_state()
    assert np.array_equal(q_after, q_before) and np.array_equal(v_after, v_before)
    _rollout(ctx, wl, 1, 3, q)
    assert np.array_equal(q, q_ref)
    # the same through fe_apply_preconditioner
    r = np.random.default_rng(5).standard_normal(ctx.n)
    r[(3 * wl.mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)] = 0.0
    z_ref = ref.apply_preconditioner(r)
    ctx.hold_front(_root_front(ctx))
    with pytest.raises(gpu_lib.FEError) as ei:
        ctx.apply_preconditioner(r)
    assert ei.value.status == 8
    assert np.array_equal(ctx.apply_preconditioner(r), z_ref)
    ref.close()
    ctx.close()


def test_hold_front_arguments(gpu_lib):
    wl = fi.workload("tet-mr", a=2, b=2, c=4)
    ctx = gpu_lib.FEContext.from_workload(wl)
    nf = ctx.info()["n_fronts"]
    for front, extra in ((-1, 1), (nf, 1), (0, 0)):
        with pytest.raises(gpu_lib.FEError) as ei:
            ctx.hold_front(front, extra)
        assert ei.value.status == 1
    ctx.close()
