"""GPU: warm-started PCG (fe_options.warm_start).  Each step's solve starts
from the previous step's acceleration instead of 0; the stopping test
||b - A a|| <= tol ||b|| is the same, so the rollout follows the oracle to
the same tolerances as a cold start, with fewer iterations once the motion
is smooth.  The host-driven and the whole-step-graph solves run the same
kernels in the same order (bit-identical), and fe_set_state resets the
guess, so a rollout repeated from the same state is reproduced exactly."""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O

pytestmark = pytest.mark.gpu


def _rollout(fe, wl, steps, **kw):
    ctx = fe.FEContext.from_workload(wl, spmv_variant=4, **kw)
    q, v = np.empty(ctx.n), np.empty(ctx.n)
    its = [ctx.step(wl.p(t).reshape(-1), q, v).iters for t in range(steps)]
    ctx.close()
    return q, v, its


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-5)])
def test_warm_start_follows_the_oracle_with_fewer_iterations(gpu_lib, precision, tol):
    wl = fi.workload("tet-mr", a=4, b=4, c=12)
    wl.precision = precision
    steps = 10
    q_cold, _, it_cold = _rollout(gpu_lib, wl, steps)
    q_warm, _, it_warm = _rollout(gpu_lib, wl, steps, warm_start=1)
    om = O.Model.from_workload(wl)
    q = wl.mesh.X.reshape(-1).copy()
    v = np.zeros_like(q)
    for t in range(steps):
        q, v, _ = om.step(q, v, wl.p(t).reshape(-1))
    X = wl.mesh.X.reshape(-1)
    err = np.linalg.norm(q_warm - q) / np.linalg.norm(q - X)
    assert err <= tol, err
    assert sum(it_warm) <= sum(it_cold), (it_warm, it_cold)
    print(f"precision {precision}: iterations cold {it_cold}, warm {it_warm}; error {err:.2e}")


@pytest.mark.parametrize("precision", [0, 1])
def test_warm_start_graph_equals_host_driven(gpu_lib, precision):
    wl = fi.workload("tet-mr", a=3, b=3, c=10)
    wl.precision = precision
    q0, v0, it0 = _rollout(gpu_lib, wl, 7, refactor_every=3, warm_start=1)
    q1, v1, it1 = _rollout(gpu_lib, wl, 7, refactor_every=3, warm_start=1, use_graph=1)
    assert it0 == it1
    np.testing.assert_array_equal(q0, q1)
    np.testing.assert_array_equal(v0, v1)


def test_set_state_resets_the_warm_start(gpu_lib):
    wl = fi.workload("tet-mr", a=3, b=3, c=10)
    ctx = gpu_lib.FEContext.from_workload(wl, refactor_every=1, warm_start=1)
    X = wl.mesh.X.reshape(-1).copy()
    out = []
    for _ in range(2):
        ctx.set_state(X, np.zeros_like(X))
        q = np.empty(ctx.n)
        for t in range(4):
            ctx.step(wl.p(t).reshape(-1), q, None)
        out.append(q.copy())
    np.testing.assert_array_equal(out[0], out[1])
    ctx.close()
