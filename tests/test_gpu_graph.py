"""PCG iterations replayed as CUDA graphs (fe_options.use_graph): iterations
enqueued past convergence exit at once, so a rollout is bit-identical to the
one with a host check after every iteration, and the iteration cap is still
reported."""
import numpy as np
import pytest

import fe_inputs as fi

pytestmark = pytest.mark.gpu


def _rollout(fe, wl, steps, **kw):
    ctx = fe.FEContext.from_workload(wl, **kw)
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


def test_graph_replay_reports_the_iteration_cap(gpu_lib):
    wl = fi.workload("tet4x4x16-svk-fp64")
    ctx = gpu_lib.FEContext.from_workload(wl, precision=0, max_iters=2, refactor_every=100, tol=1e-14,
                                          use_graph=1)
    ctx.step(wl.p(0).reshape(-1))  # step 0: exact factor, converges at once
    with pytest.raises(gpu_lib.FEError) as ei:
        for t in range(1, 6):
            ctx.step(wl.p(t).reshape(-1))
    assert ei.value.status == 5
    ctx.close()
