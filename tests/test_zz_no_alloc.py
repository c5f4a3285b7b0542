"""The allocation-free preconditioner application against the regular one.

fe_apply_preconditioner_noalloc serves callers that cannot call cudaMalloc
(a simulator's real-time loop, or a device whose memory another allocator
already holds): its work vectors live in a static device array instead of
context buffers.  It must give what fe_apply_preconditioner gives, on two
calls in a row (the array keeps the previous call's contents), in FP64 and
in the mixed path.  This file is collected last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest

import fe_inputs as fi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,fp16", [(0, 0), (1, 0), (1, 1)])
def test_noalloc_apply_matches_regular_apply(gpu_lib, precision, fp16):
    import torch
    fe = gpu_lib
    lib = fe.load()
    mesh = fi.tet_beam(3, 4, 9)
    ctx = fe.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.NEOHOOKE, 1000.0,
                       (3.4e3, 3.1e4, 0.0), 0.01, 0.1, 0.01, precision=precision, precond_fp16=fp16)
    rng = np.random.default_rng(11)
    q = mesh.X.reshape(-1) + 0.01 * 0.01 * rng.standard_normal(ctx.n)
    fixed = (3 * mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)
    q[fixed] = mesh.X.reshape(-1)[fixed]
    ctx.set_state(q, None)
    ctx.assemble(np.zeros(ctx.n))
    ctx.factor_now()
    stream = torch.cuda.current_stream()
    for call in range(2):
        r = rng.standard_normal(ctx.n)
        r[fixed] = 0.0
        z_ref = ctx.apply_preconditioner(r)
        r_d = torch.tensor(r, dtype=torch.float64, device="cuda")
        z_d = torch.full((ctx.n,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.fe_apply_preconditioner_noalloc(ctx.ctx, ct.c_void_p(r_d.data_ptr()),
                                                 ct.c_void_p(z_d.data_ptr()),
                                                 ct.c_void_p(stream.cuda_stream))
        torch.cuda.synchronize()
        assert st == 0, lib.fe_last_error(ctx.ctx)
        z = z_d.cpu().numpy()
        tol = 1e-12 if precision == 0 else 1e-6
        np.testing.assert_allclose(z, z_ref, rtol=0, atol=tol * np.abs(z_ref).max())
        assert np.all(z[fixed] == 0.0)
    ctx.close()


def test_noalloc_apply_needs_a_factor(gpu_lib):
    import torch
    fe = gpu_lib
    lib = fe.load()
    mesh = fi.tet_beam(2, 2, 3)
    ctx = fe.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.SVK, 1000.0,
                       (1e3, 1e4, 0.0), 0.01, 0.1, 0.01)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    st = lib.fe_apply_preconditioner_noalloc(ctx.ctx, ct.c_void_p(x.data_ptr()), ct.c_void_p(x.data_ptr()),
                                             None)
    assert st == 9
    ctx.close()


def _call_noalloc(lib, ctx, r_d, z_d, stream):
    return lib.fe_apply_preconditioner_noalloc(ctx.ctx, ct.c_void_p(r_d.data_ptr()), ct.c_void_p(z_d.data_ptr()),
                                               ct.c_void_p(stream.cuda_stream))


def test_noalloc_then_steps_back_to_back(gpu_lib):
    """The call runs on a caller's stream while the context's own steps (on
    the library's stream) follow at once, refactorising every second step
    into the factor buffer the call reads.  The call is ordered after the
    context's queued work and the steps after the call, so z and the states
    equal those of a reference context that does the same sequentially."""
    import torch
    fe = gpu_lib
    lib = fe.load()
    wl = fi.workload("tet-mr", a=3, b=4, c=9)
    kw = dict(precision=1, refactor_every=2, factor_lag=1, spmv_variant=4)
    ref = fe.FEContext.from_workload(wl, **kw)
    ctx = fe.FEContext.from_workload(wl, **kw)
    q_ref, q = np.empty(ref.n), np.empty(ctx.n)
    for c, qq in ((ref, q_ref), (ctx, q)):
        for t in range(2):
            c.step(wl.p(t).reshape(-1), qq, None)
    rng = np.random.default_rng(21)
    r = rng.standard_normal(ctx.n)
    r[(3 * wl.mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)] = 0.0
    z_ref = ref.apply_preconditioner(r)
    for t in range(2, 5):
        ref.step(wl.p(t).reshape(-1), q_ref, None)
    side = torch.cuda.Stream()
    r_d = torch.tensor(r, dtype=torch.float64, device="cuda")
    z_d = torch.full((ctx.n,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = _call_noalloc(lib, ctx, r_d, z_d, side)
    assert st == 0, lib.fe_last_error(ctx.ctx)
    for t in range(2, 5):                    # back to back, no synchronisation in between
        ctx.step(wl.p(t).reshape(-1), q, None)
    torch.cuda.synchronize()
    np.testing.assert_allclose(z_d.cpu().numpy(), z_ref, rtol=0, atol=1e-6 * np.abs(z_ref).max())
    assert np.array_equal(q, q_ref)
    ref.close()
    ctx.close()


def test_noalloc_wait_timeout_is_reported_by_the_next_step(gpu_lib):
    """A dependency wait of the call that runs out (a root front held with a
    pending child that nothing completes, dep_wait_s = 20 ms) leaves z
    incomplete; the context's next step reports FE_ERR_TIMEOUT naming the
    call, once, with the state unchanged, and the step after it runs
    normally."""
    import torch
    fe = gpu_lib
    lib = fe.load()
    wl = fi.workload("tet-mr", a=3, b=4, c=9)
    kw = dict(precision=1, refactor_every=1, dep_wait_s=0.02, spmv_variant=4)
    ref = fe.FEContext.from_workload(wl, **kw)
    ctx = fe.FEContext.from_workload(wl, **kw)
    q_ref, q = np.empty(ref.n), np.empty(ctx.n)
    for t in range(2):
        ref.step(wl.p(t).reshape(-1), q_ref, None)
    ctx.step(wl.p(0).reshape(-1), q, None)
    order = ctx.ordering()
    root = [f for f in np.nonzero(order["parent"] < 0)[0] if np.any(order["parent"] == f)][0]
    ctx.hold_front(int(root))
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    z = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    assert _call_noalloc(lib, ctx, x, z, torch.cuda.current_stream()) == 0
    torch.cuda.synchronize()
    q_before, _ = ctx.get_state()
    with pytest.raises(fe.FEError) as ei:
        ctx.step(wl.p(1).reshape(-1), q, None)
    assert ei.value.status == 8 and "noalloc" in str(ei.value)
    assert np.array_equal(ctx.get_state()[0], q_before)
    ctx.step(wl.p(1).reshape(-1), q, None)
    assert np.array_equal(q, q_ref)
    ref.close()
    ctx.close()
