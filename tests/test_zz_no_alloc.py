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
