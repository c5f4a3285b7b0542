"""CPU tests of the C-ABI library: symbols, and the host setup (Section 4.2
pattern + map C, as two transposes of the triplet stream define them; Section
5.1 constraints, Section 6.1
nested dissection and multifrontal structure) against the oracle."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fe():
    from paper_2306_05893_gb300 import build
    build.build()
    import paper_2306_05893_gb300 as fe
    fe.load()
    return fe


def test_library_exports_every_declared_symbol(fe):
    header = open(os.path.join(ROOT, "include", "fe_hotpath.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char \*)\s*(fe_\w+)\s*\(", header, re.M))
    assert {"fe_create", "fe_step", "fe_build_pattern", "fe_destroy"} <= declared
    lib = ct.CDLL(fe.lib_path())
    for name in sorted(declared):
        assert hasattr(lib, name), name
    from paper_2306_05893_gb300 import _abi
    assert declared == set(_abi.SIGNATURES), declared ^ set(_abi.SIGNATURES)


def test_create_rejects_bad_input(fe):
    mesh = fi.tet_beam(1, 1, 1)
    conn = mesh.conn.copy()
    conn[0, 0] = 10_000
    with pytest.raises(fe.FEError):
        fe.fe_create(0, mesh.X, conn, mesh.fixed_nodes, 0, 1000.0, [1.0, 1.0, 0.0], 0.01, 0.1, 0.01)
    with pytest.raises(fe.FEError):
        fe.fe_create(0, mesh.X, mesh.conn, mesh.fixed_nodes, 0, 1000.0, [1.0, 1.0, 0.0], -1.0, 0.1, 0.01)
    # the adjoint differentiates the single-linearisation step only
    with pytest.raises(fe.FEError) as ei:
        fe.fe_create(0, mesh.X, mesh.conn, mesh.fixed_nodes, 0, 1000.0, [1.0, 1.0, 0.0], 0.01, 0.1, 0.01,
                     fe.options(newton_iters=3, keep_checkpoints=1))
    assert ei.value.status == 1


def test_create_rejects_non_finite_and_negative_damping(fe):
    mesh = fi.tet_beam(1, 1, 1)
    args = (0, mesh.X, mesh.conn, mesh.fixed_nodes, 0, 1000.0, [1.0, 1.0, 0.0])
    for h, al, be in [(np.inf, 0.1, 0.01), (0.01, -0.1, 0.01), (0.01, 0.1, -1e-3), (0.01, np.nan, 0.01),
                      (0.01, 0.1, np.inf)]:
        with pytest.raises(fe.FEError) as ei:
            fe.fe_create(*args, h, al, be)
        assert ei.value.status == 1
    X = mesh.X.copy()
    X[3, 1] = np.nan
    with pytest.raises(fe.FEError):
        fe.fe_create(0, X, mesh.conn, mesh.fixed_nodes, 0, 1000.0, [1.0, 1.0, 0.0], 0.01, 0.1, 0.01)
    with pytest.raises(fe.FEError):
        fe.fe_create(0, mesh.X, mesh.conn, mesh.fixed_nodes, 0, 1000.0, [1.0, np.inf, 0.0], 0.01, 0.1, 0.01)
    with pytest.raises(fe.FEError):
        fe.fe_create(0, mesh.X, mesh.conn, mesh.fixed_nodes, 0, np.inf, [1.0, 1.0, 0.0], 0.01, 0.1, 0.01)
    # zero damping is a valid Rayleigh model
    ctx = fe.fe_create(0, mesh.X, mesh.conn, mesh.fixed_nodes, 0, 1000.0, [1.0, 1.0, 0.0], 0.01, 0.0, 0.0)
    fe.fe_destroy(ctx)


def _ctx(fe, mesh, **kw):
    return fe.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, 0, 1000.0,
                        [1e3, 1e4, 0.0], 0.01, 0.1, 0.01, **kw)


MESHES = {
    "tet-2x3x4": lambda: fi.tet_beam(2, 3, 4),
    "tet-4x4x16": lambda: fi.tet_beam(4, 4, 16),
    "hex-2x3x4-jitter": lambda: fi.hex_beam(2, 3, 4, jitter=0.1),
    "hex-3x3x7": lambda: fi.hex_beam(3, 3, 7),
    "tet-1x1x1-nofix": lambda: fi.TetBeam(1, 1, 1, fi.tet_beam(1, 1, 1).X, fi.tet_beam(1, 1, 1).conn,
                                          np.zeros(0, np.int32)),
    # element order shuffled (row segments then hold triplets from scattered elements)
    "tet-3x3x5-shuffled": lambda: _replace(fi.tet_beam(3, 3, 5), conn=_shuffled(fi.tet_beam(3, 3, 5).conn)),
    # fixed nodes inside the mesh, not on one face
    "hex-2x3x4-interior-fix": lambda: _replace(fi.hex_beam(2, 3, 4, jitter=0.1),
                                               fixed_nodes=np.array([0, 7, 19, 30, 41], np.int32)),
    # every node fixed: the pattern is the identity, no triplet is kept
    "tet-2x2x3-all-fixed": lambda: _replace(fi.tet_beam(2, 2, 3),
                                            fixed_nodes=np.arange(3 * 3 * 4, dtype=np.int32)),
}


def _replace(mesh, **kw):
    import dataclasses
    return dataclasses.replace(mesh, **kw)


def _shuffled(conn, seed=5):
    return conn[np.random.default_rng(seed).permutation(conn.shape[0])].copy()


@pytest.mark.parametrize("name", list(MESHES))
def test_pattern_and_map_bit_exact(fe, name):
    mesh = MESHES[name]()
    ctx = _ctx(fe, mesh)
    n = 3 * mesh.n_nodes
    fixed = (3 * mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)
    rp, ci, C = O.csr_pattern(n, mesh.conn, fixed)
    np.testing.assert_array_equal(ctx.rowptr, rp)
    np.testing.assert_array_equal(ctx.colind, ci)
    np.testing.assert_array_equal(ctx.C, C)
    # inverse map: every kept triplet once, slots ascending, ids ascending in a slot
    slot_ptr, slot_src = ctx.inverse_map()
    kept = np.nonzero(C >= 0)[0]
    assert slot_src.size == kept.size
    np.testing.assert_array_equal(np.sort(slot_src), kept)
    for s in range(0, ctx.nnz, max(1, ctx.nnz // 200)):
        seg = slot_src[slot_ptr[s]:slot_ptr[s + 1]]
        assert np.all(C[seg] == s)
        assert np.all(np.diff(seg) > 0)
    ctx.close()


def test_setup_products_do_not_depend_on_host_threads(fe, monkeypatch):
    """The pattern, C, its inverse and the mass are built on several host
    threads with output ranges fixed beforehand: 1, 3 and all threads give
    the same arrays bit for bit."""
    base = fi.tet_beam(8, 8, 24)  # 2,025 nodes: every parallel phase takes several chunks
    mesh = _replace(base, conn=_shuffled(base.conn))
    outs = []
    for nt in ("1", "3", None):
        if nt is None:
            monkeypatch.delenv("FE_HOST_THREADS", raising=False)
        else:
            monkeypatch.setenv("FE_HOST_THREADS", nt)
        ctx = _ctx(fe, mesh)
        sp_, ss = ctx.inverse_map()
        outs.append((ctx.rowptr, ctx.colind, ctx.C, sp_, ss, ctx.mass()))
        ctx.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert a.dtype == b.dtype and np.array_equal(a, b)


def test_set_state_checks_host_arrays_before_device_work(fe):
    mesh = fi.tet_beam(1, 1, 2)
    ctx = _ctx(fe, mesh)
    q = mesh.X.reshape(-1).copy()
    v = np.zeros_like(q)
    bad_q = q.copy()
    bad_q[7] = np.nan
    bad_v = v.copy()
    bad_v[-1] = np.inf
    moving_fixed = v.copy()
    moving_fixed[3 * int(mesh.fixed_nodes[0])] = 1e-3
    for qq, vv in [(bad_q, None), (None, bad_v), (q, moving_fixed)]:
        with pytest.raises(fe.FEError) as ei:
            ctx.set_state(qq, vv)
        assert ei.value.status == 1  # FE_ERR_ARG, decided on the host
    ctx.close()


def test_all_fixed_pattern_is_the_identity(fe):
    mesh = MESHES["tet-2x2x3-all-fixed"]()
    ctx = _ctx(fe, mesh)
    n = 3 * mesh.n_nodes
    np.testing.assert_array_equal(ctx.rowptr, np.arange(n + 1))
    np.testing.assert_array_equal(ctx.colind, np.arange(n))
    assert np.all(ctx.C == -1)
    slot_ptr, slot_src = ctx.inverse_map()
    assert slot_src.size == 0 and np.all(slot_ptr == 0)
    ctx.close()


def test_free_node_outside_every_element_is_rejected(fe):
    mesh = fi.tet_beam(1, 1, 2)
    X = np.vstack([mesh.X, [[1.0, 1.0, 1.0]]])  # an extra node no element uses
    with pytest.raises(fe.FEError) as ei:
        fe.FEContext(mesh.elem_type, X, mesh.conn, mesh.fixed_nodes, 0, 1000.0, [1e3, 1e4, 0.0],
                     0.01, 0.1, 0.01)
    assert ei.value.status == 1 and "belongs to no element" in str(ei.value)
    # fixed, the same node is accepted (its row is a lone diagonal)
    fixed = np.append(mesh.fixed_nodes, mesh.n_nodes).astype(np.int32)
    ctx = fe.FEContext(mesh.elem_type, X, mesh.conn, fixed, 0, 1000.0, [1e3, 1e4, 0.0], 0.01, 0.1, 0.01)
    r = 3 * mesh.n_nodes
    assert list(ctx.colind[ctx.rowptr[r]:ctx.rowptr[r + 3]]) == [r, r + 1, r + 2]
    ctx.close()


@pytest.mark.parametrize("name", ["tet-2x3x4", "hex-2x3x4-jitter"])
def test_mass_on_pattern(fe, name):
    mesh = MESHES[name]()
    ctx = _ctx(fe, mesh)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, 0, (1, 1, 0), 1000.0, .01, .1, .01)
    fixed = m.fixed_dofs
    Mp = O.project(m.M, fixed)
    expect = O.values_in_pattern(Mp, ctx.rowptr, ctx.colind)
    fixed_rows = np.zeros(ctx.n, bool)
    fixed_rows[fixed] = True
    slot_row = np.repeat(np.arange(ctx.n), np.diff(ctx.rowptr))
    expect[fixed_rows[slot_row]] = 0.0   # the library keeps 0 mass on projected rows
    np.testing.assert_allclose(ctx.mass(), expect, rtol=1e-13, atol=1e-18)
    ctx.close()


@pytest.mark.parametrize("name,leaf", [("tet-4x4x16", 8), ("tet-4x4x16", 64), ("hex-3x3x7", 4),
                                       ("hex-2x3x4-jitter", 6)])
def test_nested_dissection_structure(fe, name, leaf):
    """perm is a permutation of the free DOFs; fronts are contiguous pivot
    blocks in postorder; every A entry couples a front with itself or with
    an ancestor (the separator property of Eq. "regional problem"), and lies
    in the column front's pivot or update rows."""
    mesh = MESHES[name]()
    ctx = _ctx(fe, mesh, nd_leaf_nodes=leaf)
    o = ctx.ordering()
    perm, first, npiv, parent, level = o["perm"], o["first"], o["npiv"], o["parent"], o["level"]
    n = ctx.n
    fixed = np.zeros(n, bool)
    fixed[(3 * mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)] = True
    np.testing.assert_array_equal(np.sort(perm), np.nonzero(~fixed)[0])
    nf = first.size
    assert first[0] == 0 and np.all(first[1:] == first[:-1] + npiv[:-1])
    assert first[-1] + npiv[-1] == perm.size
    for f in range(nf):
        if parent[f] >= 0:
            assert parent[f] > f and level[parent[f]] > level[f]
    iperm = -np.ones(n, np.int64)
    iperm[perm] = np.arange(perm.size)
    front_of = np.repeat(np.arange(nf), npiv)
    anc = [set() for _ in range(nf)]
    for f in range(nf - 1, -1, -1):
        p = parent[f]
        anc[f] = {f} | (anc[p] if p >= 0 else set())
    rows_of = [set(ctx_rows.tolist()) for ctx_rows in (fe.fe_get_front_rows(ctx.ctx, f) for f in range(nf))]
    slot_row = np.repeat(np.arange(n), np.diff(ctx.rowptr))
    for s in range(ctx.nnz):
        i, j = slot_row[s], ctx.colind[s]
        if fixed[i] or fixed[j]:
            continue
        fi_, fj = front_of[iperm[i]], front_of[iperm[j]]
        assert fi_ in anc[fj] or fj in anc[fi_]
        if iperm[i] > iperm[j] and fi_ != fj:       # lower entry outside the pivot block
            assert i in rows_of[fj]
    ctx.close()


def test_device_calls_fail_loudly_without_gpu(fe):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    mesh = fi.tet_beam(1, 1, 2)
    ctx = _ctx(fe, mesh)
    with pytest.raises(fe.FEError) as ei:
        ctx.step(np.zeros(ctx.n))
    assert ei.value.status == 2
    ctx.close()


def test_contact_arguments_checked_on_the_host(fe):
    """fe_set_contacts validates on the host (no device needed): node range,
    zero normals, non-finite offsets, the contact count limit, and the
    combinations the contact step does not cover (checkpoints, Newton)."""
    mesh = fi.tet_beam(1, 1, 2)
    ctx = _ctx(fe, mesh)
    ok_nodes, ok_normals, ok_offsets = [mesh.n_nodes - 1], [[0.0, 0.0, 1.0]], [-0.01]
    ctx.set_contacts(ok_nodes, ok_normals, ok_offsets)
    for nodes, normals, offsets in (([mesh.n_nodes], ok_normals, ok_offsets),
                                    ([-1], ok_normals, ok_offsets),
                                    (ok_nodes, [[0.0, 0.0, 0.0]], ok_offsets),
                                    (ok_nodes, ok_normals, [float("nan")])):
        with pytest.raises(fe.FEError) as ei:
            ctx.set_contacts(nodes, normals, offsets)
        assert ei.value.status == 1
    many = np.zeros(4097, np.int32)
    with pytest.raises(fe.FEError):
        ctx.set_contacts(many, np.tile([0.0, 0.0, 1.0], (4097, 1)), np.zeros(4097))
    ctx.set_contacts(np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros(0))  # removing them is fine
    ctx.close()
    for kw in ({"keep_checkpoints": 1}, {"newton_iters": 2}):
        c2 = _ctx(fe, mesh, **kw)
        with pytest.raises(fe.FEError) as ei:
            c2.set_contacts(ok_nodes, ok_normals, ok_offsets)
        assert ei.value.status == 9
        c2.close()


def test_contact_option_defaults(fe):
    o = fe.options()
    assert o.contact_sweeps == 200 and o.contact_tol == 1e-12
    assert o.precond_fp16 == 0 and o.factor_tf32 == 0


def test_schedule_and_wait_option_defaults(fe):
    o = fe.options()
    assert o.factor_lag == 1 and o.dep_wait_s == 1.0 and o.element_fp64 == 0
    assert o.warm_start == 0 and o.spmv_variant == -1
    assert o.apply_sm_share == 0.0 and o.update_bf16 == 1


def test_spmv_variant_is_checked_on_the_host(fe):
    mesh = fi.tet_beam(1, 1, 2)
    for v in (-1, 0, 3, 5):
        _ctx(fe, mesh, spmv_variant=v).close()
    for v in (-2, 6):
        with pytest.raises(fe.FEError) as ei:
            _ctx(fe, mesh, spmv_variant=v)
        assert ei.value.status == 1


def test_factor_lag_is_checked_on_the_host(fe):
    """The lag k of the asynchronous factor (Eq. "asynchronous
    preconditioner") must not exceed R: two factor buffers hold the factor in
    use and the one being made, so the next snapshot must come after the
    swap."""
    mesh = fi.tet_beam(1, 1, 2)
    for R, k in ((5, 5), (5, 1), (3, 2), (1, 7)):       # k is ignored for R = 1
        _ctx(fe, mesh, refactor_every=R, factor_lag=k).close()
    with pytest.raises(fe.FEError) as ei:
        _ctx(fe, mesh, refactor_every=3, factor_lag=4)
    assert ei.value.status == 1


def _apply_work_bytes(info, ts, fwd_parts, bwd_parts, tickets):
    """The allocation-free call's work vectors, each rounded up to 256 bytes:
    input and output [n], update vectors [sum of update rows], permuted pivot
    vector [n_free], split-task partial sums and tickets."""
    r = lambda b: (b + 255) // 256 * 256
    return 2 * r(info["n"] * ts) + r(info["u_total"] * ts) + r(info["n_free"] * ts) + \
        r(fwd_parts * ts) + r(bwd_parts * ts) + r(tickets * 4)


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_scratch_size(fe, precision):
    """fe_info.noalloc_bytes covers the regular application's work vectors:
    at least the vectors whose sizes the setup fixes (n, the fronts' update
    rows, the free DOFs), at most those plus the split tasks' partial sums
    (bounded by one 256-row block per forward task and one 32-column block per
    backward task, the tasks counted at their finest sizes: 64 forward pivot
    columns and 64 rows, 256 backward rows); FP64 needs about twice the mixed
    path's bytes."""
    mesh = fi.tet_beam(6, 6, 24)
    ctx = _ctx(fe, mesh, precision=precision)
    info = ctx.info()
    order = ctx.ordering()
    info["u_total"] = int(order["nupd"].sum())
    ts = 8 if precision == 0 else 4
    lo = _apply_work_bytes(info, ts, 1, 1, 1)
    n_fwd = sum(int(np.ceil(m / 64.0)) * int(np.ceil(p / 64.0)) for m, p in
                zip(order["npiv"] + order["nupd"], order["npiv"]))
    n_bwd = sum(int(np.ceil(m / 256.0)) * int(np.ceil(p / 32.0)) for m, p in
                zip(order["npiv"] + order["nupd"], order["npiv"]))
    hi = _apply_work_bytes(info, ts, 256 * n_fwd, 32 * n_bwd, n_fwd + n_bwd)
    assert lo <= info["noalloc_bytes"] <= hi, (lo, info["noalloc_bytes"], hi)
    ctx.close()


def test_noalloc_rejects_oversize_mesh_on_the_host(fe):
    """A mesh whose work vectors exceed the 64 MiB array (an FP64 beam of
    660,633 DOF needs about 70 MiB) is refused with FE_ERR_ARG before any GPU
    work, so the check runs here without a device; a small mesh passes the
    size check and is refused only for the missing factor (FE_ERR_STATE)."""
    lib = fe.load()
    big = fi.tet_beam(40, 40, 130)
    ctx = _ctx(fe, big)
    assert ctx.info()["noalloc_bytes"] > 64 * 2 ** 20
    dummy = ct.c_void_p(16)      # never dereferenced: the call stops at the size check
    st = lib.fe_apply_preconditioner_noalloc(ctx.ctx, dummy, dummy, None)
    assert st == 1
    assert b"bytes of scratch" in lib.fe_last_error(ctx.ctx)
    ctx.close()
    small = _ctx(fe, fi.tet_beam(1, 1, 2))
    assert 0 < small.info()["noalloc_bytes"] <= 64 * 2 ** 20
    assert lib.fe_apply_preconditioner_noalloc(small.ctx, dummy, dummy, None) == 9
    small.close()


def test_noalloc_scratch_size_and_over_size_refusal(fe):
    """The allocation-free application's scratch (fe_info.noalloc_bytes) holds
    at least the two work vectors of length n, the update vectors (the sum of
    the fronts' update rows) and the permuted pivot vector, each 256-byte
    aligned, at 8 bytes per value in FP64 and 4 in the mixed path.  A mesh
    whose scratch exceeds the library's 64 MiB array is refused with
    FE_ERR_ARG before any device work, so the call runs on a host without a
    GPU (the pointers are never dereferenced)."""
    mesh = fi.tet_beam(10, 10, 40)
    sizes = {}
    for prec, ts in ((0, 8), (1, 4)):
        ctx = _ctx(fe, mesh, precision=prec)
        o = ctx.ordering()
        need = ctx.info()["noalloc_bytes"]
        low = (2 * ctx.n + int(np.sum(o["nupd"])) + int(np.sum(o["npiv"]))) * ts
        assert need % 256 == 0 and need >= low
        sizes[prec] = need
        ctx.close()
    # the same layout at half the value size (the task tickets are 4-byte ints in both)
    assert sizes[1] < sizes[0] <= 2 * sizes[1]

    big = fi.tet_beam(40, 40, 160)  # 811,923 DOF: about 92 MiB of scratch in FP64
    ctx = _ctx(fe, big, precision=0)
    need = ctx.info()["noalloc_bytes"]
    assert need > 64 << 20
    dummy = (ct.c_double * 1)()
    st = fe.load().fe_apply_preconditioner_noalloc(ctx.ctx, ct.cast(dummy, ct.c_void_p), ct.cast(dummy, ct.c_void_p),
                                                   None)
    assert st == 1  # FE_ERR_ARG
    msg = fe.load().fe_last_error(ctx.ctx).decode()
    assert str(need) in msg and str(64 << 20) in msg
    ctx.close()
