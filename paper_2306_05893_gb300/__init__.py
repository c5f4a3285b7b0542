"""Python binding of the GB300 implicit-FE library (argument marshalling only).

Every numerical step runs in the CUDA library ``_build/libfe_hotpath.so``
(built by ``build.build()``); this module only converts numpy arrays / torch
tensors to pointers and status codes to exceptions.  There is no CPU path:
calls fail with ``FEError`` when the library or a GPU is missing.

The functions keep the C names (``fe_create``, ``fe_build_pattern``,
``fe_step`` ...); ``FEContext`` bundles them with the handle's lifetime.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import _abi
from ._abi import (FE_COROTATIONAL, FE_FP64, FE_HEX8, FE_MIXED, FE_MOONEY_RIVLIN, FE_NEOHOOKE,  # noqa: F401
                   FE_SVK, FE_TET4, FeOptions, FeStepInfo)

_LIB = None
_HERE = os.path.dirname(os.path.abspath(__file__))


class FEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_abi.STATUS.get(status, status)}: {msg}")
        self.status = status


def lib_path():
    return os.environ.get("FE_HOTPATH_LIB") or os.path.join(_HERE, "_build", "libfe_hotpath.so")


def load(path=None):
    """Load (once) and return the CUDA library; raises if it is not built."""
    global _LIB
    if _LIB is None:
        p = path or lib_path()
        if not os.path.exists(p):
            raise FEError(-1, f"CUDA library not built ({p}); call paper_2306_05893_gb300.build.build()")
        _LIB = _abi.bind(ct.CDLL(p))
    return _LIB


def _check(ctx, status):
    if status != 0:
        msg = _LIB.fe_last_error(ctx) if ctx else b""
        raise FEError(status, (msg or b"").decode())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    """Pointer of a numpy array (host) or a torch tensor (device or host)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ct.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ct.c_void_p)


def _arr(ptr, count, dtype):
    """Copy of a library-owned array; empty arrays may come with a NULL pointer."""
    count = int(count)
    if count == 0 or not ptr:
        if count:
            raise FEError(-1, "library returned a NULL pointer for a non-empty array")
        return np.zeros(0, dtype)
    return np.ctypeslib.as_array(ptr, (count,)).copy()


def _dptr(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def options(**kw) -> FeOptions:
    load()
    o = FeOptions()
    _LIB.fe_options_default(ct.byref(o))
    for k, v in kw.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream if hasattr(v, "cuda_stream") else int(v)
        setattr(o, k, v)
    return o


# ------------------------------------------------------------ C-named calls

def fe_create(elem_type, X, conn, fixed_nodes, model, rho, params, h, alpha, beta, opts=None):
    lib = load()
    X = _f64(X).reshape(-1, 3)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    fixed = np.ascontiguousarray(fixed_nodes, dtype=np.int32).reshape(-1)
    params = _f64(params)
    per_elem = 1 if params.ndim == 2 else 0
    mesh = _abi.FeMesh(elem_type, X.shape[0], conn.shape[0], _dptr(X),
                       conn.ctypes.data_as(ct.POINTER(ct.c_int32)), fixed.size,
                       fixed.ctypes.data_as(ct.POINTER(ct.c_int32)))
    mat = _abi.FeMaterial(model, float(rho), _dptr(params), per_elem)
    opts = opts if opts is not None else options()
    h_ctx = ct.c_void_p()
    st = lib.fe_create(ct.byref(mesh), ct.byref(mat), float(h), float(alpha), float(beta),
                       ct.byref(opts), ct.byref(h_ctx))
    if st != 0:
        raise FEError(st, "fe_create rejected its arguments")
    return h_ctx


def fe_create_batch(members, h, alpha, beta, rho, opts=None):
    """members: list of (elem_type, X, conn, fixed_nodes, model, params)."""
    lib = load()
    keep = []
    meshes = (_abi.FeMesh * len(members))()
    mats = (_abi.FeMaterial * len(members))()
    for k, (et, X, conn, fixed, model, params) in enumerate(members):
        X = _f64(X).reshape(-1, 3)
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        fixed = np.ascontiguousarray(fixed, dtype=np.int32).reshape(-1)
        params = _f64(params)
        keep += [X, conn, fixed, params]
        meshes[k] = _abi.FeMesh(et, X.shape[0], conn.shape[0], _dptr(X),
                                conn.ctypes.data_as(ct.POINTER(ct.c_int32)), fixed.size,
                                fixed.ctypes.data_as(ct.POINTER(ct.c_int32)))
        mats[k] = _abi.FeMaterial(model, float(rho), _dptr(params), 1 if params.ndim == 2 else 0)
    opts = opts if opts is not None else options()
    h_ctx = ct.c_void_p()
    st = lib.fe_create_batch(len(members), meshes, mats, float(h), float(alpha), float(beta),
                             ct.byref(opts), ct.byref(h_ctx))
    if st != 0:
        raise FEError(st, "fe_create_batch rejected its arguments")
    return h_ctx


def fe_get_batch_layout(ctx):
    nb = ct.c_int32()
    mem = ct.POINTER(ct.c_int32)()
    no, eo = ct.POINTER(ct.c_int64)(), ct.POINTER(ct.c_int64)()
    _check(ctx, load().fe_get_batch_layout(ctx, ct.byref(nb), ct.byref(mem), ct.byref(no), ct.byref(eo)))
    k = nb.value
    return (np.ctypeslib.as_array(mem, (k,)).copy(), np.ctypeslib.as_array(no, (k + 1,)).copy(),
            np.ctypeslib.as_array(eo, (k + 1,)).copy())


def fe_get_batch_stats(ctx, nb):
    it = np.zeros(nb, np.int32)
    rr = np.zeros(nb)
    _check(ctx, load().fe_get_batch_stats(ctx, it.ctypes.data_as(ct.POINTER(ct.c_int32)), _dptr(rr)))
    return it, rr


def fe_build_pattern(ctx):
    _check(ctx, load().fe_build_pattern(ctx))


def fe_get_pattern(ctx):
    n, nnz, nt = ct.c_int64(), ct.c_int64(), ct.c_int64()
    rp, ci, sc = (ct.POINTER(ct.c_int32)() for _ in range(3))
    _check(ctx, load().fe_get_pattern(ctx, ct.byref(n), ct.byref(nnz), ct.byref(rp), ct.byref(ci),
                                      ct.byref(nt), ct.byref(sc)))
    return (_arr(rp, n.value + 1, np.int32), _arr(ci, nnz.value, np.int32), _arr(sc, nt.value, np.int32))


def fe_get_inverse_map(ctx, nnz):
    sp_, ss = ct.POINTER(ct.c_int64)(), ct.POINTER(ct.c_int32)()
    _check(ctx, load().fe_get_inverse_map(ctx, ct.byref(sp_), ct.byref(ss)))
    slot_ptr = _arr(sp_, nnz + 1, np.int64)
    return slot_ptr, _arr(ss, int(slot_ptr[-1]), np.int32)


def fe_get_mass(ctx, nnz):
    mp = ct.POINTER(ct.c_double)()
    _check(ctx, load().fe_get_mass(ctx, ct.byref(mp)))
    return _arr(mp, nnz, np.float64)


def fe_get_ordering(ctx):
    nf, nfr = ct.c_int64(), ct.c_int64()
    ptrs = [ct.POINTER(ct.c_int32)() for _ in range(6)]
    _check(ctx, load().fe_get_ordering(ctx, ct.byref(nf), ct.byref(ptrs[0]), ct.byref(nfr),
                                       *[ct.byref(p) for p in ptrs[1:]]))
    perm = _arr(ptrs[0], nf.value, np.int32)
    fr = [_arr(p, nfr.value, np.int32) for p in ptrs[1:]]
    return dict(perm=perm, first=fr[0], npiv=fr[1], nupd=fr[2], parent=fr[3], level=fr[4])


def fe_get_front_rows(ctx, f):
    nu = ct.c_int64()
    rp = ct.POINTER(ct.c_int32)()
    _check(ctx, load().fe_get_front_rows(ctx, int(f), ct.byref(nu), ct.byref(rp)))
    return _arr(rp, nu.value, np.int32)


def fe_set_state(ctx, q=None, v=None):
    _check(ctx, load().fe_set_state(ctx, _ptr(q), _ptr(v)))


def fe_get_state(ctx, q=None, v=None):
    _check(ctx, load().fe_get_state(ctx, _ptr(q), _ptr(v)))


def fe_element_eval(ctx, q=None, f_e=None, K_e=None):
    _check(ctx, load().fe_element_eval(ctx, _ptr(q), _ptr(f_e), _ptr(K_e)))


def fe_assemble(ctx, p_ext=None, A_vals=None, b=None):
    _check(ctx, load().fe_assemble(ctx, _ptr(p_ext), _ptr(A_vals), _ptr(b)))


def fe_factor_now(ctx):
    _check(ctx, load().fe_factor_now(ctx))


def fe_apply_preconditioner(ctx, r, z):
    _check(ctx, load().fe_apply_preconditioner(ctx, _ptr(r), _ptr(z)))


def fe_set_contacts(ctx, nodes, normals, offsets):
    nodes = np.ascontiguousarray(nodes, dtype=np.int32).reshape(-1)
    normals = _f64(normals).reshape(-1)
    offsets = _f64(offsets).reshape(-1)
    m = nodes.size
    if normals.size != 3 * m or offsets.size != m:
        raise ValueError("nodes [m], normals [m, 3] and offsets [m] disagree")
    _check(ctx, load().fe_set_contacts(ctx, m, _ptr(nodes), _ptr(normals), _ptr(offsets)))


def fe_get_contact_forces(ctx, m):
    lam = np.zeros(m)
    if m:
        _check(ctx, load().fe_get_contact_forces(ctx, _ptr(lam)))
    return lam


def fe_step(ctx, p_ext=None, q_out=None, v_out=None):
    info = FeStepInfo()
    st = load().fe_step(ctx, _ptr(p_ext), _ptr(q_out), _ptr(v_out), ct.byref(info))
    _check(ctx, st)
    return info


def fe_get_info(ctx):
    info = _abi.FeInfo()
    _check(ctx, load().fe_get_info(ctx, ct.byref(info)))
    return {k: getattr(info, k) for k, _ in info._fields_}


def fe_get_stage_times(ctx):
    ms = (ct.c_double * len(_abi.STAGES))()
    calls = (ct.c_int64 * len(_abi.STAGES))()
    launches = ct.c_int64()
    _check(ctx, load().fe_get_stage_times(ctx, ms, calls, ct.byref(launches)))
    return ({k: ms[i] for i, k in enumerate(_abi.STAGES)},
            {k: calls[i] for i, k in enumerate(_abi.STAGES)}, launches.value)


def fe_get_update_flops(ctx):
    f = ct.c_double()
    _check(ctx, load().fe_get_update_flops(ctx, ct.byref(f)))
    return f.value


def fe_get_update_bf16_flops(ctx):
    f = ct.c_double()
    _check(ctx, load().fe_get_update_bf16_flops(ctx, ct.byref(f)))
    return f.value


def fe_get_update_bf16_tiles(ctx):
    t = ct.c_int64()
    _check(ctx, load().fe_get_update_bf16_tiles(ctx, ct.byref(t)))
    return t.value


def fe_reset_stage_times(ctx):
    _check(ctx, load().fe_reset_stage_times(ctx))


def fe_set_params(ctx, params):
    _check(ctx, load().fe_set_params(ctx, _ptr(_f64(params))))


def fe_adjoint(ctx, dL_dqT, dL_dvT=None, dL_ds=None, dL_dp=None):
    _check(ctx, load().fe_adjoint(ctx, _ptr(dL_dqT), _ptr(dL_dvT), _ptr(dL_ds), _ptr(dL_dp)))


def fe_clear_checkpoints(ctx):
    _check(ctx, load().fe_clear_checkpoints(ctx))


def fe_num_checkpoints(ctx):
    k = ct.c_int64()
    _check(ctx, load().fe_num_checkpoints(ctx, ct.byref(k)))
    return k.value


def fe_debug_hold_front(ctx, front, extra=1):
    _check(ctx, load().fe_debug_hold_front(ctx, int(front), int(extra)))


def fe_destroy(ctx):
    if ctx:
        load().fe_destroy(ctx)


# ------------------------------------------------- generic triplet ingestion

def _check_trip(t, status):
    if status != 0:
        msg = _LIB.fe_trip_last_error(t) if t else b""
        raise FEError(status, (msg or b"").decode())


def fe_trip_create(n):
    lib = load()
    h = ct.c_void_p()
    st = lib.fe_trip_create(int(n), ct.byref(h))
    if st:
        raise FEError(st, "fe_trip_create failed")
    return h


def fe_trip_assemble(t, rows, cols, vals, stream=None):
    """rows/cols int32 and vals float64, all numpy (host) or all CUDA tensors
    (device, on `stream`).  Returns True when the pattern was rebuilt."""
    dev = hasattr(vals, "data_ptr") and getattr(vals, "is_cuda", False)
    if not dev:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        vals = _f64(vals)
    s = None if stream is None else ct.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    rebuilt = ct.c_int32()
    _check_trip(t, load().fe_trip_assemble(t, int(rows.shape[0]), _ptr(rows), _ptr(cols), _ptr(vals),
                                           1 if dev else 0, s, ct.byref(rebuilt)))
    return bool(rebuilt.value)


def fe_trip_pattern(t, n):
    nnz = ct.c_int64()
    rp, ci, C = (ct.POINTER(ct.c_int32)() for _ in range(3))
    _check_trip(t, load().fe_trip_pattern(t, ct.byref(nnz), ct.byref(rp), ct.byref(ci), ct.byref(C)))
    return (np.ctypeslib.as_array(rp, (n + 1,)).copy(),
            np.ctypeslib.as_array(ci, (nnz.value,)).copy() if nnz.value else np.zeros(0, np.int32),
            nnz.value, C)


def fe_trip_values(t, nnz):
    out = np.empty(nnz, dtype=np.float64)
    if nnz:
        _check_trip(t, load().fe_trip_values(t, _ptr(out), 0, None))
    return out


class TripletAssembler:
    """Owns one fe_trip: merges a caller's (row, col, value) stream into an
    n x n CSR matrix on the GPU, keeping the pattern while the filling order
    is unchanged."""

    def __init__(self, n):
        self.n = int(n)
        self.t = fe_trip_create(self.n)
        self.ntrip = 0

    def assemble(self, rows, cols, vals, stream=None):
        self.ntrip = int(rows.shape[0])
        return fe_trip_assemble(self.t, rows, cols, vals, stream)

    def pattern(self):
        rp, ci, nnz, C = fe_trip_pattern(self.t, self.n)
        return rp, ci, (np.ctypeslib.as_array(C, (self.ntrip,)).copy() if self.ntrip else np.zeros(0, np.int32))

    def values(self):
        rp, _, nnz, _ = fe_trip_pattern(self.t, self.n)
        return fe_trip_values(self.t, nnz)

    def close(self):
        if self.t:
            load().fe_trip_destroy(self.t)
            self.t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- wrapper

class FEContext:
    """Owns one fe_ctx.  Host numpy arrays or (device_ptrs=1) CUDA tensors."""

    def __init__(self, elem_type, X, conn, fixed_nodes, model, rho, params, h, alpha, beta,
                 build=True, **opts):
        self.n = 3 * np.asarray(X).reshape(-1, 3).shape[0]
        self.n_elems = np.asarray(conn).shape[0]
        self.npe = np.asarray(conn).shape[1]
        self.opts = options(**opts)
        self.ctx = fe_create(elem_type, X, conn, fixed_nodes, model, rho, params, h, alpha, beta,
                             self.opts)
        if build:
            fe_build_pattern(self.ctx)
            self.rowptr, self.colind, self.C = fe_get_pattern(self.ctx)
            self.nnz = self.colind.size

    @classmethod
    def from_workload(cls, wl, params=None, **opts):
        m = wl.mesh
        kw = dict(precision=wl.precision, tol=wl.tol, refactor_every=wl.refactor_every)
        kw.update(opts)
        return cls(m.elem_type, m.X, m.conn, m.fixed_nodes, wl.model, wl.rho,
                   wl.params if params is None else params, wl.h, wl.alpha, wl.beta, **kw)

    def close(self):
        if self.ctx:
            fe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # convenience host-side helpers (copies)
    def inverse_map(self):
        return fe_get_inverse_map(self.ctx, self.nnz)

    def mass(self):
        return fe_get_mass(self.ctx, self.nnz)

    def ordering(self):
        return fe_get_ordering(self.ctx)

    def info(self):
        return fe_get_info(self.ctx)

    def stage_times(self):
        return fe_get_stage_times(self.ctx)

    def update_flops(self):
        return fe_get_update_flops(self.ctx)

    def update_bf16_flops(self):
        return fe_get_update_bf16_flops(self.ctx)

    def update_bf16_tiles(self):
        return fe_get_update_bf16_tiles(self.ctx)

    def reset_stage_times(self):
        fe_reset_stage_times(self.ctx)

    def set_params(self, params):
        fe_set_params(self.ctx, np.asarray(params, dtype=np.float64).reshape(-1, 3))

    def clear_checkpoints(self):
        fe_clear_checkpoints(self.ctx)

    def adjoint(self, dL_dqT, dL_dvT=None, with_dp=True):
        """Host arrays: returns (dL/ds [n_elems], dL/dp [T, n] or None)."""
        T = fe_num_checkpoints(self.ctx)
        ds = np.empty(self.n_elems)
        dp = np.empty((T, self.n)) if with_dp else None
        fe_adjoint(self.ctx, _f64(dL_dqT), None if dL_dvT is None else _f64(dL_dvT), ds, dp)
        return ds, dp

    def set_state(self, q=None, v=None):
        fe_set_state(self.ctx, q, v)

    def get_state(self):
        q = np.empty(self.n)
        v = np.empty(self.n)
        fe_get_state(self.ctx, q, v)
        return q, v

    def element_eval(self, q=None):
        m = 3 * self.npe
        f = np.empty(self.n_elems * m)
        K = np.empty(self.n_elems * m * m)
        fe_element_eval(self.ctx, None if q is None else _f64(q), f, K)
        return f.reshape(self.n_elems, m), K

    def assemble(self, p=None):
        A = np.empty(self.nnz)
        b = np.empty(self.n)
        fe_assemble(self.ctx, None if p is None else _f64(p), A, b)
        return A, b

    def factor_now(self):
        fe_factor_now(self.ctx)

    def hold_front(self, front, extra=1):
        """Test hook (fe_debug_hold_front): the next application waits on
        front `front` until fe_options.dep_wait_s runs out."""
        fe_debug_hold_front(self.ctx, front, extra)

    def apply_preconditioner(self, r):
        z = np.empty(self.n)
        fe_apply_preconditioner(self.ctx, _f64(r), z)
        return z

    def set_contacts(self, nodes, normals, offsets):
        """Frictionless contacts against rigid planes n . x >= c for the
        following steps (fe_set_contacts); empty arrays remove them."""
        fe_set_contacts(self.ctx, nodes, normals, offsets)
        self.n_contacts = int(np.asarray(nodes).size)

    def contact_forces(self):
        """Multipliers of the last step with contacts (fe_get_contact_forces)."""
        return fe_get_contact_forces(self.ctx, getattr(self, "n_contacts", 0))

    def step(self, p=None, q_out=None, v_out=None):
        p_arg = p if (p is None or hasattr(p, "data_ptr")) else _f64(p)
        return fe_step(self.ctx, p_arg, q_out, v_out)


class FEBatch(FEContext):
    """Independent meshes stepped together (fe_create_batch).  State and force
    vectors are concatenations in the stored member order (grouped by
    material model); `member`, `node_off` give that order and the offsets."""

    def __init__(self, members, h, alpha, beta, rho, build=True, **opts):
        self.n = 3 * sum(np.asarray(m[1]).reshape(-1, 3).shape[0] for m in members)
        self.n_elems = sum(np.asarray(m[2]).shape[0] for m in members)
        self.npe = np.asarray(members[0][2]).shape[1]
        self.opts = options(**opts)
        self.ctx = fe_create_batch(members, h, alpha, beta, rho, self.opts)
        self.member, self.node_off, self.elem_off = fe_get_batch_layout(self.ctx)
        self.nb = len(members)
        if build:
            fe_build_pattern(self.ctx)
            self.rowptr, self.colind, self.C = fe_get_pattern(self.ctx)
            self.nnz = self.colind.size

    def concat(self, per_member):
        """Concatenate per-member [n_k] (or [n_nodes_k, 3]) arrays in stored order."""
        return np.concatenate([np.asarray(per_member[k], dtype=np.float64).reshape(-1) for k in self.member])

    def split(self, vec):
        """Inverse of concat: list of per-member arrays in the caller's order."""
        out = [None] * self.nb
        for s, k in enumerate(self.member):
            out[k] = vec[3 * self.node_off[s]:3 * self.node_off[s + 1]]
        return out

    def stats(self):
        return fe_get_batch_stats(self.ctx, self.nb)
