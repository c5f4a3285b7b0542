"""GPU parity of the generic triplet ingestion (fe_trip_*) against the
oracle's triplets_to_csr: pattern, map C and merged values bit-exact (both
sum every slot in ascending stream order in FP64), the filling-order test
(pattern kept / rebuilt), host and device inputs, edge cases."""
import json
import os

import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _check(T, n, rows, cols, vals):
    _, rp, ci, C, v = O.triplets_to_csr(n, rows, cols, vals)
    grp, gci, gC = T.pattern()
    np.testing.assert_array_equal(grp, rp)
    np.testing.assert_array_equal(gci, ci)
    np.testing.assert_array_equal(gC, C)
    np.testing.assert_array_equal(T.values(), v)


def test_hand_example(gpu_lib):
    g = json.load(open(os.path.join(GOLDEN, "triplets_3x3.json")))
    T = gpu_lib.TripletAssembler(g["n"])
    assert T.assemble(np.array(g["rows"]), np.array(g["cols"]), np.array(g["vals"]))
    grp, gci, gC = T.pattern()
    assert grp.tolist() == g["rowptr"] and gci.tolist() == g["colind"] and gC.tolist() == g["C"]
    assert T.values().tolist() == g["values"]
    T.close()


def test_element_stream_keep_and_rebuild(gpu_lib):
    """A mesh's element tangents as an external stream, three steps: new
    values in the same order keep the pattern; a reordered stream rebuilds."""
    mesh = fi.hex_beam(3, 3, 7, jitter=0.1, seed=4)
    n = 3 * mesh.n_nodes
    row, col = O.triplet_dofs(mesh.conn)
    m = O.Model(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, O.NEOHOOKE, (3.4e3, 3.1e4, 0.0),
                1000.0, 0.01, 0.1, 0.01)
    rng = np.random.default_rng(1)
    T = gpu_lib.TripletAssembler(n)
    for step in range(3):
        q = mesh.X.reshape(-1) + 1e-3 * rng.standard_normal(n)
        vals = O.element_values_fill_order(m.element_tangent(q))
        rows, cols = row, col
        if step == 2:  # the caller's filling order changes (elements visited backwards)
            order = np.arange(row.size).reshape(mesh.n_elems, -1)[::-1].reshape(-1)
            rows, cols, vals = row[order], col[order], vals[order]
        rebuilt = T.assemble(rows, cols, vals)
        assert rebuilt == (step != 1)
        _check(T, n, rows, cols, vals)
    T.close()


def test_device_inputs(gpu_lib):
    import torch
    rng = np.random.default_rng(3)
    n, t = 300, 50_000
    rows = rng.integers(0, n, t).astype(np.int32)
    cols = rng.integers(0, n, t).astype(np.int32)
    T = gpu_lib.TripletAssembler(n)
    dr, dc = torch.tensor(rows, device="cuda"), torch.tensor(cols, device="cuda")
    for k in range(3):
        vals = rng.standard_normal(t)
        rebuilt = T.assemble(dr, dc, torch.tensor(vals, device="cuda"))
        torch.cuda.synchronize()
        assert rebuilt == (k == 0)
        _check(T, n, rows, cols, vals)
    # one index changed on the device: detected, rebuilt
    rows2 = rows.copy()
    rows2[t // 2] = (rows2[t // 2] + 1) % n
    vals = rng.standard_normal(t)
    assert T.assemble(torch.tensor(rows2, device="cuda"), dc, torch.tensor(vals, device="cuda"))
    torch.cuda.synchronize()
    _check(T, n, rows2, cols, vals)
    T.close()


def test_edge_cases(gpu_lib):
    T = gpu_lib.TripletAssembler(5)
    # empty stream
    assert T.assemble(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    rp, ci, C = T.pattern()
    assert rp.tolist() == [0] * 6 and ci.size == 0
    # a shorter or longer stream than the previous one rebuilds
    assert T.assemble(np.array([4, 0]), np.array([4, 0]), np.array([1.0, 2.0]))
    assert not T.assemble(np.array([4, 0]), np.array([4, 0]), np.array([3.0, 5.0]))
    assert T.assemble(np.array([4, 0, 4]), np.array([4, 0, 4]), np.array([1.0, 2.0, 3.0]))
    _check(T, 5, np.array([4, 0, 4]), np.array([4, 0, 4]), np.array([1.0, 2.0, 3.0]))
    # out-of-range index
    with pytest.raises(gpu_lib.FEError) as ei:
        T.assemble(np.array([5]), np.array([0]), np.array([1.0]))
    assert ei.value.status == 1
    T.close()
