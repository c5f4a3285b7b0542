"""Pins of the oracle's compression of a caller's triplet stream (Section 4.2,
"Collect data" / "Build matrix pattern"): the hand example of
tests/golden/triplets_3x3.json, the library routine scipy coo -> csr, the
element stream against the element pattern, and the filling-order test of
Algorithm "add"."""
import json
import os

import numpy as np
import scipy.sparse as sp

import fe_inputs as fi
from oracle import fe_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_hand_example():
    g = json.load(open(os.path.join(GOLDEN, "triplets_3x3.json")))
    keep, rowptr, colind, C, values = O.triplets_to_csr(g["n"], g["rows"], g["cols"], g["vals"])
    assert not keep
    assert rowptr.tolist() == g["rowptr"]
    assert colind.tolist() == g["colind"]
    assert C.tolist() == g["C"]
    assert values.tolist() == g["values"]


def test_against_scipy_coo_to_csr():
    rng = np.random.default_rng(5)
    n, t = 57, 4000
    rows = rng.integers(0, n, t)
    cols = rng.integers(0, n, t)
    vals = rng.standard_normal(t)
    _, rowptr, colind, C, values = O.triplets_to_csr(n, rows, cols, vals)
    S = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    np.testing.assert_array_equal(rowptr, S.indptr)
    np.testing.assert_array_equal(colind, S.indices)
    np.testing.assert_allclose(values, S.data, rtol=1e-14, atol=1e-14)
    # C points every triplet at the slot of its own (row, col)
    r_of_slot = np.repeat(np.arange(n), np.diff(rowptr))
    np.testing.assert_array_equal(r_of_slot[C], rows)
    np.testing.assert_array_equal(colind[C], cols)


def test_element_stream_matches_element_pattern():
    mesh = fi.hex_beam(2, 2, 3, jitter=0.1)
    n = 3 * mesh.n_nodes
    row, col = O.triplet_dofs(mesh.conn)
    _, rowptr, colind, C, _ = O.triplets_to_csr(n, row, col, np.ones(row.shape[0]))
    rp2, ci2, C2 = O.csr_pattern(n, mesh.conn, np.zeros(0, np.int64))
    np.testing.assert_array_equal(rowptr, rp2)
    np.testing.assert_array_equal(colind, ci2)
    np.testing.assert_array_equal(C, C2)


def test_filling_order_test():
    rows, cols = np.array([0, 1, 2, 1]), np.array([0, 1, 2, 0])
    v = np.ones(4)
    assert O.triplets_to_csr(3, rows, cols, v, prev=(rows.copy(), cols.copy()))[0]
    assert not O.triplets_to_csr(3, rows, cols, v, prev=(rows[:3], cols[:3]))[0]       # longer stream
    assert not O.triplets_to_csr(3, rows[:3], cols[:3], v[:3], prev=(rows, cols))[0]   # shorter stream
    order = np.array([3, 1, 2, 0])
    assert not O.triplets_to_csr(3, rows[order], cols[order], v, prev=(rows, cols))[0]  # same set, new order
    # the test compares both indices of every triplet: one column changed with
    # every row the same, or one row changed with every column the same
    cols2 = cols.copy()
    cols2[1] = 2
    assert not O.triplets_to_csr(3, rows, cols2, v, prev=(rows, cols))[0]
    rows2 = rows.copy()
    rows2[3] = 2
    assert not O.triplets_to_csr(3, rows2, cols, v, prev=(rows, cols))[0]
