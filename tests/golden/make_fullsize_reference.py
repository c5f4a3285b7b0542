"""Writes tests/golden/tet30x30x120_mr_rollout.json: the FP64 oracle's
positions and velocities of the 348,843-DOF Mooney-Rivlin tet beam (30 x 30
x 120 cubes, 6 tets each; gravity plus the sinusoidal end traction) after
10 backward-Euler steps from rest (Eqs. "dynamic equation2" and "implicit
integration"), at a fixed sample of DOFs.

The oracle's direct solve does not finish in minutes at this size, so every
step solves its system with the oracle's Jacobi CG to ||b - A a|| <= 1e-12
||b|| (oracle.fe_oracle.Model.step_cg), four orders below the 1e-8 the GPU
path is held to.  (The true residual of FP64 CG on this system levels off
near 4e-13 of ||b||, so 1e-13 is out of reach.)  Calls only the oracle and
the seeded workload generator; run from the repository root:

    python tests/golden/make_fullsize_reference.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import fe_inputs as fi  # noqa: E402
from oracle import fe_oracle as O  # noqa: E402

STEPS = 10
TOL = 1e-12


def sample_dofs(n_nodes, X):
    """Every 97th node (all three components) plus every node of the free
    end face, where the displacement is largest."""
    nodes = set(range(0, n_nodes, 97))
    nodes.update(np.nonzero(X[:, 0] == X[:, 0].max())[0].tolist())
    nodes = np.array(sorted(nodes), dtype=np.int64)
    return (3 * nodes[:, None] + np.arange(3)).reshape(-1)


def main():
    wl = fi.workload("tet30x30x120-mr")
    m = O.Model.from_workload(wl)
    X = wl.mesh.X.reshape(-1)
    q, v = X.copy(), np.zeros_like(X)
    its = []
    t0 = time.time()
    for t in range(STEPS):
        q, v, _, k = m.step_cg(q, v, wl.p(t).reshape(-1), TOL)
        its.append(int(k))
        print(f"step {t}: {k} CG iterations, {time.time() - t0:.0f} s", flush=True)
    S = sample_dofs(wl.mesh.n_nodes, wl.mesh.X)
    out = {
        "source": "FP64 oracle (tests/golden/make_fullsize_reference.py): tet30x30x120-mr from rest, "
                  f"{STEPS} steps, each system solved by the oracle's Jacobi CG to {TOL:g}",
        "workload": "tet30x30x120-mr", "steps": STEPS, "cg_tol": TOL, "cg_iterations": its,
        "dofs": S.tolist(),
        "q": q[S].tolist(), "v": v[S].tolist(),
        "disp_norm_full": float(np.linalg.norm(q - X)),
        "v_norm_full": float(np.linalg.norm(v)),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tet30x30x120_mr_rollout.json")
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print("wrote", path, len(S), "DOFs")


if __name__ == "__main__":
    main()
