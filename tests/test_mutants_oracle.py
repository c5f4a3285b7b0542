"""The oracle's pins catch plausible mistakes: each mutant below plants one
mistake in a copy of the oracle (on the CPU, in a temporary directory) and the
oracle pin files (tests/test_oracle_*.py) must fail on it, while the
unmodified copy passes.

The mistakes cover the step's system (Eqs. "dynamic equation1/2": a dropped
or sign-flipped damping term, a wrong stiffness or mass coefficient, the
projection of fixed rows, Section 5.1), the integration (Eq. "implicit
integration"), the material laws and the hex quadrature (Section 3.1), the
consistent mass (Section 4.1), the co-rotational rotation (Eq. "eqmodel"), the
pattern (Section 4.2), the contact stages (Section "Lagrangian
multipliers": projection, offset scaling, correction sign), the filling-order
test of Algorithm "add" (Section 4.2), Newton's corrections, the discrete
adjoint (not in the paper: the chain of one step's residual) and the Jacobi
CG solve of the full-size reference (Section 6.2's stopping test).
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = [
    ("damping alpha M v dropped from b",
     "b = p - f - (al * (self.M @ v) + (be + h) * (K @ v))", "b = p - f - ((be + h) * (K @ v))"),
    ("sign of (beta + h) K v in b",
     "b = p - f - (al * (self.M @ v) + (be + h) * (K @ v))",
     "b = p - f - (al * (self.M @ v) - (be + h) * (K @ v))"),
    ("h (beta + h) K -> h beta K in A",
     "A = (1.0 + h * al) * self.M + h * (be + h) * K", "A = (1.0 + h * al) * self.M + h * be * K"),
    ("(1 + h alpha) M -> M in A",
     "A = (1.0 + h * al) * self.M + h * (be + h) * K", "A = self.M + h * (be + h) * K"),
    ("Mooney-Rivlin J^-2/3 -> J^-1/3",
     "return (c10 * (J ** (-2.0 / 3.0) * I1 - 3.0)", "return (c10 * (J ** (-1.0 / 3.0) * I1 - 3.0)"),
    ("neo-Hookean -mu ln J dropped",
     "return 0.5 * mu * (I1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ",
     "return 0.5 * mu * (I1 - 3.0) + 0.5 * lam * lnJ * lnJ"),
    ("tet consistent mass /20 -> /24",
     "base = (np.ones((4, 4)) + np.eye(4)) / 20.0", "base = (np.ones((4, 4)) + np.eye(4)) / 24.0"),
    ("q+ = q + h v with the old v", "q1 = q + self.h * v1", "q1 = q + self.h * v"),
    ("hex Gauss points at +-1/2", "return _hex_corners() / math.sqrt(3.0)", "return _hex_corners() * 0.5"),
    ("fixed rows of b not cleared",
     "        b[self.fixed_dofs] = 0.0\n        return project(A, self.fixed_dofs), b",
     "        return project(A, self.fixed_dofs), b"),
    ("PGS without the projection onto lambda >= 0",
     "new = max(0.0, lam[i] + (r[i] - W[i] @ lam) / W[i, i])", "new = lam[i] + (r[i] - W[i] @ lam) / W[i, i]"),
    ("contact offset divided by h, not h^2", "x_pred)) / (h * h)", "x_pred)) / h"),
    ("contact correction with the wrong sign", "a = a_free + Z @ lam", "a = a_free - Z @ lam"),
    ("co-rotational rotation transposed", "    return U @ Vt\n", "    return np.swapaxes(U @ Vt, 1, 2)\n"),
    ("pattern: fixed rows without their diagonal slot",
     "uniq = np.unique(np.concatenate([keys, fd * n_dof + fd]))", "uniq = np.unique(keys)"),
    ("adjoint: a_bar without the h^2 q_bar term",
     "a_bar = h * v_bar + h * h * q_bar", "a_bar = h * v_bar + h * q_bar"),
    ("adjoint: v_bar update without alpha M lambda",
     "gv = al * (model.M @ lam) + (be + h) * Klam", "gv = (be + h) * Klam"),
    ("adjoint: third-derivative term dK[lambda] dropped",
     "gq = _scatter_elem(model.n_dof, conn, dKu + Kl)", "gq = _scatter_elem(model.n_dof, conn, Kl)"),
    ("Newton: correction added with the wrong sign", "            a = a + delta\n", "            a = a - delta\n"),
    ("Newton: K taken at the start of the step", "            K = self.stiffness(qk)\n",
     "            K = self.stiffness(q)\n"),
    ("filling-order test compares the rows only",
     "np.array_equal(prev[0], rows) and np.array_equal(prev[1], cols))", "np.array_equal(prev[0], rows))"),
    ("CG without the Jacobi preconditioner's scaling of z", "        z = dinv * r\n        rz_new", "        z = r\n        rz_new"),
    ("CG stops on the recursive residual alone",
     "            r = b - A @ x                     # the recursion's residual drifts: confirm with the true one\n",
     ""),
]


def _pin_files(root):
    d = os.path.join(root, "tests")
    return sorted(os.path.join("tests", f) for f in os.listdir(d)
                  if f.startswith("test_oracle") and f.endswith(".py"))


def _run_pins(root):
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *_pin_files(root)],
                       cwd=root, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-400:]


@pytest.fixture(scope="module")
def copy_root(tmp_path_factory):
    root = str(tmp_path_factory.mktemp("oracle_copy"))
    for d in ("tests", "oracle", "fe_inputs"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(root, d),
                        ignore=shutil.ignore_patterns("__pycache__"))
    return root


def test_unmodified_copy_passes_the_pins(copy_root):
    rc, out = _run_pins(copy_root)
    assert rc == 0, out


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(copy_root, name, old, new):
    path = os.path.join(copy_root, "oracle", "fe_oracle.py")
    src = open(os.path.join(ROOT, "oracle", "fe_oracle.py")).read()
    assert src.count(old) == 1, f"mutation site of '{name}' not found once"
    try:
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        rc, out = _run_pins(copy_root)
    finally:
        with open(path, "w") as f:
            f.write(src)
    assert rc != 0, f"no pin caught: {name}\n{out}"
