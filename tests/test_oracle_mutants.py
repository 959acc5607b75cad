"""Planted mistakes in the oracle (no GPU): each case below copies the
oracle's C source, plants one plausible slip (a dropped factor in the
gradient, candidates from the wrong triangle, a reversed ranking or
tie-break, a transposed operand in the Cholesky update, a missing square
root, the wrong triangle in the back substitution, the printed scaling
without its square root, an inverted exit test, an unsorted pattern, an
inverted alpha or beta in PCG, a PCG that stops on the recursive residual
alone, G instead of G^T in the application, a
gather that drops the off-diagonal entries, a locality bound one power too
wide), compiles it, and runs the pins of test_oracle_pins.py and
test_oracle_locality.py against it in a child process.
The pins must fail for every slip, and pass for an unmodified copy built
the same way (the control).  (Transposing the stripe table of the locality
bound is no slip: the stripe adjacency of a symmetric A and its powers are
symmetric.)"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = [os.path.join(ROOT, "tests", "test_oracle_pins.py"), os.path.join(ROOT, "tests", "test_oracle_locality.py")]

MUTANTS = [
    ("gradient drops g",
     "w->acc[j] = fma(A->val[e], gr, w->acc[j]);",
     "w->acc[j] = fma(A->val[e], 1.0, w->acc[j]);"),
    ("candidates above the diagonal",
     "if (j >= i) continue;",
     "if (j == i) continue;"),
    ("smallest gradients ranked first",
     "return (abs_a > abs_b) || (abs_a == abs_b && col_a < col_b);",
     "return (abs_a < abs_b) || (abs_a == abs_b && col_a < col_b);"),
    ("tie-break on the larger column",
     "return (abs_a > abs_b) || (abs_a == abs_b && col_a < col_b);",
     "return (abs_a > abs_b) || (abs_a == abs_b && col_a > col_b);"),
    ("Cholesky update with a transposed operand",
     "M[(size_t)r * m + q] = fma(-M[(size_t)r * m + c], M[(size_t)q * m + c], M[(size_t)r * m + q]);",
     "M[(size_t)r * m + q] = fma(-M[(size_t)r * m + c], M[(size_t)r * m + c], M[(size_t)r * m + q]);"),
    ("pivot without square root",
     "double d = sqrt(piv);",
     "double d = piv;"),
    ("back substitution from the wrong triangle",
     "for (int32_t r = 0; r < c; ++r) z[r] = fma(-M[(size_t)c * m + r], gc, z[r]);",
     "for (int32_t r = 0; r < c; ++r) z[r] = fma(-M[(size_t)r * m + c], gc, z[r]);"),
    ("scaling without the square root",
     "double sq = sqrt(w->g[m - 1]);",
     "double sq = w->g[m - 1];"),
    ("exit test inverted",
     "stop = (psi_prev - psi) < eps * psi_prev; /* R2, default */",
     "stop = (psi_prev - psi) > eps * psi_prev; /* R2, default */"),
    ("pattern left unsorted",
     "while (pos > 0 && w->P[pos - 1] > j) {",
     "while (0) {"),
    ("PCG beta inverted",
     "double beta = rz_new / rz;",
     "double beta = rz / rz_new;"),
    ("application with G instead of G^T",
     "oracle_spmv_t(n, Grp, Gcol, Gval, t, z);",
     "oracle_spmv(n, Grp, Gcol, Gval, t, z);"),
    ("gather keeps only the diagonal",
     "if (P[b] == c) M[(size_t)a * m + b] = A->val[e];",
     "if (P[b] == c && a == b) M[(size_t)a * m + b] = A->val[e];"),
    ("literal exit test inverted",
     "stop = (psi / psi0) <= eps;",
     "stop = (psi / psi0) >= eps;"),
    ("PCG alpha inverted",
     "double alpha = rz / pq;",
     "double alpha = pq / rz;"),
    ("PCG stops on the recursive residual alone",
     "if (rnorm <= rtol * bnorm &&\n                true_residual_norm(n, rowptr, col, val, b, x, q) <= rtol * bnorm) {",
     "if (rnorm <= rtol * bnorm) {"),
    ("locality bound one power too high",
     "for (int32_t t = 0; t < power; ++t) {",
     "for (int32_t t = 0; t <= power; ++t) {"),
]


def _run_pins(lib):
    env = dict(os.environ, AFSAI_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS], cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=600)


def test_control_copy_passes_the_pins(oracle_mod, tmp_path):
    lib = oracle_mod.build_variant(oracle_mod.source_text(), str(tmp_path))
    r = _run_pins(lib)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(oracle_mod, tmp_path, name, old, new):
    src = oracle_mod.source_text()
    assert src.count(old) == 1, name
    lib = oracle_mod.build_variant(src.replace(old, new), str(tmp_path))
    r = _run_pins(lib)
    # pytest exit code 1: tests ran and at least one pin failed (not a
    # collection or usage error, not a crash of the child)
    assert r.returncode == 1, (name, r.returncode, r.stdout[-2000:])
    assert " failed" in r.stdout, (name, r.stdout[-2000:])
