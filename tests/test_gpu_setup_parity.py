"""GPU set-up parity: the CUDA aFSAI set-up (FP64 Cholesky) against the CPU
oracle on the same seeded matrices, through the C ABI.

Bar: identical patterns P_i and identical FP64 values of G (the kernel
mirrors the plain FP64 definition operation for operation), identical psi
and step counts, and G^T equal to the transpose of G.  Sizes span several
thread blocks and warps with ragged tails; edge cases cover the diagonal
pattern (kiter = 0), a full lower pattern, candidate-table overflow, both
exit tests and malformed or indefinite input.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2010_14175_gb300 import matgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_14175_gb300 import afsai

    afsai.load()
    return afsai


def run_gpu(afsai, A, kiter, s, eps, exit_mode=0, g_prec=0, chol_prec=0, block_rows=0, block_power=1):
    Ad = afsai.DeviceCSR.from_host(A)
    M = afsai.afsai_setup(Ad, afsai.params(kiter, s, eps, exit_mode, g_prec, chol_prec, block_rows, block_power))
    rp, ci, va = M.export()
    trp, tci, tva = M.export(transpose=True)
    psi, steps = M.rows()
    info = M.info()
    M.close()
    return dict(rowptr=rp, col=ci, val=va, trowptr=trp, tcol=tci, tval=tva, psi=psi, steps=steps, info=info)


def assert_identical(g, ref, A):
    assert np.array_equal(g["rowptr"], ref.rowptr), "row lengths differ"
    assert np.array_equal(g["col"], ref.col), "patterns differ"
    if not np.array_equal(g["val"], ref.val):
        d = np.abs(g["val"] - ref.val) / np.abs(ref.val)
        raise AssertionError(f"G values differ: max rel {d.max():.3e} at {int(np.argmax(d))}")
    assert np.array_equal(g["psi"], ref.psi)
    assert np.array_equal(g["steps"], ref.steps)
    # explicit transpose: rows sorted, values identical to G^T
    Gt = sp.csr_matrix((ref.val, ref.col, ref.rowptr), shape=(A.n, A.n)).T.tocsr()
    Gt.sort_indices()
    assert np.array_equal(g["trowptr"], Gt.indptr)
    assert np.array_equal(g["tcol"], Gt.indices)
    assert np.array_equal(g["tval"], Gt.data)


CASES = [
    ("poisson20", lambda: mg.poisson7(20), 5, 2, 1e-3, 0),
    ("poisson_ragged", lambda: mg.poisson7(13, 7, 11), 5, 2, 1e-3, 0),
    ("laplace1d", lambda: mg.laplace1d(1001), 10, 1, 0.05, 0),
    ("laplace1d_literal", lambda: mg.laplace1d(777), 10, 1, 0.6, 1),
    ("hetero24", lambda: mg.diffusion7_hetero(24, 99), 5, 2, 1e-3, 0),
    ("elast6", lambda: mg.elasticity_hex(6, 17), 10, 3, 1e-3, 0),
    ("fe27_aniso", lambda: mg.stencil27_fe(9, 8, 7, scale=(1.0, 1.0, 100.0)), 8, 2, 1e-3, 0),
    ("poisson2d_aniso", lambda: mg.poisson5_2d(41, 37, scale=(1.0, 1e3)), 8, 2, 1e-3, 0),
    ("random_spd", lambda: mg.random_spd(700, 0.01, 5), 6, 3, 1e-3, 0),
    ("eps0_full_kiter", lambda: mg.poisson7(9), 7, 2, 0.0, 0),
    ("kiter0_jacobi", lambda: mg.diffusion7_hetero(10, 3), 0, 1, 1e-3, 0),
    ("dense_full_pattern", lambda: mg.random_spd(40, 1.0, 2, dense=True), 1, 64, 0.0, 0),
    ("large_s", lambda: mg.poisson7(8), 3, 20, 1e-3, 0),
    ("mcap_128", lambda: mg.random_spd(300, 0.05, 8), 21, 6, 0.0, 0),
]


@pytest.mark.parametrize("name,make,kiter,s,eps,mode", CASES, ids=[c[0] for c in CASES])
def test_setup_bit_identical(gpu, oracle_mod, name, make, kiter, s, eps, mode):
    A = make()
    ref = oracle_mod.afsai_setup(A, kiter, s, eps, mode)
    g = run_gpu(gpu, A, kiter, s, eps, mode)
    assert g["info"]["nnz_G"] == ref.nnz
    assert_identical(g, ref, A)


def test_candidate_table_overflow_retry(gpu, oracle_mod):
    # ~300 entries per row and 7-entry patterns: well over 1000 distinct
    # candidates for the later rows, beyond the shared-memory table
    A = mg.random_spd(3000, 0.1, 41)
    ref = oracle_mod.afsai_setup(A, 3, 2, 0.0)
    g = run_gpu(gpu, A, 3, 2, 0.0)
    assert g["info"]["n_retry"] > 0
    assert_identical(g, ref, A)


def test_single_row_and_tiny(gpu, oracle_mod):
    from paper_2010_14175_gb300.matgen import CSR

    A = CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    ref = oracle_mod.afsai_setup(A, 5, 2, 1e-3)
    g = run_gpu(gpu, A, 5, 2, 1e-3)
    assert_identical(g, ref, A)
    A2 = mg.laplace1d(2)
    assert_identical(run_gpu(gpu, A2, 5, 2, 1e-3), oracle_mod.afsai_setup(A2, 5, 2, 1e-3), A2)


def test_malformed_csr_rejected(gpu):
    import torch

    afsai = gpu
    A = mg.poisson7(4)

    def setup_of(rowptr, col, val, n=None):
        Ad = afsai.DeviceCSR(A.n if n is None else n, torch.from_numpy(rowptr).cuda(), torch.from_numpy(col).cuda(),
                             torch.from_numpy(val).cuda())
        return afsai.afsai_setup(Ad, afsai.params(5, 2, 1e-3))

    col = A.col.copy()
    col[1], col[2] = col[2], col[1]  # unsorted row
    with pytest.raises(afsai.AfsaiError) as e:
        setup_of(A.rowptr, col, A.val)
    assert e.value.status == afsai.EINVAL
    col = A.col.copy()
    col[5] = A.n  # out of range
    with pytest.raises(afsai.AfsaiError) as e:
        setup_of(A.rowptr, col, A.val)
    assert e.value.status == afsai.EINVAL
    val = A.val.copy()
    val[A.col == np.repeat(np.arange(A.n), np.diff(A.rowptr))] *= -1.0  # negative diagonal
    with pytest.raises(afsai.AfsaiError) as e:
        setup_of(A.rowptr, A.col, val)
    assert e.value.status == afsai.EINVAL
    rp = A.rowptr.copy()
    rp[3] = rp[2] - 1  # non-monotone
    with pytest.raises(afsai.AfsaiError) as e:
        setup_of(rp, A.col, A.val)
    assert e.value.status == afsai.EINVAL
    with pytest.raises(afsai.AfsaiError) as e:
        afsai.afsai_setup(afsai.DeviceCSR.from_host(A), afsai.params(20, 7, 1e-3))  # 1 + kiter*s > 128
    assert e.value.status == afsai.ENOTSUP


def test_indefinite_matrix_reports_not_spd(gpu, oracle_mod):
    afsai = gpu
    from paper_2010_14175_gb300.matgen import CSR

    # positive diagonal, indefinite: [[1, 2], [2, 1]]
    A = CSR(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([1.0, 2.0, 2.0, 1.0]))
    with pytest.raises(RuntimeError):
        oracle_mod.afsai_setup(A, 1, 1, 0.0)
    with pytest.raises(afsai.AfsaiError) as e:
        afsai.afsai_setup(afsai.DeviceCSR.from_host(A), afsai.params(1, 1, 0.0))
    assert e.value.status == afsai.ENOTSPD


# Locality bound of the distributed set-up (Section 4): stripes of
# block_rows rows, candidates only from stripes allowed by Ahat^power.  Both
# set-up paths (stepwise for patterns of <= 20 entries, fused above) and the
# overflow retry must apply the same bound as the oracle.
BOUND_CASES = [
    ("poisson_stepwise", lambda: mg.poisson7(17, 13, 11), 5, 2, 1e-3, [(0.11, 1), (0.05, 2), (0.2, 0), (1e-9, 1)]),
    ("elast_fused", lambda: mg.elasticity_hex(6, 17), 10, 3, 1e-3, [(0.1, 1), (0.25, 0), (0.06, 2)]),
    ("fe27_fused", lambda: mg.stencil27_fe(9, 8, 7, scale=(1.0, 1.0, 100.0)), 8, 3, 1e-3, [(0.13, 1), (0.3, 2)]),
    ("random_spd", lambda: mg.random_spd(700, 0.01, 5), 6, 3, 1e-3, [(0.07, 1), (0.5, 0)]),
    ("single_stripe", lambda: mg.poisson7(9), 5, 2, 1e-3, [(1.0, 1), (1.7, 3)]),
]


@pytest.mark.parametrize("name,make,kiter,s,eps,bounds", BOUND_CASES, ids=[c[0] for c in BOUND_CASES])
def test_locality_bound_bit_identical(gpu, oracle_mod, name, make, kiter, s, eps, bounds):
    A = make()
    for frac, power in bounds:
        br = max(1, int(round(frac * A.n)))
        ref = oracle_mod.afsai_setup(A, kiter, s, eps, block_rows=br, block_power=power)
        g = run_gpu(gpu, A, kiter, s, eps, block_rows=br, block_power=power)
        assert g["info"]["nnz_G"] == ref.nnz, (br, power)
        assert_identical(g, ref, A)


def test_locality_bound_overflow_retry(gpu, oracle_mod):
    A = mg.random_spd(3000, 0.1, 41)
    ref = oracle_mod.afsai_setup(A, 3, 2, 0.0, block_rows=700, block_power=1)
    g = run_gpu(gpu, A, 3, 2, 0.0, block_rows=700, block_power=1)
    assert_identical(g, ref, A)


def test_locality_bound_arguments(gpu):
    afsai = gpu
    A = mg.poisson7(6)
    Ad = afsai.DeviceCSR.from_host(A)
    for br, pw, st in ((-1, 1, afsai.EINVAL), (8, -1, afsai.EINVAL), (8, 65, afsai.EINVAL), (1, 1, None)):
        if st is None:
            afsai.afsai_setup(Ad, afsai.params(3, 2, 1e-3, 0, 0, 0, br, pw)).close()
            continue
        with pytest.raises(afsai.AfsaiError) as e:
            afsai.afsai_setup(Ad, afsai.params(3, 2, 1e-3, 0, 0, 0, br, pw))
        assert e.value.status == st
    big = mg.laplace1d(9000)
    with pytest.raises(afsai.AfsaiError) as e:  # more than 8192 stripes
        afsai.afsai_setup(afsai.DeviceCSR.from_host(big), afsai.params(3, 2, 1e-3, 0, 0, 0, 1, 1))
    assert e.value.status == afsai.ENOTSUP


# Every set-up path must stay bit-identical to the oracle, not only the
# default one per pattern size: the fused kernel for all sizes, the
# one-lane-per-row stepwise solve, the other lane widths, and the
# small-stencil kernels at full capacity for every step or with only the
# smaller solve capacity of the early steps.  The path
# switches are read once per process, so each runs in a child process.
_PATH_SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
import oracle
from paper_2010_14175_gb300 import afsai, matgen as mg
afsai.load()
cases = [(mg.poisson7(13, 7, 11), 5, 2), (mg.elasticity_hex(6, 17), 10, 3),
         (mg.stencil27_fe(9, 8, 7, scale=(1.0, 1.0, 100.0)), 8, 2), (mg.random_spd(700, 0.01, 5), 6, 3)]
for A, kiter, s in cases:
    ref = oracle.afsai_setup(A, kiter, s, 1e-3)
    M = afsai.afsai_setup(afsai.DeviceCSR.from_host(A), afsai.params(kiter, s, 1e-3))
    rp, ci, va = M.export()
    psi, steps = M.rows()
    M.close()
    assert np.array_equal(rp, ref.rowptr) and np.array_equal(ci, ref.col), "pattern"
    assert np.array_equal(va, ref.val) and np.array_equal(psi, ref.psi) and np.array_equal(steps, ref.steps), "values"
print("ok")
"""


@pytest.mark.parametrize("env", [{"AFSAI_SETUP_FUSED_ONLY": "1"}, {"AFSAI_STEPWISE_SMALL_LPR": "1"},
                                 {"AFSAI_STEPWISE_SMALL_LPR": "4", "AFSAI_STEPWISE_WIDE": "4"},
                                 {"AFSAI_STEPWISE_WIDE": "0"}, {"AFSAI_LANE_SMALL": "0"},
                                 {"AFSAI_LANE_SMALL": "2"}],
                         ids=["fused_only", "lane_per_row", "lpr4_wide4", "wide_off", "lane_full_capacity",
                              "lane_small_solve_only"])
def test_setup_paths_bit_identical(gpu, env):
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _PATH_SCRIPT.format(root=root)], env={**os.environ, **env},
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stderr[-2000:]


_MIXED_SCRIPT = r"""
import hashlib
import sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_2010_14175_gb300 import afsai, matgen as mg
afsai.load()
cases = [(mg.stencil27_fe(9, 8, 7, scale=(1.0, 1.0, 100.0)), 8, 2), (mg.elasticity_hex(4, 17), 5, 3),
         (mg.poisson7(13, 7, 11), 5, 2)]
h = hashlib.sha256()
for A, kiter, s in cases:
    M = afsai.afsai_setup(afsai.DeviceCSR.from_host(A), afsai.params(kiter, s, 1e-3, 0, 1, 1))
    rp, ci, va = M.export()
    psi, steps = M.rows()
    M.close()
    for arr in (rp, ci, va, psi, steps):
        h.update(np.ascontiguousarray(arr).tobytes())
print(h.hexdigest())
"""


def test_mixed_form_paths_bit_identical(gpu):
    """The mixed form (FP32 Cholesky + one FP64 refinement step) gives the
    same G on every set-up path: the stepwise kernels (the table gather with
    the FP32-Cholesky solve for 27-point and elasticity rows, the lane path
    for the 7-point stencil) against the fused kernel, bit for bit."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    digests = []
    for env in ({}, {"AFSAI_SETUP_FUSED_ONLY": "1"}):
        out = subprocess.run([sys.executable, "-c", _MIXED_SCRIPT.format(root=root)], env={**os.environ, **env},
                             capture_output=True, text=True, timeout=600)
        assert out.returncode == 0, out.stderr[-2000:]
        digests.append(out.stdout.strip().splitlines()[-1])
    assert digests[0] == digests[1]
