"""GPU PCG and preconditioner-application parity against the CPU oracle,
through the C ABI.

Bars: afsai_apply equals G^T (G r) of the oracle within a rounding bound
derived from the sums (|G|^T |G| |r| times a few ulps); PCG stops after
exactly the oracle's iteration count with a true residual at most 1e-8
(both stop on the recursive residual and then require the true one,
reading R9 of Section 5.2).  The two sum their dot products in different
orders, so the iterates differ by rounding; each case therefore also checks
that the oracle's recursive residual is clear of the tolerance on both
sides of its stopping iteration (by more than 1e-6 relative), so that the
equality of the counts is not an accident of rounding.  The end-to-end host
entry point returns the same solution as the device path."""
import numpy as np
import pytest

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


def _gpu_solve(afsai, A, b, kiter, s, eps, g_prec=0, chol_prec=0, rtol=1e-8, maxit=20000):
    import torch

    Ad = afsai.DeviceCSR.from_host(A)
    M = afsai.afsai_setup(Ad, afsai.params(kiter, s, eps, 0, g_prec, chol_prec))
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    info = afsai.pcg_solve(Ad, M, bd, x, rtol=rtol, maxit=maxit)
    return x.cpu().numpy(), info, M


@pytest.mark.parametrize("name,make,kiter,s,eps", [
    ("poisson20", lambda: mg.poisson7(20), 5, 2, 1e-3),
    ("hetero20", lambda: mg.diffusion7_hetero(20, 4), 5, 2, 1e-3),
    ("elast6", lambda: mg.elasticity_hex(6, 17), 10, 3, 1e-3),
    ("fe27", lambda: mg.stencil27_fe(10, scale=(1.0, 1.0, 50.0)), 8, 2, 1e-3),
])
def test_apply_matches_oracle(gpu, oracle_mod, name, make, kiter, s, eps):
    import torch

    afsai = gpu
    A = make()
    ref = oracle_mod.afsai_setup(A, kiter, s, eps)
    M = afsai.afsai_setup(afsai.DeviceCSR.from_host(A), afsai.params(kiter, s, eps))
    r = np.random.default_rng(7).standard_normal(A.n)
    z = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    afsai.afsai_apply(M, torch.from_numpy(r).cuda(), z)
    zg = z.cpu().numpy()
    zo = oracle_mod.apply(ref, r)
    Gs = ref.to_scipy()
    absG = abs(Gs)
    bound = 64 * np.finfo(float).eps * (absG.T @ (absG @ np.abs(r)))
    assert np.all(np.abs(zg - zo) <= bound + 1e-300)
    # spmv with A
    y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    afsai.afsai_spmv(afsai.DeviceCSR.from_host(A), torch.from_numpy(r).cuda(), y)
    yo = oracle_mod.spmv(A, r)
    absA = abs(A.to_scipy())
    assert np.all(np.abs(y.cpu().numpy() - yo) <= 64 * np.finfo(float).eps * (absA @ np.abs(r)))


def clear_of_tolerance(hist, rtol=1e-8, margin=1e-6):
    """The oracle's recursive relative residual at its last iteration lies
    below rtol, and at the one before above it, each by more than `margin`
    relative: a rounding-level difference cannot move the stop."""
    return hist[-1] < rtol * (1 - margin) and hist[-2] > rtol * (1 + margin)


@pytest.mark.parametrize("name,make,kiter,s,eps", [
    ("poisson20", lambda: mg.poisson7(20), 5, 2, 1e-3),
    ("poisson20_jacobi", lambda: mg.poisson7(20), 0, 1, 1e-3),
    ("hetero24", lambda: mg.diffusion7_hetero(24, 4), 5, 2, 1e-3),
    ("elast8", lambda: mg.elasticity_hex(8, 21), 10, 3, 1e-3),
    ("poisson2d_aniso", lambda: mg.poisson5_2d(60, 50, scale=(1.0, 300.0)), 8, 2, 1e-3),
])
def test_pcg_matches_oracle(gpu, oracle_mod, name, make, kiter, s, eps):
    A = make()
    b, xs = mg.rhs(A, mg.BASE_SEED + 77)
    ref = oracle_mod.afsai_setup(A, kiter, s, eps)
    xo, it_o, rr_o, rt_o, hist = oracle_mod.pcg(A, ref, b, rtol=1e-8, history=True)
    assert clear_of_tolerance(hist), hist[-2:]
    x, info, M = _gpu_solve(gpu, A, b, kiter, s, eps)
    assert info["converged"] == 1
    assert info["iters"] == it_o, (info["iters"], it_o)
    assert info["relres_rec"] <= 1e-8
    assert info["relres_true"] <= 1e-8
    # same iterate up to the rounding-order difference of the solve
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def test_pcg_unpreconditioned_and_zero_rhs(gpu, oracle_mod):
    import torch

    afsai = gpu
    A = mg.poisson7(10)
    Ad = afsai.DeviceCSR.from_host(A)
    b, _ = mg.rhs(A, 3)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    info = afsai.pcg_solve(Ad, None, bd, x, rtol=1e-8, maxit=5000)
    assert info["converged"] == 1 and info["relres_true"] <= 1e-8
    # b = 0: converged at iteration 0 with x = 0
    x0 = torch.zeros_like(bd)
    info0 = afsai.pcg_solve(Ad, None, torch.zeros_like(bd), x0, rtol=1e-8, maxit=10)
    assert info0["iters"] == 0 and float(x0.abs().max()) == 0.0
    # maxit reached -> ENOCONV
    x1 = torch.zeros_like(bd)
    info1 = afsai.pcg_solve(Ad, None, bd, x1, rtol=1e-14, maxit=3, raise_on_noconv=False)
    assert info1["status"] == afsai.ENOCONV and info1["iters"] == 3


def test_solve_host_matches_device_path(gpu, oracle_mod):
    afsai = gpu
    A = mg.poisson7(16)
    b, _ = mg.rhs(A, 11)
    x_dev, info_dev, M = _gpu_solve(afsai, A, b, 5, 2, 1e-3)
    x = np.zeros(A.n)
    sinf, pinf = afsai.afsai_solve_host(A, afsai.params(5, 2, 1e-3), b, x, rtol=1e-8, maxit=5000)
    assert pinf["iters"] == info_dev["iters"]
    assert np.array_equal(x, x_dev)
    assert sinf["nnz_G"] == M.info()["nnz_G"]


def _refinement_bound(A, G_ref, rows_same, g_prec):
    """Entrywise relative error bound of a row of G from an FP32 Cholesky
    of A[P,P] (m x m) followed by one FP64 refinement step, per row:
    the FP32 solve leaves a relative error e0 <= kappa * g32 (g32 = m u32 /
    (1 - m u32), kappa the 2-norm condition number of A[P,P]); one step of
    refinement with an FP64 residual and an FP32 correction leaves
    e1 <= kappa * g32 * e0 + kappa * g64; the final scaling by 1/sqrt(g_m)
    at most doubles it, and FP32/BF16 storage adds one rounding."""
    u32, u64 = 2.0 ** -24, 2.0 ** -53
    S = A.to_scipy().tocsr()
    store = {0: 0.0, 1: 2.0 ** -24, 2: 2.0 ** -8}[g_prec]
    out = {}
    for i in rows_same:
        P = G_ref.col[G_ref.rowptr[i]:G_ref.rowptr[i + 1]]
        m = len(P)
        App = S[P][:, P].toarray()
        kappa = np.linalg.cond(App)
        g32, g64 = m * u32 / (1 - m * u32), m * u64 / (1 - m * u64)
        e0 = kappa * g32
        out[i] = 2 * (kappa * g32 * e0 + kappa * g64) + store
    return out


@pytest.mark.parametrize("g_prec,chol_prec", [(1, 0), (2, 0), (0, 1), (1, 1), (2, 1)])
def test_precision_forms_reach_1e8(gpu, oracle_mod, g_prec, chol_prec):
    """Mixed forms: FP32/BF16 G, FP32 Cholesky + one FP64 refinement step.
    Each must reach the true residual 1e-8; FP32 G within 10% more
    iterations than the FP64 oracle, BF16 G within 20% (BF16 misses the 10%
    bar on the 256^3 diffusion problem, +14%); G's error against the FP64
    oracle is bounded entrywise: by the storage rounding for an FP64
    Cholesky (same patterns), by the refinement bound above on the rows
    whose pattern is the oracle's for the FP32 Cholesky."""
    afsai = gpu
    A = mg.diffusion7_hetero(24, 4)
    b, _ = mg.rhs(A, 5)
    ref = oracle_mod.afsai_setup(A, 5, 2, 1e-3)
    _, it_o, _, _ = oracle_mod.pcg(A, ref, b, rtol=1e-8)
    x, info, M = _gpu_solve(afsai, A, b, 5, 2, 1e-3, g_prec=g_prec, chol_prec=chol_prec)
    assert info["converged"] == 1
    assert info["relres_true"] <= 1e-8
    bar = 1.10 if g_prec != 2 else 1.20
    assert info["iters"] <= int(np.ceil(bar * it_o)), (info["iters"], it_o)
    rp, ci, va = M.export()
    if chol_prec == 0:
        assert np.array_equal(ci, ref.col)
        unit = {0: 0.0, 1: 2.0 ** -24, 2: 2.0 ** -8}[g_prec]
        assert np.all(np.abs(va - ref.val) <= unit * np.abs(ref.val))
    else:
        same = [i for i in range(A.n) if np.array_equal(ci[rp[i]:rp[i + 1]], ref.col[ref.rowptr[i]:ref.rowptr[i + 1]])]
        assert len(same) >= 0.9 * A.n
        rng = np.random.default_rng(3)
        rows = sorted(rng.choice(same, size=min(600, len(same)), replace=False))
        bound = _refinement_bound(A, ref, rows, g_prec)
        for i in rows:
            a, b_ = ref.rowptr[i], ref.rowptr[i + 1]
            err = np.abs(va[rp[i]:rp[i + 1]] - ref.val[a:b_]) / np.abs(ref.val[a:b_])
            assert np.all(err <= bound[i]), (i, err.max(), bound[i])
