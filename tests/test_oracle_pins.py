"""Pins of the CPU oracle against values the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: a closed
form, a textbook special case reduced to a library routine (numpy Cholesky,
dense solves, slogdet, scipy CG), an invariant of the method, or brute force
on tiny inputs.  The cases are chosen so that a plausible slip anywhere in
the oracle (a dropped term in the gradient, a transposed gather, a wrong
sign in the back substitution, a missing square root in the scaling, an
inverted exit test, a wrong tie-break) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as sla

from paper_2010_14175_gb300 import matgen as mg

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
CASES = {c["name"]: c for c in GOLDEN["cases"]}


def _rows(G):
    for i in range(G.n):
        a, b = G.rowptr[i], G.rowptr[i + 1]
        yield i, G.col[a:b], G.val[a:b]


# --------------------------------------------------------------------------
# closed forms (tests/golden/closed_forms.json)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["params_mode0", "params_mode1"])
def test_laplace1d_closed_form(oracle_mod, mode):
    case = CASES["laplace1d_contiguous_pattern"]
    p = case[mode]
    n = 40
    A = mg.laplace1d(n)
    G = oracle_mod.afsai_setup(A, p["kiter"], p["s"], p["eps"], p["exit_mode"])
    L = np.linalg.cholesky(A.to_scipy().toarray())
    Linv = np.linalg.inv(L)
    for i, cols, vals in _rows(G):
        if i >= 4:
            assert list(cols - i) == case["interior_row_pattern_offsets"]
            assert G.steps[i] == case["interior_row_steps"]
            m = 5
            expect = np.array([(c + 1) / math.sqrt(m * (m + 1)) for c in range(m)])
            np.testing.assert_allclose(vals, expect, rtol=1e-14)
            assert G.psi[i] == pytest.approx(6.0 / 5.0, rel=1e-14)
        else:
            # boundary rows reach the full lower pattern: exact inverse factor
            assert list(cols) == list(range(i + 1))
            np.testing.assert_allclose(vals, Linv[i, : i + 1], rtol=1e-13)


def test_poisson_first_step_tie_break(oracle_mod):
    case = CASES["poisson7_first_step_tie"]
    p = case["params"]
    A = mg.poisson7(20)
    G = oracle_mod.afsai_setup(A, p["kiter"], p["s"], p["eps"], p["exit_mode"])
    nx = 20
    checked = 0
    for i, cols, _ in _rows(G):
        x, y, z = i % nx, (i // nx) % nx, i // (nx * nx)
        if 0 < x < nx - 1 and 0 < y < nx - 1 and 0 < z < nx - 1:
            assert list(cols - i) == case["interior_row_pattern_offsets"]
            checked += 1
    assert checked == 18 ** 3


def test_jacobi_special_case(oracle_mod):
    p = CASES["jacobi_special_case"]["params"]
    A = mg.diffusion7_hetero(12, 7)
    G = oracle_mod.afsai_setup(A, p["kiter"], p["s"], p["eps"], p["exit_mode"])
    d = A.to_scipy().diagonal()
    assert G.nnz == A.n
    assert np.array_equal(G.col, np.arange(A.n))
    np.testing.assert_allclose(G.val, 1.0 / np.sqrt(d), rtol=4e-16)
    # PCG with G^T G = diag(A)^{-1} is Jacobi-PCG: same iteration count as scipy
    b, _ = mg.rhs(A, 5)
    _, it, rr, rt = oracle_mod.pcg(A, G, b, rtol=1e-8)
    S = A.to_scipy()
    cnt = [0]
    M = sla.LinearOperator(S.shape, matvec=lambda v: v / d)
    sla.cg(S, b, rtol=1e-8, atol=0.0, M=M, maxiter=5000, callback=lambda xk: cnt.__setitem__(0, cnt[0] + 1))
    assert abs(it - cnt[0]) <= 1
    assert rt <= 1.01e-8


def test_full_pattern_is_inverse_cholesky_factor(oracle_mod):
    p = CASES["full_pattern_inverse_factor"]["params"]
    for seed in (1, 2, 3):
        A = mg.random_spd(12, 1.0, seed, dense=True)
        G = oracle_mod.afsai_setup(A, p["kiter"], p["s"], p["eps"], p["exit_mode"])
        Ad = A.to_scipy().toarray()
        Gd = G.to_scipy().toarray()
        Linv = np.linalg.inv(np.linalg.cholesky(Ad))
        np.testing.assert_allclose(Gd, Linv, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(Gd.T @ Gd @ Ad, np.eye(A.n), atol=1e-12)
        # exact preconditioner: PCG converges in one iteration
        b, _ = mg.rhs(A, seed)
        _, it, _, rt = oracle_mod.pcg(A, G, b, rtol=1e-8)
        assert it == 1 and rt < 1e-12


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def _small_matrices():
    return {
        "poisson6": (mg.poisson7(6), 5, 2, 1e-3),
        "elast3": (mg.elasticity_hex(3, 11), 10, 3, 1e-3),
        "hetero8": (mg.diffusion7_hetero(8, 12), 5, 2, 1e-3),
        "fe27_5": (mg.stencil27_fe(5, scale=(1, 1, 30.0)), 8, 2, 1e-3),
        "rand60": (mg.random_spd(60, 0.08, 13), 6, 2, 1e-3),
    }


@pytest.mark.parametrize("name", list(_small_matrices().keys()))
def test_unit_diagonal_and_kaporin_identity(oracle_mod, name):
    A, kiter, s, eps = _small_matrices()[name]
    G = oracle_mod.afsai_setup(A, kiter, s, eps)
    S = A.to_scipy()
    Gs = G.to_scipy()
    # lower triangular, diagonal present and last in each row
    for i, cols, vals in _rows(G):
        assert cols[-1] == i and np.all(np.diff(cols) > 0) and vals[-1] > 0
    # Eq. diagScal: diag(G A G^T) = I
    GAGt = (Gs @ S @ Gs.T).toarray()
    np.testing.assert_allclose(np.diag(GAGt), 1.0, rtol=0, atol=1e-13)
    # Eq. kap2: Kaporin number from the row measures psi equals the dense
    # definition (1/n) tr(GAG^T) / det(GAG^T)^{1/n}
    n = A.n
    _, logdetA = np.linalg.slogdet(S.toarray())
    kap_psi = math.exp((np.sum(np.log(G.psi)) - logdetA) / n)
    sign, logdet_gag = np.linalg.slogdet(GAGt)
    assert sign > 0
    kap_dense = (np.trace(GAGt) / n) / math.exp(logdet_gag / n)
    assert kap_psi == pytest.approx(kap_dense, rel=1e-11)
    # psi_i is the Schur complement: psi_i = 1 / G_ii^2
    np.testing.assert_allclose(G.psi, 1.0 / (Gs.diagonal() ** 2), rtol=1e-13)


@pytest.mark.parametrize("name", list(_small_matrices().keys()))
def test_trace_monotone_psi_gradient_zero_and_unit_diag_form(oracle_mod, name):
    A, kiter, s, eps = _small_matrices()[name]
    Ad = A.to_scipy().toarray()
    rng = np.random.default_rng(3)
    rows = sorted(set([A.n - 1, A.n // 2] + list(rng.integers(0, A.n, size=12))))
    for i in rows:
        tr = oracle_mod.row_trace(A, int(i), kiter, s, eps)
        psis = [t[2] for t in tr]
        # psi never increases (a larger pattern minimises over a superset)
        for a, b in zip(psis, psis[1:]):
            assert b <= a * (1 + 1e-14)
        for P, g, psi in tr:
            assert P[-1] == i and np.all(np.diff(P) > 0)
            # Eq. DensSys: A[P,P] g = e_m (independent dense solve)
            e = np.zeros(len(P))
            e[-1] = 1.0
            np.testing.assert_allclose(g, np.linalg.solve(Ad[np.ix_(P, P)], e), rtol=1e-11, atol=1e-15)
            # gradient (A g)_j vanishes on P \ {i}
            grad = Ad @ np.bincount(P, weights=g, minlength=A.n)
            scale = np.abs(g).max() * np.abs(Ad).max()
            assert np.all(np.abs(grad[P[:-1]]) <= 1e-12 * scale)
            # psi = 1/g_m equals g^T A g / g_m^2 (Eq. kap_min with g~ = g/g_m)
            gt = g / g[-1]
            assert psi == pytest.approx(float(gt @ Ad[np.ix_(P, P)] @ gt), rel=1e-12)
            # Eq. blocksys (unit-diagonal form) gives the same row
            if len(P) > 1:
                Pb = P[:-1]
                gtil = np.linalg.solve(Ad[np.ix_(Pb, Pb)], -Ad[Pb, i])
                psi_b = Ad[i, i] + Ad[i, Pb] @ gtil
                np.testing.assert_allclose(np.append(gtil, 1.0) / math.sqrt(psi_b), g / math.sqrt(g[-1]), rtol=1e-11)


def test_brute_force_pattern_selection(oracle_mod):
    """Every step adds exactly the s largest |(A g)_j| over eligible j < i
    (dense numpy gradient, exhaustive sort); random values, so no ties."""
    for seed in (21, 22):
        A = mg.random_spd(45, 0.15, seed)
        Ad = A.to_scipy().toarray()
        kiter, s = 6, 2
        for i in range(A.n):
            tr = oracle_mod.row_trace(A, i, kiter, s, 0.0)
            for (P0, g0, _), (P1, _, _) in zip(tr, tr[1:]):
                grad = Ad @ np.bincount(P0, weights=g0, minlength=A.n)
                elig = [j for j in range(i) if j not in set(P0) and abs(grad[j]) > 0]
                elig.sort(key=lambda j: (-abs(grad[j]), j))
                expect = sorted(set(P0) | set(elig[:s]))
                assert list(P1) == expect
            # the row stopped only for lack of candidates or at kiter
            if len(tr) - 1 < kiter:
                P, g, _ = tr[-1]
                grad = Ad @ np.bincount(P, weights=g, minlength=A.n)
                assert all(j in set(P) or grad[j] == 0 for j in range(i))


def test_exit_test_extremes(oracle_mod):
    A = mg.poisson7(6)
    # eps = 1 (relative decrease): (psi_prev - psi) < psi_prev always -> one step
    G1 = oracle_mod.afsai_setup(A, 5, 2, 1.0, 0)
    assert np.all(G1.steps[1:] == 1)
    # eps = 0: never stops early; interior rows run all kiter steps
    G0 = oracle_mod.afsai_setup(A, 5, 2, 0.0, 0)
    assert G0.steps.max() == 5
    lens = np.diff(G0.rowptr)
    assert np.all(lens <= 11) and np.all(lens[G0.steps == 5] >= 6)
    assert np.count_nonzero(lens == 11) > A.n // 2
    # literal mode with eps = 1: psi_1 / psi_0 <= 1 always -> one step
    G2 = oracle_mod.afsai_setup(A, 5, 2, 1.0, 1)
    assert np.all(G2.steps[1:] == 1)
    # literal mode with a tiny eps never fires on a diffusion matrix
    G3 = oracle_mod.afsai_setup(A, 5, 2, 1e-3, 1)
    assert np.array_equal(G3.steps, G0.steps)


def test_pcg_matches_scipy_cg_with_afsai(oracle_mod):
    A, b, xs, p = mg.workload("poisson20")
    G = oracle_mod.afsai_setup(A, **p)
    x, it, rr, rt = oracle_mod.pcg(A, G, b, rtol=1e-8)
    assert rr <= 1e-8 and rt <= 1.05e-8
    S = A.to_scipy()
    Gs = G.to_scipy()
    cnt = [0]
    M = sla.LinearOperator(S.shape, matvec=lambda v: Gs.T @ (Gs @ v))
    xs_cg, info = sla.cg(S, b, rtol=1e-8, atol=0.0, M=M, maxiter=5000,
                         callback=lambda xk: cnt.__setitem__(0, cnt[0] + 1))
    assert info == 0
    assert abs(it - cnt[0]) <= 1
    np.testing.assert_allclose(x, xs_cg, rtol=0, atol=1e-6 * np.abs(xs_cg).max())
    # aFSAI beats Jacobi in iterations (Section 5.2)
    G0 = oracle_mod.afsai_setup(A, 0, 1, 1e-3)
    _, it0, _, _ = oracle_mod.pcg(A, G0, b, rtol=1e-8)
    assert it < it0


def _scaled_poisson_smooth_solution(N=10, decades=8):
    """D A D for the 7-point Poisson matrix A and a diagonal D spanning
    `decades` orders of magnitude, with b = (D A D) x* for a smooth x* in
    the scaled variables: ||D A D|| ||x*|| / ||b|| is large, so the true
    residual ||b - A x_k|| of CG stagnates near 5e-15 while the recursive
    one keeps falling (a textbook property of finite-precision CG)."""
    import scipy.sparse as sp

    A0 = mg.poisson7(N).to_scipy()
    n = A0.shape[0]
    d = np.logspace(-decades / 2, decades / 2, n)
    np.random.default_rng(3).shuffle(d)
    S = sp.csr_matrix(sp.diags(d) @ A0 @ sp.diags(d))
    S.sort_indices()
    g = np.arange(1, N + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    mode = (np.sin(np.pi * X / (N + 1)) * np.sin(np.pi * Y / (N + 1)) * np.sin(np.pi * Z / (N + 1))).ravel(order="F")
    return mg.from_scipy(S), S @ (mode / d)


def test_pcg_stops_on_the_true_residual(oracle_mod):
    """Reading R9 (Section 5.2, 8 orders of reduction of the residual): a
    solve is converged only when the true residual meets the tolerance.
    Below the attainable accuracy the recursive residual meets it while the
    true one cannot, and the oracle must report no convergence; above it,
    every converged solve has a true residual within the tolerance.  The
    true residual is recomputed here with scipy, independently."""
    A, b = _scaled_poisson_smooth_solution()
    S = A.to_scipy()
    G = oracle_mod.afsai_setup(A, 0, 1, 1e-3)  # Jacobi
    bn = np.linalg.norm(b)
    x, it, rr, rt = oracle_mod.pcg(A, G, b, rtol=1e-15, maxit=200)
    assert it == 201, it  # maxit + 1: not converged
    assert rr <= 1e-15 and rt > 1e-15
    assert rt == pytest.approx(np.linalg.norm(b - S @ x) / bn, rel=1e-6)
    for rtol in (1e-14, 3e-14, 1e-12, 1e-8):
        x, it, rr, rt = oracle_mod.pcg(A, G, b, rtol=rtol, maxit=200)
        assert it <= 200
        assert np.linalg.norm(b - S @ x) / bn <= rtol


def test_apply_is_gt_g(oracle_mod):
    A = mg.random_spd(50, 0.1, 31)
    G = oracle_mod.afsai_setup(A, 4, 2, 1e-3)
    r = np.random.default_rng(0).standard_normal(A.n)
    Gs = G.to_scipy().toarray()
    np.testing.assert_allclose(oracle_mod.apply(G, r), Gs.T @ (Gs @ r), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle_mod.spmv(A, r), A.to_scipy() @ r, rtol=1e-13, atol=1e-13)


def test_row_subset_equals_full(oracle_mod):
    A = mg.poisson7(7)
    Gf = oracle_mod.afsai_setup(A, 5, 2, 1e-3)
    Gs = oracle_mod.afsai_setup(A, 5, 2, 1e-3, rows=(100, 200), nthreads=1)
    a, b = Gf.rowptr[100], Gf.rowptr[200]
    assert np.array_equal(Gs.col, Gf.col[a:b]) and np.array_equal(Gs.val, Gf.val[a:b])
