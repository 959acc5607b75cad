"""Pins of the oracle's locality-bounded candidate set (no GPU).

Section 4 of the paper ("aFSAI set-up on a distributed memory computer")
bounds the pattern search: with the rows cut into stripes (one per process),
Ahat the stripe adjacency of A and k a small power, the stripe graph of G
must lie in the lower part of Ahat^k; each process gathers the blocks of A
among its allowed stripes into a local matrix and runs the set-up on it.

The pins check the oracle's bounded set-up against that construction and
against closed forms, never against itself:
  * one stripe (block_rows >= n) is the unbounded method, bit for bit;
  * power 0 equals the unbounded method on the block-diagonal part of A;
  * any power equals the unbounded method on the paper's gathered local
    matrix, with the allowed stripes computed here by numpy boolean powers;
  * block_rows = 1, power 1 with a saturating search is classic FSAI on the
    lower pattern of A (numpy dense solves);
  * on the 1D Laplacian with stripes of two rows the patterns and values
    have a closed form.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2010_14175_gb300 import matgen as mg


def _stripe_reach(A, block_rows, power):
    """(Ahat^power != 0) by numpy: Ahat_IJ = 1 iff block (I, J) of A has a
    nonzero; Ahat^0 = identity."""
    n = A.n
    nb = -(-n // block_rows)
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    ahat = np.zeros((nb, nb), dtype=np.int64)
    ahat[rows // block_rows, A.col // block_rows] = 1
    reach = np.eye(nb, dtype=np.int64)
    for _ in range(power):
        reach = ((reach @ ahat) > 0).astype(np.int64)
    return reach.astype(bool)


def _masked(A, keep_rows_cols):
    """A with the entries (r, c) kept only where both r and c are allowed;
    the other rows get a unit diagonal so that the matrix stays well formed
    (they are never touched by the rows whose search is bounded to the
    allowed set)."""
    M = A.to_scipy().tocoo()
    ok = keep_rows_cols[M.row] & keep_rows_cols[M.col]
    r = np.concatenate([M.row[ok], np.flatnonzero(~keep_rows_cols)])
    c = np.concatenate([M.col[ok], np.flatnonzero(~keep_rows_cols)])
    v = np.concatenate([M.data[ok], np.ones(int((~keep_rows_cols).sum()))])
    return mg.from_scipy(sp.csr_matrix((v, (r, c)), shape=M.shape))


def _same(G1, G2):
    assert np.array_equal(G1.rowptr, G2.rowptr)
    assert np.array_equal(G1.col, G2.col)
    assert np.array_equal(G1.val, G2.val)
    assert np.array_equal(G1.psi, G2.psi) and np.array_equal(G1.steps, G2.steps)


MATS = {
    "poisson7_8": lambda: mg.poisson7(8),
    "stencil27_6": lambda: mg.stencil27_fe(6, scale=(1.0, 1.0, 10.0)),
    "random_spd_300": lambda: mg.random_spd(300, 0.05, mg.BASE_SEED + 71),
}


@pytest.mark.parametrize("name", sorted(MATS))
def test_single_stripe_is_unbounded(oracle_mod, name):
    A = MATS[name]()
    G0 = oracle_mod.afsai_setup(A, 5, 2, 1e-3)
    for br in (A.n, A.n + 17):
        _same(oracle_mod.afsai_setup(A, 5, 2, 1e-3, block_rows=br, block_power=1), G0)


@pytest.mark.parametrize("name", sorted(MATS))
def test_power_zero_is_block_diagonal(oracle_mod, name):
    A = MATS[name]()
    br = 61  # stripes that do not divide n
    stripe = np.arange(A.n) // br
    M = A.to_scipy().tocoo()
    ok = stripe[M.row] == stripe[M.col]
    Ab = mg.from_scipy(sp.csr_matrix((M.data[ok], (M.row[ok], M.col[ok])), shape=M.shape))
    _same(oracle_mod.afsai_setup(A, 4, 3, 1e-3, block_rows=br, block_power=0), oracle_mod.afsai_setup(Ab, 4, 3, 1e-3))


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("power", [1, 2])
def test_gathered_local_matrix(oracle_mod, name, power):
    """The bounded rows of stripe I equal the unbounded rows computed on the
    local matrix that gathers A's blocks among the allowed stripes of I."""
    A = MATS[name]()
    br = max(8, A.n // 9)
    reach = _stripe_reach(A, br, power)
    G = oracle_mod.afsai_setup(A, 6, 2, 1e-3, block_rows=br, block_power=power)
    stripe = np.arange(A.n) // br
    for I in range(reach.shape[0]):
        r0, r1 = I * br, min(A.n, (I + 1) * br)
        AI = _masked(A, reach[I][stripe])
        GI = oracle_mod.afsai_setup(AI, 6, 2, 1e-3, rows=(r0, r1))
        a, b = G.rowptr[r0], G.rowptr[r1]
        assert np.array_equal(np.diff(G.rowptr[r0:r1 + 1]), np.diff(GI.rowptr))
        assert np.array_equal(G.col[a:b], GI.col)
        assert np.array_equal(G.val[a:b], GI.val)
        # every entry lies in an allowed lower stripe
        assert reach[I][stripe[G.col[a:b]]].all()


@pytest.mark.parametrize("name", sorted(MATS))
def test_lower_pattern_fsai(oracle_mod, name):
    """block_rows 1, power 1: candidates are the row's own lower neighbours;
    with s >= the row length and eps = 0 the first step takes them all and
    the second finds none, so G is classic FSAI on the lower pattern of A:
    G[i,P] = g / sqrt(g_m) with A[P,P] g = e_m (numpy dense solve)."""
    A = MATS[name]()
    smax = int(np.diff(A.rowptr).max())
    G = oracle_mod.afsai_setup(A, 3, smax, 0.0, block_rows=1, block_power=1)
    D = A.to_scipy().toarray()
    for i in range(A.n):
        P = np.array([j for j in A.col[A.rowptr[i]:A.rowptr[i + 1]] if j <= i])
        a, b = G.rowptr[i], G.rowptr[i + 1]
        assert np.array_equal(G.col[a:b], P)
        e = np.zeros(len(P))
        e[-1] = 1.0
        g = np.linalg.solve(D[np.ix_(P, P)], e)
        np.testing.assert_allclose(G.val[a:b], g / math.sqrt(g[-1]), rtol=1e-12, atol=1e-14)
        assert G.steps[i] == (1 if len(P) > 1 else 0)


def test_laplace1d_two_row_stripes(oracle_mod):
    """1D Laplacian (2 on the diagonal, -1 off), stripes of two rows,
    power 1: each step adds min(P) - 1 until it leaves stripes I-1, I, so
    P = [2 max(I-1, 0), i] and, for the m x m tridiagonal system,
    G[i, P_c] = (c + 1) / sqrt(m (m + 1)), psi = (m + 1) / m."""
    n = 24
    A = mg.laplace1d(n)
    G = oracle_mod.afsai_setup(A, 6, 1, 0.0, block_rows=2, block_power=1)
    for i in range(n):
        lo = 2 * max(i // 2 - 1, 0)
        m = i - lo + 1
        a, b = G.rowptr[i], G.rowptr[i + 1]
        assert list(G.col[a:b]) == list(range(lo, i + 1))
        expect = np.array([(c + 1) / math.sqrt(m * (m + 1)) for c in range(m)])
        np.testing.assert_allclose(G.val[a:b], expect, rtol=1e-14)
        assert G.psi[i] == pytest.approx((m + 1) / m, rel=1e-14)


def test_invalid_bound_arguments(oracle_mod):
    A = mg.poisson7(4)
    for br, pw in ((-1, 1), (4, -1)):
        with pytest.raises(RuntimeError):
            oracle_mod.afsai_setup(A, 3, 2, 1e-3, block_rows=br, block_power=pw)
