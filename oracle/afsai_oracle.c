/*
 * Plain FP64 CPU oracle for adaptive FSAI (aFSAI) and aFSAI-preconditioned
 * conjugate gradients.  TEST INFRASTRUCTURE ONLY: this file is compiled and
 * called by the tests, by the package's smoke check and by the CPU-baseline
 * leg of the benchmark.  The product (the CUDA library) never links, loads
 * or calls it, and it shares no code with the CUDA library.
 *
 * Arithmetic conventions (so that a reader can check it line by line):
 *   - IEEE double throughout; the file is compiled with -ffp-contract=off so
 *     the compiler fuses nothing; every fused multiply-add is an explicit
 *     fma() call; sqrt() and '/' are the correctly rounded IEEE operations.
 *   - Rows are independent (Section 2: each psi_i depends on row i only), so
 *     the set-up loop over rows may run on several OpenMP threads without
 *     changing any result.
 *
 * Method (Section 2 of the paper):
 *   FSAI: M^{-1} = G^T G with G lower triangular (Eq. "prec").  For row i
 *   with pattern P (sorted ascending, i last, so that i is the position of
 *   the last canonical vector e_m), solve the dense SPD system
 *   A[P,P] g = e_m (Eq. "DensSys"); psi_i = g^T A g / g_m^2 = 1 / g_m is the
 *   Schur complement of the unit-diagonal form (Eq. "blocksys"); the scaled
 *   row G[i,P] = g / sqrt(g_m) makes diag(G A G^T) = I (Eq. "diagScal", with
 *   D_G = psi^{-1/2}).
 *   Adaptive pattern (Eqs. "kap2", "grapsi"): starting from P = {i}, each
 *   step computes the gradient (A g)_j for the candidates j < i (A symmetric,
 *   so a_jr is read from row r), adds the s candidates of largest |gradient|
 *   that are not yet in P, re-solves, and stops after kiter steps or when
 *   the Kaporin-number reduction test fires (Eq. "exit_crit").
 *
 * Readings where the paper is silent or ambiguous (stated here, used below):
 *   R1  D_G = psi^{-1/2} (the printed Eq. "diagScal2" lacks the square root).
 *   R2  exit_mode 0: stop after step k when (psi_{k-1} - psi_k) <
 *       eps * psi_{k-1}; exit_mode 1: the literal psi_k / psi_0 <= eps.  The
 *       pattern of step k is kept in both cases.
 *   R3  gradient = A g (full row including the diagonal); the factor 2 and
 *       the positive scale g_m do not change the ranking.
 *   R4  ties in |gradient| are broken by the smaller column index.
 *   R5  only j not in P with |gradient| > 0 are eligible; if none, the row
 *       stops.
 *   R6  kiter counts enlargement steps (|P| <= 1 + kiter * s).
 *   R7  P is kept sorted ascending (i is its largest element, hence last).
 *   R8  the gradient sum for column j is accumulated over r in P in
 *       ascending order, each row of A in CSR (ascending column) order,
 *       acc = fma(a_rj, g_r, acc) starting from acc = 0.
 *   R9  PCG: x0 = 0, stop when ||r_k||_2 <= rtol ||b||_2 for the recursive
 *       residual (Section 5.2: "reduce the initial residual of 8 orders")
 *       and the true residual ||b - A x_k||_2 meets the same tolerance;
 *       while it does not, the iteration continues.
 *   R13 locality bound (Section 4): stripes are runs of block_rows
 *       consecutive rows (the last one may be shorter); Ahat includes the
 *       diagonal blocks; power 0 keeps each row inside its own stripe;
 *       block_rows = 0 means no bound.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENOTSPD 3

/* Per-thread scratch for the sparse gradient accumulator. */
typedef struct {
    double* acc;    /* n entries, zero outside the touched list */
    uint8_t* mark;  /* n entries, 1 if touched */
    int32_t* touched;
    int32_t ntouched;
    int32_t* P;     /* pattern, capacity mcap */
    double* g;      /* current unscaled solution g (e_m form) */
    double* M;      /* dense mcap x mcap system, factorised in place */
    int32_t* cand;  /* candidate columns */
    double* cabs;   /* |gradient| of candidates */
    int32_t* order; /* per-candidate flag: >= 0 free, -1 taken */
} row_ws;

typedef struct {
    int32_t n;
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
} csr_view;

/* Diagonal entry a_ii (0 if absent). */
static double diag_entry(const csr_view* A, int32_t i) {
    for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e)
        if (A->col[e] == i) return A->val[e];
    return 0.0;
}

static int in_pattern(const int32_t* P, int32_t m, int32_t j) {
    for (int32_t t = 0; t < m; ++t)
        if (P[t] == j) return 1;
    return 0;
}

/* Candidate order R4: |gradient| descending, then column ascending. */
static int cand_better(double abs_a, int32_t col_a, double abs_b, int32_t col_b) {
    return (abs_a > abs_b) || (abs_a == abs_b && col_a < col_b);
}

/*
 * Solve A[P,P] g = e_m by Cholesky (Eq. "DensSys").
 * Gather (Section 2, "systems gather"): M[a][b] = A[P_a, P_b], 0 where A has
 * no entry.  Right-looking Cholesky M = L L^T, in place in the lower half:
 *   for c: L_cc = sqrt(M_cc); L_rc = M_rc / L_cc (r > c);
 *          M_rq = fma(-L_rc, L_qc, M_rq) for c < q <= r.
 * Forward solve L z = e_m gives z = e_m / L_mm (only the last entry is
 * nonzero); back substitution L^T g = z, column oriented:
 *   for c = m-1..0: g_c = z_c / L_cc; z_r = fma(-L_cr, g_c, z_r) (r < c).
 * Returns 0, or ORC_ENOTSPD if a pivot is not positive.
 */
static int solve_em(const csr_view* A, const int32_t* P, int32_t m, double* M, double* g) {
    memset(M, 0, sizeof(double) * (size_t)m * (size_t)m);
    for (int32_t a = 0; a < m; ++a) {
        int32_t r = P[a];
        for (int32_t e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e) {
            int32_t c = A->col[e];
            for (int32_t b = 0; b < m; ++b)
                if (P[b] == c) M[(size_t)a * m + b] = A->val[e];
        }
    }
    for (int32_t c = 0; c < m; ++c) {
        double piv = M[(size_t)c * m + c];
        if (!(piv > 0.0)) return ORC_ENOTSPD;
        double d = sqrt(piv);
        M[(size_t)c * m + c] = d;
        for (int32_t r = c + 1; r < m; ++r) M[(size_t)r * m + c] = M[(size_t)r * m + c] / d;
        for (int32_t r = c + 1; r < m; ++r)
            for (int32_t q = c + 1; q <= r; ++q)
                M[(size_t)r * m + q] = fma(-M[(size_t)r * m + c], M[(size_t)q * m + c], M[(size_t)r * m + q]);
    }
    /* z = e_m / L_mm, then back substitution into g */
    for (int32_t r = 0; r < m; ++r) g[r] = 0.0;
    double* z = g; /* z and g share storage: g_c is written after z_c is consumed */
    z[m - 1] = 1.0 / M[(size_t)(m - 1) * m + (m - 1)];
    for (int32_t c = m - 1; c >= 0; --c) {
        double gc = z[c] / M[(size_t)c * m + c];
        z[c] = gc;
        for (int32_t r = 0; r < c; ++r) z[r] = fma(-M[(size_t)c * m + r], gc, z[r]);
    }
    return ORC_OK;
}

/*
 * Locality bound of the distributed set-up (Section 4, "aFSAI set-up on a
 * distributed memory computer").  The rows are cut into stripes of
 * block_rows consecutive rows (one stripe per process there).  Ahat is the
 * stripe adjacency of A (Ahat_IJ = 1 iff block (I, J) of A holds a
 * nonzero) and the stripe graph of G must lie in the lower part of
 * Ahat^power.  Each process gathers only the blocks of A among its allowed
 * stripes, so a row i of stripe I can only ever see candidates j of stripes
 * J with (Ahat^power)_IJ = 1 (and J <= I, which j < i already implies):
 * filtering the candidates is the same computation as running on the
 * gathered local matrix.  Returns the np x np table reach (1 = allowed),
 * built by power-fold boolean products starting from the identity; NULL
 * when out of memory.
 */
static uint8_t* block_reach(const csr_view* A, int32_t block_rows, int32_t power, int32_t* np_out) {
    int32_t np = (int32_t)(((int64_t)A->n + block_rows - 1) / block_rows);
    size_t nn = (size_t)np * (size_t)np;
    uint8_t* ahat = (uint8_t*)calloc(nn, 1);
    uint8_t* reach = (uint8_t*)calloc(nn, 1);
    uint8_t* next = (uint8_t*)calloc(nn, 1);
    if (!ahat || !reach || !next) {
        free(ahat);
        free(reach);
        free(next);
        return NULL;
    }
    for (int32_t r = 0; r < A->n; ++r)
        for (int32_t e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e)
            ahat[(size_t)(r / block_rows) * np + A->col[e] / block_rows] = 1;
    for (int32_t I = 0; I < np; ++I) reach[(size_t)I * np + I] = 1; /* Ahat^0 = identity */
    for (int32_t t = 0; t < power; ++t) {
        memset(next, 0, nn);
        for (int32_t I = 0; I < np; ++I)
            for (int32_t K = 0; K < np; ++K) {
                if (!reach[(size_t)I * np + K]) continue;
                for (int32_t J = 0; J < np; ++J)
                    if (ahat[(size_t)K * np + J]) next[(size_t)I * np + J] = 1;
            }
        memcpy(reach, next, nn);
    }
    free(ahat);
    free(next);
    *np_out = np;
    return reach;
}

/* Optional per-step trace of one row (for tests). */
typedef struct {
    int32_t max_steps;
    int32_t mcap;
    int32_t* m_k;     /* [max_steps+1] pattern size after step k (k=0: 1) */
    int32_t* P_k;     /* [(max_steps+1) * mcap] pattern after step k */
    double* g_k;      /* [(max_steps+1) * mcap] unscaled g after step k */
    double* psi_k;    /* [max_steps+1] psi after step k */
    int32_t nsteps;   /* number of recorded steps after k=0 */
} row_trace;

/*
 * aFSAI for one row i (Section 2).  Writes the scaled row into Gcol/Gval
 * (sorted columns), its length into *m_out, the final psi and the number of
 * enlargement steps performed.  Returns ORC_OK or ORC_ENOTSPD.
 */
static int afsai_row(const csr_view* A, int32_t i, int32_t kiter, int32_t s, double eps, int32_t exit_mode,
                     const uint8_t* reach, int32_t np, int32_t block_rows, row_ws* w, int32_t* Gcol, double* Gval,
                     int32_t* m_out, double* psi_out, int32_t* steps_out, row_trace* tr) {
    double aii = diag_entry(A, i);
    if (!(aii > 0.0)) return ORC_ENOTSPD;
    int32_t m = 1;
    w->P[0] = i;
    w->g[0] = 1.0 / aii; /* A[P,P] g = e_1 with P = {i} (G_0 = I, Section 2) */
    double psi0 = aii;   /* psi_0 = e_i^T A e_i */
    double psi_prev = psi0;
    int32_t steps = 0;
    if (tr) {
        tr->m_k[0] = 1;
        tr->P_k[0] = i;
        tr->g_k[0] = w->g[0];
        tr->psi_k[0] = psi0;
        tr->nsteps = 0;
    }
    for (int32_t k = 1; k <= kiter; ++k) {
        /* Kaporin gradient over j < i (Eq. "grapsi", readings R3, R8) */
        w->ntouched = 0;
        for (int32_t t = 0; t < m; ++t) {
            int32_t r = w->P[t];
            double gr = w->g[t];
            for (int32_t e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e) {
                int32_t j = A->col[e];
                if (j >= i) continue;
                /* locality bound (block_reach): stripes outside the gathered set */
                if (reach && !reach[(size_t)(i / block_rows) * np + j / block_rows]) continue;
                if (!w->mark[j]) {
                    w->mark[j] = 1;
                    w->acc[j] = 0.0;
                    w->touched[w->ntouched++] = j;
                }
                w->acc[j] = fma(A->val[e], gr, w->acc[j]);
            }
        }
        /* eligible candidates (R5) */
        int32_t nc = 0;
        for (int32_t u = 0; u < w->ntouched; ++u) {
            int32_t j = w->touched[u];
            double a = fabs(w->acc[j]);
            if (a > 0.0 && !in_pattern(w->P, m, j)) {
                w->cand[nc] = j;
                w->cabs[nc] = a;
                w->order[nc] = nc;
                ++nc;
            }
        }
        for (int32_t u = 0; u < w->ntouched; ++u) {
            w->mark[w->touched[u]] = 0;
            w->acc[w->touched[u]] = 0.0;
        }
        if (nc == 0) break;
        /* the s largest (R4), by repeated selection of the best remaining */
        int32_t add = nc < s ? nc : s;
        for (int32_t u = 0; u < add; ++u) {
            int32_t best = -1;
            for (int32_t v = 0; v < nc; ++v) {
                if (w->order[v] < 0) continue;
                if (best < 0 || cand_better(w->cabs[v], w->cand[v], w->cabs[best], w->cand[best])) best = v;
            }
            w->order[best] = -1; /* taken */
            /* insert into the sorted pattern (R7) */
            int32_t j = w->cand[best];
            int32_t pos = m;
            while (pos > 0 && w->P[pos - 1] > j) {
                w->P[pos] = w->P[pos - 1];
                --pos;
            }
            w->P[pos] = j;
            ++m;
        }
        ++steps;
        int st = solve_em(A, w->P, m, w->M, w->g);
        if (st != ORC_OK) return st;
        double psi = 1.0 / w->g[m - 1];
        if (tr && k <= tr->max_steps) {
            tr->m_k[k] = m;
            memcpy(tr->P_k + (size_t)k * tr->mcap, w->P, sizeof(int32_t) * m);
            memcpy(tr->g_k + (size_t)k * tr->mcap, w->g, sizeof(double) * m);
            tr->psi_k[k] = psi;
            tr->nsteps = k;
        }
        int stop;
        if (exit_mode == 0)
            stop = (psi_prev - psi) < eps * psi_prev; /* R2, default */
        else
            stop = (psi / psi0) <= eps; /* R2, literal Eq. "exit_crit" */
        psi_prev = psi;
        if (stop) break;
    }
    /* diagonal scaling (Eq. "diagScal", R1): G[i,P] = g / sqrt(g_m) */
    double sq = sqrt(w->g[m - 1]);
    for (int32_t t = 0; t < m; ++t) {
        Gcol[t] = w->P[t];
        Gval[t] = w->g[t] / sq;
    }
    *m_out = m;
    *psi_out = psi_prev;
    *steps_out = steps;
    return ORC_OK;
}

static int ws_alloc(row_ws* w, int32_t n, int32_t mcap, int64_t candcap) {
    memset(w, 0, sizeof(*w));
    w->acc = (double*)calloc((size_t)n, sizeof(double));
    w->mark = (uint8_t*)calloc((size_t)n, 1);
    w->touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)(candcap > 0 ? candcap : 1));
    w->P = (int32_t*)malloc(sizeof(int32_t) * (size_t)mcap);
    w->g = (double*)malloc(sizeof(double) * (size_t)mcap);
    w->M = (double*)malloc(sizeof(double) * (size_t)mcap * (size_t)mcap);
    w->cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(candcap > 0 ? candcap : 1));
    w->cabs = (double*)malloc(sizeof(double) * (size_t)(candcap > 0 ? candcap : 1));
    w->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(candcap > 0 ? candcap : 1));
    return (w->acc && w->mark && w->touched && w->P && w->g && w->M && w->cand && w->cabs && w->order) ? ORC_OK
                                                                                                      : ORC_ENOMEM;
}

static void ws_free(row_ws* w) {
    free(w->acc);
    free(w->mark);
    free(w->touched);
    free(w->P);
    free(w->g);
    free(w->M);
    free(w->cand);
    free(w->cabs);
    free(w->order);
}

static int32_t max_row_nnz(const csr_view* A) {
    int32_t mx = 0;
    for (int32_t i = 0; i < A->n; ++i) {
        int32_t l = A->rowptr[i + 1] - A->rowptr[i];
        if (l > mx) mx = l;
    }
    return mx;
}

/*
 * aFSAI set-up over rows [row_begin, row_end).  Output rows are written at
 * a fixed stride mcap = 1 + kiter*s: Gcol/Gval[(i-row_begin)*mcap + t] for
 * t < m_out[i-row_begin].  psi_out and steps_out get the final psi and step
 * count.  Returns ORC_OK, or ORC_ENOTSPD if any row met a non-positive pivot
 * (its m_out is then 0).  nthreads <= 0 uses the OpenMP default.
 */
int oracle_afsai_rows(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val, int32_t kiter,
                      int32_t s, double eps, int32_t exit_mode, int32_t block_rows, int32_t block_power,
                      int32_t row_begin, int32_t row_end, int32_t nthreads, int32_t* Gcol, double* Gval,
                      int32_t* m_out, double* psi_out, int32_t* steps_out) {
    if (n <= 0 || kiter < 0 || s < 1 || row_begin < 0 || row_end > n || row_begin > row_end) return ORC_EINVAL;
    if (block_rows < 0 || block_power < 0) return ORC_EINVAL;
    csr_view A = {n, rowptr, col, val};
    uint8_t* reach = NULL;
    int32_t np = 0;
    if (block_rows > 0) {
        reach = block_reach(&A, block_rows, block_power, &np);
        if (!reach) return ORC_ENOMEM;
    }
    int64_t mcap = 1 + (int64_t)kiter * s;
    int64_t candcap = mcap * (int64_t)max_row_nnz(&A) + 1;
    int status = ORC_OK;
#ifdef _OPENMP
    /* thread count of this call only (the default is restored after) */
    const int nt_before = omp_get_max_threads();
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        row_ws w;
        int ok = ws_alloc(&w, n, (int32_t)mcap, candcap);
        if (ok != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            status = ORC_ENOMEM;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (int32_t i = row_begin; i < row_end; ++i) {
                int64_t o = (int64_t)(i - row_begin);
                int st = afsai_row(&A, i, kiter, s, eps, exit_mode, reach, np, block_rows, &w, Gcol + o * mcap,
                                   Gval + o * mcap, &m_out[o], &psi_out[o], &steps_out[o], NULL);
                if (st != ORC_OK) {
                    m_out[o] = 0;
#ifdef _OPENMP
#pragma omp critical
#endif
                    status = st;
                }
            }
        }
        ws_free(&w);
    }
#ifdef _OPENMP
    omp_set_num_threads(nt_before);
#endif
    free(reach);
    return status;
}

/*
 * One row with a per-step trace: pattern, unscaled g and psi after every
 * step k = 0..nsteps (k = 0 is the initial diagonal pattern).  Arrays are
 * sized (max_steps+1) and (max_steps+1)*mcap with mcap = 1 + kiter*s.
 */
int oracle_afsai_row_trace(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val, int32_t kiter,
                           int32_t s, double eps, int32_t exit_mode, int32_t i, int32_t* m_k, int32_t* P_k,
                           double* g_k, double* psi_k, int32_t* nsteps) {
    if (n <= 0 || i < 0 || i >= n || kiter < 0 || s < 1) return ORC_EINVAL;
    csr_view A = {n, rowptr, col, val};
    int64_t mcap = 1 + (int64_t)kiter * s;
    int64_t candcap = mcap * (int64_t)max_row_nnz(&A) + 1;
    row_ws w;
    if (ws_alloc(&w, n, (int32_t)mcap, candcap) != ORC_OK) {
        ws_free(&w);
        return ORC_ENOMEM;
    }
    row_trace tr = {kiter, (int32_t)mcap, m_k, P_k, g_k, psi_k, 0};
    int32_t* Gc = (int32_t*)malloc(sizeof(int32_t) * (size_t)mcap);
    double* Gv = (double*)malloc(sizeof(double) * (size_t)mcap);
    int32_t mo, so;
    double po;
    int st = afsai_row(&A, i, kiter, s, eps, exit_mode, NULL, 0, 0, &w, Gc, Gv, &mo, &po, &so, &tr);
    *nsteps = tr.nsteps;
    free(Gc);
    free(Gv);
    ws_free(&w);
    return st;
}

/* ---------------------------------------------------------------------- */
/* Sparse kernels of PCG                                                    */
/* ---------------------------------------------------------------------- */

/* y = A x, each row summed in CSR order with fma from 0. */
void oracle_spmv(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* x,
                 double* y) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int32_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) acc = fma(val[e], x[col[e]], acc);
        y[i] = acc;
    }
}

/* y = A^T x for a CSR A (scatter by rows in ascending order). */
void oracle_spmv_t(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* x,
                   double* y) {
    for (int32_t j = 0; j < n; ++j) y[j] = 0.0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) y[col[e]] = fma(val[e], x[i], y[col[e]]);
}

/* Preconditioner application z = G^T (G r) (Eq. "prec"); t is n scratch. */
void oracle_apply(int32_t n, const int32_t* Grp, const int32_t* Gcol, const double* Gval, const double* r,
                  double* t, double* z) {
    oracle_spmv(n, Grp, Gcol, Gval, r, t);
    oracle_spmv_t(n, Grp, Gcol, Gval, t, z);
}

static double dot_seq(int32_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s = fma(a[i], b[i], s);
    return s;
}

/* ||b - A x||_2 (q: n entries of scratch). */
static double true_residual_norm(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                                 const double* b, const double* x, double* q) {
    oracle_spmv(n, rowptr, col, val, x, q);
    for (int32_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
    return sqrt(dot_seq(n, q, q));
}

/*
 * Preconditioned conjugate gradients with M^{-1} = G^T G (reading R9).
 * x: output (x0 = 0).  G given in CSR (lower triangular).  Returns the
 * iteration count in *iters (maxit+1 if not converged), the recursive and
 * the true relative residual, and, if hist is not NULL, the recursive
 * relative residual after every iteration in hist[0..iters] (maxit + 1
 * entries).  Dot products are plain sequential sums.
 * Stopping rule (R9, Section 5.2 "8 orders" of residual reduction): once
 * the recursive residual meets ||r_k|| <= rtol ||b||, the true residual
 * ||b - A x_k|| is computed; the solve ends when it meets the same
 * tolerance, otherwise the recurrence goes on (the extra iterations are
 * counted) and the true residual is checked again after every iteration
 * whose recursive residual meets the tolerance.
 */
int oracle_pcg(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val, const int32_t* Grp,
               const int32_t* Gcol, const double* Gval, const double* b, double* x, double rtol, int32_t maxit,
               int32_t* iters, double* relres_rec, double* relres_true, double* hist) {
    if (n <= 0) return ORC_EINVAL;
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    double* p = (double*)malloc(sizeof(double) * (size_t)n);
    double* q = (double*)malloc(sizeof(double) * (size_t)n);
    double* t = (double*)malloc(sizeof(double) * (size_t)n);
    if (!r || !z || !p || !q || !t) {
        free(r); free(z); free(p); free(q); free(t);
        return ORC_ENOMEM;
    }
    for (int32_t i = 0; i < n; ++i) {
        x[i] = 0.0;
        r[i] = b[i];
    }
    double bnorm = sqrt(dot_seq(n, b, b));
    double rnorm = sqrt(dot_seq(n, r, r));
    int32_t it = 0;
    int converged = (rnorm <= rtol * bnorm);
    if (hist) hist[0] = (bnorm > 0.0) ? rnorm / bnorm : 0.0;
    if (!converged) {
        oracle_apply(n, Grp, Gcol, Gval, r, t, z);
        for (int32_t i = 0; i < n; ++i) p[i] = z[i];
        double rz = dot_seq(n, r, z);
        for (it = 1; it <= maxit; ++it) {
            oracle_spmv(n, rowptr, col, val, p, q);
            double pq = dot_seq(n, p, q);
            double alpha = rz / pq;
            for (int32_t i = 0; i < n; ++i) {
                x[i] = fma(alpha, p[i], x[i]);
                r[i] = fma(-alpha, q[i], r[i]);
            }
            rnorm = sqrt(dot_seq(n, r, r));
            if (hist) hist[it] = (bnorm > 0.0) ? rnorm / bnorm : 0.0;
            if (rnorm <= rtol * bnorm &&
                true_residual_norm(n, rowptr, col, val, b, x, q) <= rtol * bnorm) {
                converged = 1;
                break;
            }
            oracle_apply(n, Grp, Gcol, Gval, r, t, z);
            double rz_new = dot_seq(n, r, z);
            double beta = rz_new / rz;
            rz = rz_new;
            for (int32_t i = 0; i < n; ++i) p[i] = fma(beta, p[i], z[i]);
        }
    }
    *iters = converged ? it : maxit + 1;
    *relres_rec = (bnorm > 0.0) ? rnorm / bnorm : 0.0;
    *relres_true = (bnorm > 0.0) ? true_residual_norm(n, rowptr, col, val, b, x, q) / bnorm : 0.0;
    free(r); free(z); free(p); free(q); free(t);
    return ORC_OK;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
