// aFSAI set-up on the GPU (Section 2 of the paper; kernels of Section 3).
//
// Two paths compute the same rows bit for bit (FP64 form):
//   fused     one warp owns one row i for the whole adaptive iteration: the
//             three kernels the paper launches per step (Kaporin gradient +
//             selection, systems gather, batched Cholesky) and the exit test
//             run in one launch with no intermediate global state (below);
//   stepwise  per step a gather kernel (warp per row) and a solve kernel
//             with several rows per warp, so that each FP64 square root and
//             division warp operation serves several rows (section
//             "Stepwise set-up" further down).  Used for FP64 patterns of up
//             to 32 entries and for the mixed form of 21 to 32 entries.
//
// The fused kernel:
//
//   init      P = {i}, g = 1/a_ii, psi_0 = a_ii              (G_0 = I)
//   step k    gradient  (A g)_j over j < i, accumulated in a per-warp hash
//                       table in shared memory: rows r in P in ascending
//                       order, each row's entries spread over the lanes
//                       (distinct columns per row, so no two lanes touch one
//                       slot in the same pass), acc = fma(a_rj, g_r, acc)
//                                                        (Eq. "grapsi")
//             select    s times a warp-shuffle arg-max of |acc| (ties to the
//                       smaller column) over the slots not in P
//             merge     sorted insertion into P (i stays last)
//             gather    A[P,P] lower triangle, packed, in shared memory
//                       (aliases the hash table, which is dead by then)
//             Cholesky  right-looking; the trailing update of each column is
//                       spread over all lanes as (r, q) pairs so FP64 warp
//                       instructions stay full           (Eq. "DensSys")
//             solve     L z = e_m, L^T g = z column by column
//             exit      psi = 1/g_m; relative-decrease or literal test
//                                                        (Eq. "exit_crit")
//   finish    G[i,P] = g / sqrt(g_m)                     (Eq. "diagScal")
//
// Every floating-point operation mirrors the plain FP64 definition of the
// method one for one (explicit fma, IEEE division and square root, fixed
// order per element), so the FP64 set-up is bit-identical to it: same
// patterns, same values.  The TU is compiled with --fmad=false so that no
// multiply-add is contracted behind the code's back.
//
// With chol_prec = 1 the dense solve runs in FP32 (factorisation and both
// triangular solves) followed by one FP64 refinement step
//   res = e_m - A[P,P] g (FP64),  L L^T d = res (FP32),  g += d (FP64),
// while the gradient and the selection stay FP64.
//
// Rows whose candidate set overflows the shared-memory table are listed and
// redone by a second launch that keeps the table in global memory.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <string>

#include "afsai_internal.cuh"
#include "fp64_rn.cuh"
#include "spmv_tiled.cuh"

namespace afsai {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int32_t kRowOk = 0;
constexpr int32_t kRowNotSpd = 3;
constexpr int32_t kRowOverflow = 10;
constexpr int kSetupThreads = 256;

struct SetupArgs {
    int32_t n;
    const int32_t* __restrict__ rowptr;
    const int32_t* __restrict__ col;
    const double* __restrict__ val;
    int32_t kiter;
    int32_t s;
    int32_t exit_mode;
    double eps;
    int64_t mcap;  // row stride of the per-row outputs
    int32_t* __restrict__ out_len;
    int32_t* __restrict__ out_col;
    double* __restrict__ out_val;
    double* __restrict__ psi;
    int32_t* __restrict__ steps;
    int32_t* __restrict__ status;
    const int32_t* __restrict__ rows;  // optional row list (retry pass)
    int32_t nrows;
    int32_t* __restrict__ retry_rows;
    int32_t* __restrict__ counters;  // [0] retry count, [1] not-SPD count
    int32_t* __restrict__ gkey;      // global table (retry pass)
    double* __restrict__ gval;
    int32_t* __restrict__ glist;
    int32_t ght_log2;
    // locality bound (Section 4): reach words of each stripe (nullptr: none)
    const uint32_t* __restrict__ reach;
    int32_t reach_words;
    int32_t stripe_shift;
    uint64_t stripe_magic;
};

template <int MCAP, int HT>
struct WarpWs {
    double g[MCAP];                        // current (unscaled) solution, also the solve's z
    double Mraw[MCAP * (MCAP + 1) / 2];    // gathered A[P,P], packed lower, persists across steps
    int32_t P[MCAP];                       // pattern, sorted ascending (i last)
    int32_t newj[MCAP];                    // picks of this step (reused as FP32 scratch)
    int32_t rb[MCAP];                      // row bounds of the pattern's rows of A
    int32_t re[MCAP];
    int32_t isnew[MCAP];                   // 1 for positions inserted this step
    int32_t opos[MCAP];                    // new position of each old position
    int32_t Pn[MCAP];                      // merge buffers
    int32_t rbn[MCAP];
    int32_t ren[MCAP];
    int32_t pad_[2];
    union {
        struct {
            double val[HT];
            int32_t key[HT];
            int32_t list[HT];              // slots in insertion order (compact candidate list)
        } h;
        struct {
            double L[MCAP * (MCAP + 1) / 2];   // FP64 factor (chol_prec = 0) / old Mraw during the move
            float Lf[MCAP * (MCAP + 1) / 2];   // FP32 factor (chol_prec = 1)
        } f;
    } u;
};

__device__ __forceinline__ int tri(int r) { return (r * (r + 1)) >> 1; }

__device__ __forceinline__ int find_sorted(const int32_t* P, int m, int32_t c) {
    int lo = 0, hi = m - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int32_t v = P[mid];
        if (v == c) return mid;
        if (v < c)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

// Fibonacci hashing of a column index into 2^log2 slots.
__device__ __forceinline__ uint32_t slot_of(int32_t j, int log2) {
    return (static_cast<uint32_t>(j) * 0x9E3779B1u) >> (32 - log2);
}

// Finds j in the table or claims an empty slot for it (CAS); returns the
// slot, or -1 if every slot is taken, and sets `fresh` for a claimed slot.
__device__ __forceinline__ int table_claim(int32_t* key, int log2, int32_t j, bool& fresh) {
    const uint32_t mask = (1u << log2) - 1u;
    uint32_t h = slot_of(j, log2);
    fresh = false;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t cur = atomicCAS(&key[h], -1, j);
        if (cur == -1) {
            fresh = true;
            return static_cast<int>(h);
        }
        if (cur == j) return static_cast<int>(h);
        h = (h + 1) & mask;
    }
    return -1;
}

// Appends the slots claimed in one pass to the compact list in lane order,
// with one ballot instead of an atomic counter per new key; nk (the list
// length) is kept equal in every lane of the group.  Sets `full` once the
// table holds more than 7/8 of its slots or a probe found no slot, which
// sends the row to the retry pass with a larger table (bounded probing).
__device__ __forceinline__ void table_append(int32_t* list, int slot, bool fresh, bool failed, int& nk, bool& full,
                                             int log2, unsigned gmask) {
    const unsigned bal = __ballot_sync(gmask, fresh) & gmask;
    if (fresh) list[nk + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = slot;
    nk += __popc(bal);
    const int ht = 1 << log2;
    if (failed || nk > ht - (ht >> 3)) full = true;
}

__device__ __forceinline__ int table_find(const int32_t* key, int log2, int32_t j) {
    const uint32_t mask = (1u << log2) - 1u;
    uint32_t h = slot_of(j, log2);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t cur = key[h];
        if (cur == j) return static_cast<int>(h);
        if (cur == -1) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

// x > 0 for an IEEE double, decided on the integer pipe: positive finite or
// +inf (NaN and non-positive values give false, as the FP comparison does).
__device__ __forceinline__ bool positive(double x) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool positive(float x) {
    const int b = __float_as_int(x);
    return b > 0 && b <= 0x7f800000;
}

// Right-looking Cholesky of the packed lower triangle M (m x m) in place.
// The trailing update of column c is spread over the lanes as (r, q) pairs
// through the per-block table `pairs` (idx -> rr << 8 | qq, idx = rr(rr+1)/2
// + qq).  Returns false (warp-uniform) on a non-positive pivot.
//
// FP64 (T = double): IEEE square roots and divisions, the operations of the
// plain definition.  FP32 (T = float, the precision form, whose result is
// corrected by an FP64 refinement step): the pivot's reciprocal square root
// r = rsqrt(piv) gives L_cc = piv r and L_rc = M_rc r, and the diagonal slot
// keeps r (the reciprocal of L_cc) for the triangular solves, which then
// multiply instead of divide.
template <int GL, typename T>
__device__ bool group_cholesky(T* M, int m, int sub, unsigned gmask, const uint16_t* pairs) {
    for (int c = 0; c < m; ++c) {
        const T piv = M[tri(c) + c];
        if (!positive(piv)) return false;
        if constexpr (sizeof(T) == 4) {
            const float rinv = rsqrtf(piv);
            for (int r = c + 1 + sub; r < m; r += GL) M[tri(r) + c] = M[tri(r) + c] * rinv;
            __syncwarp(gmask);
            if (sub == 0) M[tri(c) + c] = rinv;
        } else {
            const T d = sqrt(piv);
            for (int r = c + 1 + sub; r < m; r += GL) M[tri(r) + c] = M[tri(r) + c] / d;
            __syncwarp(gmask);
            if (sub == 0) M[tri(c) + c] = d;
        }
        const int w = m - c - 1;
        const int T_ = (w * (w + 1)) >> 1;
        for (int idx = sub; idx < T_; idx += GL) {
            const int pr = pairs[idx];
            const int r = c + 1 + (pr >> 8), q = c + 1 + (pr & 0xff);
            M[tri(r) + q] = fma(-M[tri(r) + c], M[tri(q) + c], M[tri(r) + q]);
        }
        __syncwarp(gmask);
    }
    return true;
}

// Solves L L^T x = rhs in place in x (x holds rhs on entry), column
// oriented as in the plain definition: forward L z = rhs, back L^T x = z.
// When `em` is true the right-hand side is e_m and the forward solve
// reduces to z = e_m / L_mm.
// FP32: the diagonal slots hold the reciprocals of L_cc (group_cholesky).
template <int GL, typename T>
__device__ __forceinline__ T div_diag(T v, const T* L, int c) {
    if constexpr (sizeof(T) == 4)
        return v * L[tri(c) + c];
    else
        return v / L[tri(c) + c];
}

template <int GL, typename T>
__device__ void group_llt_solve(const T* L, T* x, int m, bool em, int sub, unsigned gmask) {
    if (em) {
        for (int t = sub; t < m; t += GL) x[t] = T(0);
        __syncwarp(gmask);
        if (sub == 0) x[m - 1] = div_diag<GL, T>(T(1), L, m - 1);
        __syncwarp(gmask);
    } else {
        for (int c = 0; c < m; ++c) {
            const T zc = div_diag<GL, T>(x[c], L, c);
            __syncwarp(gmask);
            if (sub == 0) x[c] = zc;
            for (int r = c + 1 + sub; r < m; r += GL) x[r] = fma(-L[tri(r) + c], zc, x[r]);
            __syncwarp(gmask);
        }
    }
    for (int c = m - 1; c >= 0; --c) {
        const T gc = div_diag<GL, T>(x[c], L, c);
        __syncwarp(gmask);
        if (sub == 0) x[c] = gc;
        for (int r = sub; r < c; r += GL) x[r] = fma(-L[tri(c) + r], gc, x[r]);
        __syncwarp(gmask);
    }
}

// Locality bound of the distributed set-up (Section 4): the rows are cut
// into stripes of block_rows rows and a row of stripe I takes candidates
// only from the stripes J whose bit is set in I's reach words (the stripe
// adjacency of A raised to the chosen power).  J = j / block_rows by a
// multiply-shift that is exact for 0 <= j < 2^31 (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994: magic =
// floor(2^(31+l) / d) + 1 with l = ceil(log2 d), shift 31 + l).
//
// The gradient table still accumulates every column j < i; the bound then
// zeroes the gradient of the columns outside the allowed stripes, which
// makes them ineligible exactly as if they had been skipped (only
// candidates with a nonzero gradient are ever taken, and the sums of the
// allowed columns do not depend on the others).  This keeps the hot
// accumulation loop free of the test.
struct StripeBound {
    const uint32_t* row = nullptr;  // reach words of the row's stripe; nullptr: no bound
    uint64_t magic = 0;
    int shift = 0;
    __device__ __forceinline__ bool allows(int32_t j) const {
        const uint32_t J = static_cast<uint32_t>((static_cast<uint64_t>(j) * magic) >> shift);
        return (__ldg(&row[J >> 5]) >> (J & 31u)) & 1u;
    }
};

__device__ __forceinline__ StripeBound stripe_bound(const uint32_t* reach, int32_t words, uint64_t magic, int shift,
                                                    int32_t i) {
    StripeBound b;
    if (reach != nullptr) {
        const uint32_t I = static_cast<uint32_t>((static_cast<uint64_t>(i) * magic) >> shift);
        b.row = reach + static_cast<size_t>(I) * words;
        b.magic = magic;
        b.shift = shift;
    }
    return b;
}

// Zeroes the gradient of the table's columns outside the row's allowed
// stripes (no-op without a bound).
__device__ __forceinline__ void apply_stripe_bound(const StripeBound& bd, const int32_t* key, double* hv,
                                                   const int32_t* list, int nk, int sub, int gl, unsigned gmask) {
    if (bd.row == nullptr) return;
    for (int t = sub; t < nk; t += gl) {
        const int sl = list[t];
        if (!bd.allows(key[sl])) hv[sl] = 0.0;
    }
    __syncwarp(gmask);
}

// Entries of one row of A held in registers: chunk q covers the entries
// rb + sub + q*GL (up to NPF chunks; longer rows continue directly).  NPF is
// 1 for short rows (small candidate tables), 4 otherwise, to keep the
// register budget of short-row kernels low.
template <int NPF>
struct RowPref {
    int32_t c[NPF];
    double v[NPF];
};

template <int GL, int NPF>
__device__ __forceinline__ void prefetch_row(RowPref<NPF>& R, const int32_t* __restrict__ colA,
                                             const double* __restrict__ valA, int32_t rb, int32_t re, int sub) {
#pragma unroll
    for (int q = 0; q < NPF; ++q) {
        const int32_t e = rb + sub + q * GL;
        R.c[q] = e < re ? __ldg(&colA[e]) : INT_MAX;
        R.v[q] = e < re ? __ldg(&valA[e]) : 0.0;
    }
}

// Accumulates one row r of A (weight gr = g_r) into the candidate table:
// acc_j = fma(a_rj, g_r, acc_j) for the row's columns j < i, in CSR order.
template <int GL, int NPF>
__device__ __forceinline__ void accumulate_row(const RowPref<NPF>& R, const int32_t* __restrict__ colA,
                                               const double* __restrict__ valA, int32_t rb, int32_t re, int32_t i,
                                               double gr, int32_t* key, double* hv, int32_t* list, int log2,
                                               int& nk, bool& ovf, int sub, unsigned gmask) {
#pragma unroll
    for (int q = 0; q < NPF; ++q) {
        const int32_t j = R.c[q];
        if (!__any_sync(gmask, j < i)) return;  // columns are sorted
        bool fresh = false;
        int slot = -1;
        if (j < i) slot = table_claim(key, log2, j, fresh);
        table_append(list, slot, fresh, j < i && slot < 0, nk, ovf, log2, gmask);
        if (slot >= 0) hv[slot] = fma(R.v[q], gr, hv[slot]);
    }
    for (int32_t e = rb + sub + NPF * GL;; e += GL) {
        const int32_t j = e < re ? __ldg(&colA[e]) : INT_MAX;
        const double v = e < re ? __ldg(&valA[e]) : 0.0;
        if (!__any_sync(gmask, j < i)) return;
        bool fresh = false;
        int slot = -1;
        if (j < i) slot = table_claim(key, log2, j, fresh);
        table_append(list, slot, fresh, j < i && slot < 0, nk, ovf, log2, gmask);
        if (slot >= 0) hv[slot] = fma(v, gr, hv[slot]);
    }
}

// Selection of the s largest |gradient| (ties: smaller column) among the
// table's candidates.  For s <= 4 in one pass: each lane keeps its own best
// four in registers, then s rounds of a warp arg-max over the lanes' heads,
// the winning lane dropping its head; (|grad| descending, column ascending)
// is a total order, so the picks and their order are those of s passes that
// each take the best remaining candidate (the pass form serves larger s).
// Writes the picks to newj; returns their number (< s when the eligible
// candidates, nonzero and not NaN, run out).
__device__ __forceinline__ bool cand_better(unsigned long long a, int32_t ja, unsigned long long b, int32_t jb) {
    return a > b || (a == b && ja < jb);
}

template <int GL>
__device__ __forceinline__ int select_top_s(const int32_t* key, double* hv, const int32_t* list, int nk, int s, int sub,
                                            unsigned gmask, int32_t* newj) {
    int npick = 0;
    if (s <= 4) {
        unsigned long long kb[4] = {0ull, 0ull, 0ull, 0ull};
        int32_t kj[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
        for (int t = sub; t < nk; t += GL) {
            const int sl = list[t];
            const int32_t j = key[sl];
            const unsigned long long ab =
                static_cast<unsigned long long>(__double_as_longlong(hv[sl])) & 0x7fffffffffffffffull;
            if (ab == 0ull || ab > 0x7ff0000000000000ull) continue;  // zero or NaN
            if (!cand_better(ab, j, kb[3], kj[3])) continue;
            kb[3] = ab;
            kj[3] = j;
#pragma unroll
            for (int q = 3; q > 0; --q) {
                if (cand_better(kb[q], kj[q], kb[q - 1], kj[q - 1])) {
                    const unsigned long long tb = kb[q];
                    kb[q] = kb[q - 1];
                    kb[q - 1] = tb;
                    const int32_t tj = kj[q];
                    kj[q] = kj[q - 1];
                    kj[q - 1] = tj;
                }
            }
        }
        for (int u = 0; u < s; ++u) {
            unsigned long long best = kb[0];
            int32_t bestj = kj[0];
#pragma unroll
            for (int off = GL / 2; off > 0; off >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(gmask, best, off, GL);
                const int32_t oj = __shfl_xor_sync(gmask, bestj, off, GL);
                if (cand_better(ob, oj, best, bestj)) {
                    best = ob;
                    bestj = oj;
                }
            }
            if (best == 0ull) break;
            if (kb[0] == best && kj[0] == bestj) {  // the owner drops its head
                kb[0] = kb[1];
                kj[0] = kj[1];
                kb[1] = kb[2];
                kj[1] = kj[2];
                kb[2] = kb[3];
                kj[2] = kj[3];
                kb[3] = 0ull;
                kj[3] = INT_MAX;
            }
            if (sub == 0) newj[npick] = bestj;
            ++npick;
        }
        __syncwarp(gmask);
        return npick;
    }
    for (int u = 0; u < s; ++u) {
        unsigned long long best = 0ull;
        int32_t bestj = INT_MAX;
        int bslot = -1;
        for (int t = sub; t < nk; t += GL) {
            const int sl = list[t];
            const int32_t j = key[sl];
            const unsigned long long ab =
                static_cast<unsigned long long>(__double_as_longlong(hv[sl])) & 0x7fffffffffffffffull;
            if (ab == 0ull || ab > 0x7ff0000000000000ull) continue;  // zero or NaN
            if (cand_better(ab, j, best, bestj)) {
                best = ab;
                bestj = j;
                bslot = sl;
            }
        }
#pragma unroll
        for (int off = GL / 2; off > 0; off >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(gmask, best, off, GL);
            const int32_t oj = __shfl_xor_sync(gmask, bestj, off, GL);
            const int os = __shfl_xor_sync(gmask, bslot, off, GL);
            if (cand_better(ob, oj, best, bestj)) {
                best = ob;
                bestj = oj;
                bslot = os;
            }
        }
        if (best == 0ull) break;
        if (sub == 0) {
            hv[bslot] = 0.0;
            newj[npick] = bestj;
        }
        ++npick;
        __syncwarp(gmask);
    }
    return npick;
}

template <int GL, int MCAP, int HT, bool CHOL32>
__device__ void afsai_row(const SetupArgs& a, int32_t i, WarpWs<MCAP, HT>& w, int32_t* key, double* hv,
                          int32_t* list, int log2, int sub, unsigned gmask, const uint16_t* pairs) {
    const int ht = 1 << log2;
    const int32_t* __restrict__ colA = a.col;
    const double* __restrict__ valA = a.val;
    // a_ii (validated present and positive)
    double aii = 0.0;
    {
        const int32_t e0 = a.rowptr[i], e1 = a.rowptr[i + 1];
        bool found = false;
        for (int32_t e = e0 + sub; e < e1; e += GL)
            if (__ldg(&colA[e]) == i) {
                aii = __ldg(&valA[e]);
                found = true;
            }
        const unsigned bal = __ballot_sync(gmask, found) & gmask;
        aii = __shfl_sync(gmask, aii, bal ? ((__ffs(bal) - 1) & (GL - 1)) : 0, GL);
        if (!bal) aii = 0.0;
        if (sub == 0) {
            w.P[0] = i;
            w.g[0] = 1.0 / aii;
            w.Mraw[0] = aii;
            w.rb[0] = e0;
            w.re[0] = e1;
        }
    }
    __syncwarp(gmask);
    int m = 1;
    const double psi0 = aii;
    double psi_prev = psi0;
    int steps = 0;
    int32_t status = positive(aii) ? kRowOk : kRowNotSpd;
    const StripeBound bd = stripe_bound(a.reach, a.reach_words, a.stripe_magic, a.stripe_shift, i);

    for (int k = 1; k <= a.kiter && status == kRowOk; ++k) {
        // ---- Kaporin gradient over j < i (Eq. "grapsi") ----
        for (int t = sub; t < ht; t += GL) {
            key[t] = -1;
            hv[t] = 0.0;
        }
        int nkr = 0;  // keys in the table, equal in every lane
        __syncwarp(gmask);
        bool ovf = false;
        {
            // rows r in P ascending; the next row's entries are loaded while
            // the current one is accumulated
            constexpr int NPF = HT <= 256 ? 1 : 4;
            RowPref<NPF> RA, RB;
            prefetch_row<GL, NPF>(RA, colA, valA, w.rb[0], w.re[0], sub);
            for (int t = 0; t < m; t += 2) {
                if (t + 1 < m) prefetch_row<GL, NPF>(RB, colA, valA, w.rb[t + 1], w.re[t + 1], sub);
                accumulate_row<GL, NPF>(RA, colA, valA, w.rb[t], w.re[t], i, w.g[t], key, hv, list, log2, nkr, ovf,
                                        sub, gmask);
                __syncwarp(gmask);
                if (t + 1 < m) {
                    if (t + 2 < m) prefetch_row<GL, NPF>(RA, colA, valA, w.rb[t + 2], w.re[t + 2], sub);
                    accumulate_row<GL, NPF>(RB, colA, valA, w.rb[t + 1], w.re[t + 1], i, w.g[t + 1], key, hv, list, log2,
                                            nkr, ovf, sub, gmask);
                    __syncwarp(gmask);
                }
            }
        }
        if (__any_sync(gmask, ovf)) {
            status = kRowOverflow;
            break;
        }
        // members of P are not eligible: zero their accumulated gradient
        for (int t = sub; t < m - 1; t += GL) {
            const int slot = table_find(key, log2, w.P[t]);
            if (slot >= 0) hv[slot] = 0.0;
        }
        __syncwarp(gmask);
        const int nk = nkr;
        apply_stripe_bound(bd, key, hv, list, nk, sub, GL, gmask);
        // ---- select the s largest |gradient| (ties: smaller column) ----
        const int npick = select_top_s<GL>(key, hv, list, nk, a.s, sub, gmask, w.newj);
        if (npick == 0) break;

        // ---- merge into the sorted pattern; move the gathered triangle ----
        const int mold = m;
        m += npick;
        ++steps;
        // old triangle -> scratch (the hash table is dead from here on)
        double* scratch = w.u.f.L;
        const int told = tri(mold);
        for (int t = sub; t < told; t += GL) scratch[t] = w.Mraw[t];
        __syncwarp(gmask);
        // new positions: an old entry moves up by the number of picks below
        // it; a pick lands after the old entries and the picks below it
        for (int t = sub; t < mold; t += GL) {
            const int32_t pt = w.P[t];
            int up = 0;
            for (int u = 0; u < npick; ++u) up += w.newj[u] < pt;
            w.opos[t] = t + up;
            w.Pn[t + up] = pt;
            w.rbn[t + up] = w.rb[t];
            w.ren[t + up] = w.re[t];
        }
        for (int u = sub; u < npick; u += GL) {
            const int32_t j = w.newj[u];
            int below = 0;
            for (int q = 0; q < npick; ++q) below += w.newj[q] < j;
            int lo = 0, hi = mold;  // old entries below j
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (w.P[mid] < j)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            w.Pn[lo + below] = j;
            w.rbn[lo + below] = -1;  // marks a new position
        }
        __syncwarp(gmask);
        for (int t = sub; t < m; t += GL) {
            w.P[t] = w.Pn[t];
            w.isnew[t] = w.rbn[t] < 0 ? 1 : 0;
            w.rb[t] = w.rbn[t];
            w.re[t] = w.ren[t];
        }
        __syncwarp(gmask);
        const int tnew = tri(m);
        for (int t = sub; t < tnew; t += GL) w.Mraw[t] = 0.0;
        // row bounds of the new rows
        for (int t = sub; t < m; t += GL)
            if (w.isnew[t]) {
                w.rb[t] = a.rowptr[w.P[t]];
                w.re[t] = a.rowptr[w.P[t] + 1];
            }
        __syncwarp(gmask);
        // old entries to their new positions (the order of old indices is kept)
        for (int t = sub; t < told; t += GL) {
            const int pr = pairs[t];
            w.Mraw[tri(w.opos[pr >> 8]) + w.opos[pr & 0xff]] = scratch[t];
        }
        __syncwarp(gmask);
        // ---- systems gather: rows of the new indices (A symmetric) ----
        for (int pj = 0; pj < m; ++pj) {
            if (!w.isnew[pj]) continue;
            const int32_t e0 = w.rb[pj], e1 = w.re[pj];
            for (int32_t e = e0 + sub; e < e1; e += GL) {
                const int32_t c = __ldg(&colA[e]);
                const double v = __ldg(&valA[e]);
                const int pc = find_sorted(w.P, m, c);
                if (pc < 0) continue;
                if (pc <= pj)
                    w.Mraw[tri(pj) + pc] = v;
                else if (!w.isnew[pc])
                    w.Mraw[tri(pc) + pj] = v;
            }
        }
        __syncwarp(gmask);

        // ---- dense solve A[P,P] g = e_m ----
        if (!CHOL32) {
            double* L = w.u.f.L;
            for (int t = sub; t < tnew; t += GL) L[t] = w.Mraw[t];
            __syncwarp(gmask);
            if (!group_cholesky<GL, double>(L, m, sub, gmask, pairs)) {
                status = kRowNotSpd;
                break;
            }
            group_llt_solve<GL, double>(L, w.g, m, true, sub, gmask);
        } else {
            float* Lf = w.u.f.Lf;
            for (int t = sub; t < tnew; t += GL) Lf[t] = static_cast<float>(w.Mraw[t]);
            __syncwarp(gmask);
            if (!group_cholesky<GL, float>(Lf, m, sub, gmask, pairs)) {
                status = kRowNotSpd;
                break;
            }
            float* xf = reinterpret_cast<float*>(w.newj);  // m floats of scratch
            group_llt_solve<GL, float>(Lf, xf, m, true, sub, gmask);
            for (int t = sub; t < m; t += GL) w.g[t] = static_cast<double>(xf[t]);
            __syncwarp(gmask);
            // one FP64 refinement step: res = e_m - A[P,P] g (symmetric, lower stored)
            for (int r = sub; r < m; r += GL) {
                double acc = (r == m - 1) ? 1.0 : 0.0;
                for (int q = 0; q < m; ++q) {
                    const double arq = (q <= r) ? w.Mraw[tri(r) + q] : w.Mraw[tri(q) + r];
                    acc = fma(-arq, w.g[q], acc);
                }
                xf[r] = static_cast<float>(acc);
            }
            __syncwarp(gmask);
            group_llt_solve<GL, float>(Lf, xf, m, false, sub, gmask);
            for (int t = sub; t < m; t += GL) w.g[t] = w.g[t] + static_cast<double>(xf[t]);
            __syncwarp(gmask);
        }
        const double psi = 1.0 / w.g[m - 1];
        const bool stop = (a.exit_mode == 0) ? ((psi_prev - psi) < a.eps * psi_prev) : ((psi / psi0) <= a.eps);
        psi_prev = psi;
        if (stop) break;
    }

    if (status == kRowOk) {
        const double sq = sqrt(w.g[m - 1]);
        const int64_t o = static_cast<int64_t>(i) * a.mcap;
        for (int t = sub; t < m; t += GL) {
            a.out_col[o + t] = w.P[t];
            a.out_val[o + t] = w.g[t] / sq;
        }
        if (sub == 0) {
            a.out_len[i] = m;
            a.psi[i] = psi_prev;
            a.steps[i] = steps;
            a.status[i] = kRowOk;
        }
    } else if (sub == 0) {
        a.out_len[i] = 0;
        a.status[i] = status;
        if (status == kRowOverflow) {
            const int32_t slot = atomicAdd(&a.counters[0], 1);
            a.retry_rows[slot] = i;
        } else {
            atomicAdd(&a.counters[1], 1);
        }
    }
    __syncwarp(gmask);
}

template <int GL, int MCAP, int HT, bool GTABLE, bool CHOL32>
__global__ void __launch_bounds__(kSetupThreads) afsai_setup_kernel(SetupArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using WS = WarpWs<MCAP, HT>;
    constexpr int kPairs = MCAP * (MCAP + 1) / 2;
    const int ngroup_blk = blockDim.x / GL;
    const int group = threadIdx.x / GL;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (GL - 1);
    const unsigned gmask = (GL == 32) ? 0xffffffffu : (((1u << GL) - 1u) << (lane & ~(GL - 1)));
    WS* ws = reinterpret_cast<WS*>(smem_raw);
    uint16_t* pairs = reinterpret_cast<uint16_t*>(ws + ngroup_blk);
    // (rr, qq) of a packed triangle, shared by the block
    for (int idx = threadIdx.x; idx < kPairs; idx += blockDim.x) {
        int r = static_cast<int>((sqrtf(8.0f * static_cast<float>(idx) + 1.0f) - 1.0f) * 0.5f);
        if (tri(r + 1) <= idx) ++r;
        if (tri(r) > idx) --r;
        pairs[idx] = static_cast<uint16_t>((r << 8) | (idx - tri(r)));
    }
    __syncthreads();
    WS& w = ws[group];
    const int64_t ggroup = static_cast<int64_t>(blockIdx.x) * ngroup_blk + group;
    const int64_t ngroups = static_cast<int64_t>(gridDim.x) * ngroup_blk;
    int32_t* key;
    double* hv;
    int32_t* list;
    int log2;
    if (GTABLE) {
        key = a.gkey + (ggroup << a.ght_log2);
        hv = a.gval + (ggroup << a.ght_log2);
        list = a.glist + (ggroup << a.ght_log2);
        log2 = a.ght_log2;
    } else {
        key = w.u.h.key;
        hv = w.u.h.val;
        list = w.u.h.list;
        log2 = __ffs(HT) - 1;
    }
    const int64_t nrows = a.rows ? a.nrows : a.n;
    for (int64_t t = ggroup; t < nrows; t += ngroups) {
        const int32_t i = a.rows ? a.rows[t] : static_cast<int32_t>(t);
        afsai_row<GL, MCAP, HT, CHOL32>(a, i, w, key, hv, list, log2, sub, gmask, pairs);
    }
}

// Shared memory per warp: the union must also hold the FP64 triangle plus
// an FP32 copy of it for the FP32 factorisation.
template <int MCAP, int HT>
constexpr size_t ws_bytes() {
    return sizeof(WarpWs<MCAP, HT>);
}

template <int GL, int MCAP, int HT, bool GTABLE, bool CHOL32>
afsai_status launch_setup(const SetupArgs& a, int64_t nrows, int64_t max_groups, cudaStream_t st) {
    auto kern = afsai_setup_kernel<GL, MCAP, HT, GTABLE, CHOL32>;
    // block size (whole warps, <= 256 threads) that maximises resident row
    // groups per SM under the shared-memory budget
    const size_t per_group = ws_bytes<MCAP, HT>();
    const size_t pairs_bytes = (sizeof(uint16_t) * (MCAP * (MCAP + 1) / 2) + 15) / 16 * 16;
    const size_t sm_budget = 227u * 1024u;
    int groups_blk = 32 / GL;
    int best_total = 0;
    for (int gb = 32 / GL; gb <= kSetupThreads / GL; gb += 32 / GL) {
        const size_t blk = per_group * gb + pairs_bytes + 1024;  // + reserved per block
        if (blk > sm_budget) break;
        const int per = static_cast<int>(std::min<size_t>(sm_budget / blk, 2048 / (gb * GL)));
        if (per * gb > best_total) {
            best_total = per * gb;
            groups_blk = gb;
        }
    }
    const int threads = groups_blk * GL;
    const size_t smem = per_group * groups_blk + pairs_bytes;
    AFSAI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int per_sm = 0;
    AFSAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return fail(AFSAI_ENOTSUP, "set-up workspace does not fit in shared memory");
    int64_t blocks = static_cast<int64_t>(per_sm) * num_sms();
    const int64_t need = (nrows + groups_blk - 1) / groups_blk;
    if (blocks > need) blocks = need;
    if (blocks * groups_blk > max_groups) blocks = max_groups / groups_blk;  // global table capacity
    if (blocks < 1) blocks = 1;
    kern<<<static_cast<unsigned>(blocks), threads, smem, st>>>(a);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFSAI_OK;
}

template <int GL, int MCAP, int HT>
afsai_status dispatch_chol(const SetupArgs& a, int64_t nrows, int64_t max_groups, bool gtable, bool chol32,
                          cudaStream_t st) {
    if (gtable)
        return chol32 ? launch_setup<GL, MCAP, HT, true, true>(a, nrows, max_groups, st)
                      : launch_setup<GL, MCAP, HT, true, false>(a, nrows, max_groups, st);
    return chol32 ? launch_setup<GL, MCAP, HT, false, true>(a, nrows, max_groups, st)
                  : launch_setup<GL, MCAP, HT, false, false>(a, nrows, max_groups, st);
}

// Lanes per row.  The row code is written for groups of GL lanes, but only
// whole warps are instantiated: groups packed into one warp diverge and
// lose more than the shared square roots and divisions gain.
template <int MCAP, int HT>
afsai_status dispatch_gl(int gl, const SetupArgs& a, int64_t nrows, int64_t max_groups, bool gtable, bool chol32,
                         cudaStream_t st) {
    (void)gl;  // one warp per row (packing rows into a warp measured slower: the groups diverge)
    return dispatch_chol<32, MCAP, HT>(a, nrows, max_groups, gtable, chol32, st);
}

afsai_status dispatch(int mcap_t, int ht, int gl, const SetupArgs& a, int64_t nrows, int64_t max_groups, bool gtable,
                      bool chol32, cudaStream_t st) {
    switch (mcap_t) {
        case 16:
            return ht == 256 ? dispatch_gl<16, 256>(gl, a, nrows, max_groups, gtable, chol32, st)
                             : dispatch_gl<16, 512>(gl, a, nrows, max_groups, gtable, chol32, st);
        case 20:
            return ht == 256 ? dispatch_gl<20, 256>(gl, a, nrows, max_groups, gtable, chol32, st)
                             : dispatch_gl<20, 512>(gl, a, nrows, max_groups, gtable, chol32, st);
        case 32:
            return ht == 256 ? dispatch_gl<32, 256>(gl, a, nrows, max_groups, gtable, chol32, st)
                             : dispatch_gl<32, 512>(gl, a, nrows, max_groups, gtable, chol32, st);
        case 64:
            return dispatch_chol<32, 64, 512>(a, nrows, max_groups, gtable, chol32, st);
        case 128:
            return dispatch_chol<32, 128, 512>(a, nrows, max_groups, gtable, chol32, st);
        default:
            return fail(AFSAI_ENOTSUP, "pattern capacity above 128");
    }
}

// Per-row compaction into CSR with value conversion, and the longest row.
// A warp takes 32 consecutive rows, whose CSR entries form one contiguous
// range: lane l handles entries l, l + 32, ... of the range and finds its
// row by a binary search over the 32 row starts, so that the writes are
// coalesced and every lane works whatever the row lengths.
template <typename VT>
__global__ void __launch_bounds__(256) compact_rows_kernel(int32_t n, int64_t mcap, const int32_t* __restrict__ len,
                                                           const int32_t* __restrict__ ocol,
                                                           const double* __restrict__ oval,
                                                           const int32_t* __restrict__ rowptr,
                                                           int32_t* __restrict__ col, VT* __restrict__ val,
                                                           int32_t* __restrict__ maxrow) {
    __shared__ int32_t srp[8][33];  // row starts of each warp's rows (blockDim.x == 256)
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    int localmax = 0;
    for (int64_t r0 = gw * 32; r0 < n; r0 += nw * 32) {
        const int nr = static_cast<int>(n - r0 < 32 ? n - r0 : 32);
        const int32_t end = rowptr[r0 + nr];
        srp[w][lane] = lane < nr ? rowptr[r0 + lane] : end;
        if (lane == 0) srp[w][32] = end;
        if (lane < nr) localmax = max(localmax, len[r0 + lane]);
        __syncwarp();
        for (int32_t k = srp[w][0] + lane; k < end; k += 32) {
            int q = 0;  // the last row starting at or before k (empty rows are skipped)
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (srp[w][q + step] <= k) q += step;
            const int64_t src = (r0 + q) * mcap + (k - srp[w][q]);
            col[k] = ocol[src];
            val[k] = static_cast<VT>(oval[src]);
        }
        __syncwarp();
    }
    if (lane == 0 && localmax > 0) atomicMax(maxrow, localmax);
}

// ---------------------------------------------------------------------------
// Stepwise set-up (patterns of up to 32 entries).
//
// The fused kernel spends its FP64 issue slots on per-column square roots
// and divisions with few useful lanes (a warp-wide FP64 division or square
// root costs the same whatever the number of active lanes).  Here every
// step k runs as two kernels, the structure of the paper's Section 3
// (gradient + selection + systems gather, then batched Cholesky):
//   A  step_gather, one warp per active row: Kaporin gradient, top-s
//      selection, merge, and the gather of A[P,P] into a per-row slot in
//      global memory (full, or incremental from the previous step's slot);
//   B  the row's Cholesky, triangular solves, psi and the exit test, in the
//      exact sequential order of the plain definition, with several rows
//      per warp: step_solve_wide (LPR lanes per row, 32 / LPR rows per
//      warp) or step_solve (one lane per row).
// Row state (P, g, psi, step count, status) lives in global memory between
// the kernels.  Results are bit-identical to the fused kernel.
// ---------------------------------------------------------------------------
constexpr int32_t kStActive = 0;   // in the loop, no system pending
constexpr int32_t kStSolve = 1;    // system gathered, solve pending
constexpr int32_t kStStop = 2;     // finished (exit test or no candidates)

struct StepArgs {
    int32_t n;
    const int32_t* __restrict__ rowptr;
    const int32_t* __restrict__ col;
    const double* __restrict__ val;
    int32_t s;
    int32_t exit_mode;
    double eps;
    int32_t mc;   // row stride of P and g
    int32_t tmc;  // row stride of the gathered triangle
    int32_t* P;
    double* g;
    double* M;
    int32_t* m;
    int32_t* steps;
    int32_t* st;
    double* psi;
    double* psi0;
    const uint32_t* reach;  // locality bound, as in SetupArgs
    int32_t reach_words;
    int32_t stripe_shift;
    uint64_t stripe_magic;
    // rows still active after the previous step: list[0 .. *count) (null
    // before the first step)
    const int32_t* list;
    const int32_t* count;
};

// The rows a step's kernels visit: the active list once at most 3/4 of the
// rows remain, else every row (skipping the finished ones).  The list adds
// a dependent load to each row's chain of loads and gives up the row
// order; on the 7-point diffusion problem (78-100% of the rows active at
// every step) visiting every row measured faster.
struct StepRows {
    const int32_t* list;
    int64_t count;
    __device__ __forceinline__ int64_t row(int64_t q) const { return list ? list[q] : q; }
};
__device__ __forceinline__ StepRows step_rows(const StepArgs& a) {
    if (a.list) {
        const int64_t c = *a.count;
        if (4 * c <= 3 * static_cast<int64_t>(a.n)) return StepRows{a.list, c};
    }
    return StepRows{nullptr, a.n};
}

// The rows of `in` (every row when `in` is null) that are still active
// after a step's solve, appended to `out` (*out_count zeroed before).  Each
// block keeps the order of its blockDim.x entries (warp ballots and a scan
// of the block's warp counts) and appends them with one atomic (one per
// warp put every warp of the GPU on the same counter); blocks append in any
// order, which changes no result (rows are independent) and keeps runs of
// neighbouring rows together for the gathers from A.  blockDim.x is a
// multiple of 32, at most 1024.
__global__ void step_compact(int32_t n, const int32_t* __restrict__ in, const int32_t* __restrict__ in_count,
                             const int32_t* __restrict__ st, int32_t* __restrict__ out, int32_t* out_count) {
    __shared__ int32_t wbase[32];
    __shared__ int32_t bbase;
    const int64_t cnt = in ? *in_count : n;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; t0 < cnt;
         t0 += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t q = t0 + threadIdx.x;
        const int32_t i = q < cnt ? (in ? in[q] : static_cast<int32_t>(q)) : -1;
        const bool keep = i >= 0 && st[i] == kStActive;
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wbase[warp] = __popc(mask);
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t tot = 0;
            for (int w = 0; w < nwarps; ++w) {
                const int32_t c = wbase[w];
                wbase[w] = tot;
                tot += c;
            }
            bbase = tot > 0 ? atomicAdd(out_count, tot) : 0;
        }
        __syncthreads();
        if (keep) out[bbase + wbase[warp] + __popc(mask & ((1u << lane) - 1u))] = i;
        __syncthreads();  // wbase and bbase are rewritten for the next rows
    }
}

__global__ void step_init(StepArgs a) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double aii = 0.0;
        for (int32_t e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e)
            if (a.col[e] == i) aii = a.val[e];
        a.P[i * a.mc] = static_cast<int32_t>(i);
        a.g[i * a.mc] = rn::div_rn(1.0, rn::make_divisor(aii));  // the IEEE quotient, on the integer pipes
        if (a.M) a.M[i * a.tmc] = aii;  // the 1 x 1 system, extended incrementally
        a.m[i] = 1;
        a.steps[i] = 0;
        a.psi[i] = aii;
        a.psi0[i] = aii;
        a.st[i] = positive(aii) ? kStActive : kRowNotSpd;
    }
}

template <int MC, int HT>
struct GatherWs {
    double g[MC];
    int32_t P[MC];
    int32_t newj[MC];
    int32_t Pn[MC];
    int32_t rb[MC];
    int32_t re[MC];
    int32_t opos[MC];   // new position of each old position (incremental gather)
    int32_t isnew[MC];  // 1 for positions inserted this step
    int32_t pad_[2];
    // the candidate table is dead once the step's picks are made; the
    // gathered system is built in the same space (the next row clears the
    // table again)
    union {
        struct {
            double val[HT];
            int32_t key[HT];
            int32_t list[HT];
        };
        double Mw[MC * (MC + 1) / 2];
    };
};

// INC: the gathered system is extended incrementally (the previous step's
// raw triangle is read back from a.M, moved to the new positions, and only
// the rows of the new indices of A are read), as in the fused kernel; else
// A[P,P] is gathered in full from the rows of P.
// GL lanes per row (32 / GL rows per warp, each group with its own
// workspace and candidate table): the work of one row is small next to a
// warp (the 7-point rows of a pattern of at most 11 entries give at most 77
// candidate entries per step), so packing rows shares the per-row fixed
// cost of every warp instruction.  Groups of one warp take consecutive
// rows, whose patterns have the same shape on a structured grid.
template <int MC, int HT, bool INC, int GL = 32>
__global__ void __launch_bounds__(256) step_gather(StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using WS = GatherWs<MC, HT>;
    static_assert(GL == 4 || GL == 8 || GL == 16 || GL == 32, "lanes per row");
    const int group = threadIdx.x / GL;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (GL - 1);
    const unsigned gmask = (GL == 32) ? 0xffffffffu : (((1u << GL) - 1u) << (lane & ~(GL - 1)));
    WS& w = reinterpret_cast<WS*>(smem_raw)[group];
    constexpr int log2 = HT == 64 ? 6 : (HT == 128 ? 7 : (HT == 256 ? 8 : 9));
    static_assert((1 << log2) == HT, "table size");
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * (blockDim.x / GL) + group;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * (blockDim.x / GL);
    const StepRows rows = step_rows(a);
    for (int64_t q = gw; q < rows.count; q += nw) {
        const int64_t ii = rows.row(q);
        if (a.st[ii] != kStActive) continue;
        const int32_t i = static_cast<int32_t>(ii);
        int m = a.m[i];
        for (int t = sub; t < m; t += GL) {
            w.P[t] = a.P[ii * a.mc + t];
            w.g[t] = a.g[ii * a.mc + t];
            w.rb[t] = a.rowptr[w.P[t]];
            w.re[t] = a.rowptr[w.P[t] + 1];
        }
        for (int t = sub; t < HT; t += GL) {
            w.key[t] = -1;
            w.val[t] = 0.0;
        }
        int nkr = 0;  // keys in the table, equal in every lane
        __syncwarp(gmask);
        // ---- Kaporin gradient over j < i (Eq. "grapsi") ----
        bool ovf = false;
        {
            constexpr int NPF = HT <= 256 ? 1 : 4;
            RowPref<NPF> RA, RB;
            prefetch_row<GL, NPF>(RA, a.col, a.val, w.rb[0], w.re[0], sub);
            for (int t = 0; t < m; t += 2) {
                if (t + 1 < m) prefetch_row<GL, NPF>(RB, a.col, a.val, w.rb[t + 1], w.re[t + 1], sub);
                accumulate_row<GL, NPF>(RA, a.col, a.val, w.rb[t], w.re[t], i, w.g[t], w.key, w.val, w.list, log2,
                                        nkr, ovf, sub, gmask);
                __syncwarp(gmask);
                if (t + 1 < m) {
                    if (t + 2 < m) prefetch_row<GL, NPF>(RA, a.col, a.val, w.rb[t + 2], w.re[t + 2], sub);
                    accumulate_row<GL, NPF>(RB, a.col, a.val, w.rb[t + 1], w.re[t + 1], i, w.g[t + 1], w.key, w.val,
                                            w.list, log2, nkr, ovf, sub, gmask);
                    __syncwarp(gmask);
                }
            }
        }
        if (__any_sync(gmask, ovf)) {
            if (sub == 0) a.st[i] = kRowOverflow;
            __syncwarp(gmask);
            continue;
        }
        for (int t = sub; t < m - 1; t += GL) {
            const int slot = table_find(w.key, log2, w.P[t]);
            if (slot >= 0) w.val[slot] = 0.0;
        }
        __syncwarp(gmask);
        const int nk = nkr;
        apply_stripe_bound(stripe_bound(a.reach, a.reach_words, a.stripe_magic, a.stripe_shift, i), w.key, w.val,
                           w.list, nk, sub, GL, gmask);
        // ---- select the s largest |gradient| (ties: smaller column) ----
        const int npick = select_top_s<GL>(w.key, w.val, w.list, nk, a.s, sub, gmask, w.newj);
        if (npick == 0) {
            if (sub == 0) a.st[i] = kStStop;
            __syncwarp(gmask);
            continue;
        }
        // ---- merge into the sorted pattern ----
        const int mold = m;
        for (int t = sub; t < mold; t += GL) {
            const int32_t pt = w.P[t];
            int up = 0;
            for (int u = 0; u < npick; ++u) up += w.newj[u] < pt;
            w.Pn[t + up] = pt;
            w.opos[t] = t + up;
            w.isnew[t + up] = 0;
        }
        for (int u = sub; u < npick; u += GL) {
            const int32_t j = w.newj[u];
            int below = 0;
            for (int q = 0; q < npick; ++q) below += w.newj[q] < j;
            int lo = 0, hi = mold;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (w.P[mid] < j)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            w.Pn[lo + below] = j;
            w.isnew[lo + below] = 1;
        }
        m = mold + npick;
        __syncwarp(gmask);
        for (int t = sub; t < m; t += GL) {
            const int32_t pt = w.Pn[t];
            w.P[t] = pt;
            a.P[ii * a.mc + t] = pt;
            w.rb[t] = a.rowptr[pt];
            w.re[t] = a.rowptr[pt + 1];
        }
        const int tm = tri(m);
        for (int t = sub; t < tm; t += GL) w.Mw[t] = 0.0;
        __syncwarp(gmask);
        if (INC) {
            // ---- systems gather, incremental: old entries to their new
            // positions, then the rows of the new indices (A symmetric) ----
            const int told = tri(mold);
            for (int t = sub; t < told; t += GL) {
                int r = static_cast<int>((sqrtf(8.0f * static_cast<float>(t) + 1.0f) - 1.0f) * 0.5f);
                if (tri(r + 1) <= t) ++r;
                if (tri(r) > t) --r;
                const int q = t - tri(r);
                w.Mw[tri(w.opos[r]) + w.opos[q]] = a.M[ii * a.tmc + t];
            }
            __syncwarp(gmask);
            for (int pj = 0; pj < m; ++pj) {
                if (!w.isnew[pj]) continue;
                for (int32_t e = w.rb[pj] + sub; e < w.re[pj]; e += GL) {
                    const int32_t c = __ldg(&a.col[e]);
                    const double v = __ldg(&a.val[e]);
                    const int pc = find_sorted(w.P, m, c);
                    if (pc < 0) continue;
                    if (pc <= pj)
                        w.Mw[tri(pj) + pc] = v;
                    else if (!w.isnew[pc])
                        w.Mw[tri(pc) + pj] = v;
                }
            }
        } else {
            // ---- systems gather: A[P,P], lower triangle, from the rows of P ----
            for (int r = 0; r < m; ++r) {
                const int32_t pr = w.P[r];
                for (int32_t e = w.rb[r] + sub; e < w.re[r]; e += GL) {
                    const int32_t c = __ldg(&a.col[e]);
                    const double v = __ldg(&a.val[e]);
                    if (c > pr) continue;
                    const int pc = find_sorted(w.P, r + 1, c);
                    if (pc >= 0) w.Mw[tri(r) + pc] = v;
                }
            }
        }
        __syncwarp(gmask);
        for (int t = sub; t < tm; t += GL) a.M[ii * a.tmc + t] = w.Mw[t];
        if (sub == 0) {
            a.m[i] = m;
            a.steps[i] += 1;
            a.st[i] = kStSolve;
        }
        __syncwarp(gmask);
    }
}

// ---------------------------------------------------------------------------
// Gather kernel for small stencils: one lane per row, 32 rows per warp.
// For rows of A with at most kLaneRowMax entries and patterns of at most 12
// entries (7-point and 5-point stencils with s <= 4), a row's step touches
// at most 11 x 8 entries of A and a few dozen distinct candidates, far too
// little work for a warp; here every warp instruction serves 32 rows.  Each
// lane owns a 48-slot open-addressing table in shared memory (lane-
// interleaved, so a warp's accesses fall in distinct banks) with its
// occupancy kept as a 64-bit mask in registers: no atomics, no clearing.
// Gradient, selection and merge are those of step_gather (same operation
// order: rows r in P ascending, each row in CSR order, acc = fma(a_rj, g_r,
// acc) from 0); the gathered system is not built here: the solve kernel
// reads A[P,P] from A itself (GATHER), so no system goes through HBM.
// A row whose candidates exceed 7/8 of the table is marked for the retry
// pass, as in the other kernels.
// ---------------------------------------------------------------------------
constexpr int kLaneHT = 48;
constexpr int kLaneRowMax = 8;

// Home slot of column j in a lane's table of HT slots (a multiplicative
// hash; HT need not be a power of two), and the next slot of a probe.
template <int HT>
__device__ __forceinline__ uint32_t lane_slot(int32_t j) {
    const uint32_t hsh = static_cast<uint32_t>(j) * 0x9E3779B1u;
    return static_cast<uint32_t>((static_cast<uint64_t>(hsh) * HT) >> 32);
}
template <int HT>
__device__ __forceinline__ uint32_t lane_next(uint32_t h) {
    return h + 1 == HT ? 0u : h + 1;
}

// Occupancy of a lane's table: one bit per slot, in registers.
template <int HT>
struct Occ {
    static constexpr int W = (HT + 63) / 64;
    uint64_t w[W];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int k = 0; k < W; ++k) w[k] = 0ull;
    }
    static_assert(W <= 2, "at most 128 slots");
    // selects instead of a dynamic index keep the words in registers
    __device__ __forceinline__ bool test(uint32_t h) const {
        const uint64_t x = (W == 2 && (h & 64u)) ? w[W - 1] : w[0];
        return (x >> (h & 63u)) & 1ull;
    }
    __device__ __forceinline__ void set(uint32_t h) {
        if (W == 2 && (h & 64u))
            w[W - 1] |= 1ull << (h & 63u);
        else
            w[0] |= 1ull << (h & 63u);
    }
};

template <int MC, int HT>
__global__ void __launch_bounds__(128) step_gather_lane(StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    static_assert(HT >= 32 && HT <= 128, "table size");
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nwb = blockDim.x >> 5;
    unsigned char* wbase = smem_raw + static_cast<size_t>(warp) * (HT * 12 + MC * 4) * 32;
    double* sv = reinterpret_cast<double*>(wbase);                    // val[HT]
    int32_t* sk = reinterpret_cast<int32_t*>(wbase + HT * 32 * 8);   // key[HT], P[MC]
#define TV(h) sv[(h) * 32 + lane]
#define TK(h) sk[(h) * 32 + lane]
#define TP(t) sk[(HT + (t)) * 32 + lane]
    const StepRows rows = step_rows(a);
    const int64_t ngroups = (rows.count + 31) / 32;
    for (int64_t grp = static_cast<int64_t>(blockIdx.x) * nwb + warp; grp < ngroups;
         grp += static_cast<int64_t>(gridDim.x) * nwb) {
        if (grp * 32 + lane >= rows.count) continue;
        const int64_t ii = rows.row(grp * 32 + lane);
        if (a.st[ii] != kStActive) continue;
        const int32_t i = static_cast<int32_t>(ii);
        const int m = a.m[ii];
        for (int t = 0; t < m; ++t) TP(t) = a.P[ii * a.mc + t];
        // ---- Kaporin gradient over j < i (Eq. "grapsi"); row t + 1 of A
        // is loaded while row t is accumulated ----
        Occ<HT> occ;
        occ.clear();
        int nk = 0;
        int32_t c0[kLaneRowMax], c1[kLaneRowMax];
        double v0[kLaneRowMax], v1[kLaneRowMax];
        double g0 = 0.0, g1 = 0.0;  // g_r of the current and the next row
        auto load_row = [&](int t, int32_t (&c)[kLaneRowMax], double (&v)[kLaneRowMax], double& gt) {
            gt = a.g[ii * a.mc + t];
            const int32_t r = TP(t);
            const int32_t rb = __ldg(&a.rowptr[r]), re = __ldg(&a.rowptr[r + 1]);
#pragma unroll
            for (int q = 0; q < kLaneRowMax; ++q) {
                const bool on = rb + q < re;
                c[q] = on ? __ldg(&a.col[rb + q]) : INT_MAX;
                v[q] = on ? __ldg(&a.val[rb + q]) : 0.0;
            }
        };
        load_row(0, c0, v0, g0);
        for (int t = 0; t < m; ++t) {
            if (t + 1 < m) load_row(t + 1, c1, v1, g1);
            const double gr = g0;
#pragma unroll
            for (int q = 0; q < kLaneRowMax; ++q) {
                const int32_t j = c0[q];
                if (j < i) {
                    uint32_t h = lane_slot<HT>(j);
                    for (int probe = 0; probe < HT; ++probe) {
                        if (!occ.test(h)) {
                            occ.set(h);
                            TK(h) = j;
                            TV(h) = 0.0;
                            ++nk;
                            break;
                        }
                        if (TK(h) == j) break;
                        h = lane_next<HT>(h);
                    }
                    TV(h) = fma(v0[q], gr, TV(h));
                }
            }
#pragma unroll
            for (int q = 0; q < kLaneRowMax; ++q) {
                c0[q] = c1[q];
                v0[q] = v1[q];
            }
            g0 = g1;
            if (nk > HT - (HT >> 3)) break;
        }
        if (nk > HT - (HT >> 3)) {
            a.st[ii] = kRowOverflow;
            continue;
        }
        // members of P are not eligible (i itself is never a candidate)
        for (int t = 0; t < m - 1; ++t) {
            const int32_t pj = TP(t);
            uint32_t h = lane_slot<HT>(pj);
            for (int probe = 0; probe < HT && occ.test(h); ++probe) {
                if (TK(h) == pj) {
                    TV(h) = 0.0;
                    break;
                }
                h = lane_next<HT>(h);
            }
        }
        // locality bound (Section 4): candidates outside the allowed stripes
        const StripeBound bd = stripe_bound(a.reach, a.reach_words, a.stripe_magic, a.stripe_shift, i);
        if (bd.row != nullptr) {
#pragma unroll
            for (int wd = 0; wd < Occ<HT>::W; ++wd)
                for (uint64_t mm = occ.w[wd]; mm; mm &= mm - 1) {
                    const uint32_t h = 64u * wd + static_cast<uint32_t>(__ffsll(static_cast<long long>(mm)) - 1);
                    if (!bd.allows(TK(h))) TV(h) = 0.0;
                }
        }
        // ---- the s (<= 4) largest |gradient|, ties to the smaller column ----
        unsigned long long kb[4] = {0ull, 0ull, 0ull, 0ull};
        int32_t kj[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
#pragma unroll
        for (int wd = 0; wd < Occ<HT>::W; ++wd)
            for (uint64_t mm = occ.w[wd]; mm; mm &= mm - 1) {
                const uint32_t h = 64u * wd + static_cast<uint32_t>(__ffsll(static_cast<long long>(mm)) - 1);
                const unsigned long long ab =
                    static_cast<unsigned long long>(__double_as_longlong(TV(h))) & 0x7fffffffffffffffull;
                if (ab == 0ull || ab > 0x7ff0000000000000ull) continue;  // zero or NaN
                const int32_t j = TK(h);
                if (!cand_better(ab, j, kb[3], kj[3])) continue;
                kb[3] = ab;
                kj[3] = j;
#pragma unroll
                for (int q = 3; q > 0; --q) {
                    if (cand_better(kb[q], kj[q], kb[q - 1], kj[q - 1])) {
                        const unsigned long long tb = kb[q];
                        kb[q] = kb[q - 1];
                        kb[q - 1] = tb;
                        const int32_t tj = kj[q];
                        kj[q] = kj[q - 1];
                        kj[q - 1] = tj;
                    }
                }
            }
        int npick = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < a.s && kb[q] != 0ull) ++npick;
        if (npick == 0) {
            a.st[ii] = kStStop;
            continue;
        }
        // picks in ascending column order (INT_MAX past npick)
        int32_t p0 = kj[0], p1 = npick > 1 ? kj[1] : INT_MAX, p2 = npick > 2 ? kj[2] : INT_MAX,
                p3 = npick > 3 ? kj[3] : INT_MAX;
#define CSWAP(x, y)                  \
    if ((y) < (x)) {                 \
        const int32_t t_ = (x);      \
        (x) = (y);                   \
        (y) = t_;                    \
    }
        CSWAP(p0, p1) CSWAP(p2, p3) CSWAP(p0, p2) CSWAP(p1, p3) CSWAP(p1, p2)
#undef CSWAP
        // ---- merge into the sorted pattern (i stays last) ----
        int ip = 0;
        const int mnew = m + npick;
        for (int o = 0; o < mnew; ++o) {
            const int32_t pa = ip < m ? TP(ip) : INT_MAX;
            int32_t out;
            if (p0 < pa) {
                out = p0;
                p0 = p1;
                p1 = p2;
                p2 = p3;
                p3 = INT_MAX;
            } else {
                out = pa;
                ++ip;
            }
            a.P[ii * a.mc + o] = out;
        }
        a.m[ii] = mnew;
        a.steps[ii] += 1;
        a.st[ii] = kStSolve;
    }
#undef TV
#undef TK
#undef TP
}

// A[P,P], lower triangle, of one row's system, gathered from the rows of
// its pattern: entry (P_t, c) of A with c <= P_t and c in P goes to packed
// position tri(t) + pos(c) (the gather of the plain definition; only the
// lower part of each row is read).  The LPR lanes of the row split the
// rows of P; rows of A have at most kLaneRowMax entries here.  Each lane
// first loads the row pointers of all its rows of P, then the entries of
// two rows at a time, so that its global loads are issued in a few
// independent batches rather than as one dependent chain per row (the
// kernel's shared memory, not its registers, bounds its occupancy).  Every
// entry has its own position, so the order of the puts changes nothing.
template <int LPR, int MC, typename F>
__device__ __forceinline__ void gather_rows_lower(const StepArgs& a, const int32_t* Ps, int m, int sub, F&& put) {
    constexpr int NT = (MC + LPR - 1) / LPR;  // rows of P per lane, at most
    constexpr int NT2 = (NT + 1) / 2 * 2;
    int32_t rb[NT2], re[NT2];
#pragma unroll
    for (int j = 0; j < NT2; ++j) {
        const int t = sub + j * LPR;
        rb[j] = 0;
        re[j] = 0;
        if (j < NT && t < m) {
            const int32_t pr = Ps[t];
            rb[j] = __ldg(&a.rowptr[pr]);
            re[j] = __ldg(&a.rowptr[pr + 1]);
        }
    }
#pragma unroll
    for (int j = 0; j < NT2; j += 2) {
        if (sub + j * LPR >= m) break;
        int32_t c[2][kLaneRowMax];
        double v[2][kLaneRowMax];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int q = 0; q < kLaneRowMax; ++q) {
                const bool on = rb[j + u] + q < re[j + u];
                c[u][q] = on ? __ldg(&a.col[rb[j + u] + q]) : INT_MAX;
                v[u][q] = on ? __ldg(&a.val[rb[j + u] + q]) : 0.0;
            }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = sub + (j + u) * LPR;
            if (t < m) {
                const int32_t pr = Ps[t];
#pragma unroll
                for (int q = 0; q < kLaneRowMax; ++q) {
                    if (c[u][q] <= pr) {
                        const int pc = find_sorted(Ps, t + 1, c[u][q]);
                        if (pc >= 0) put(tri(t) + pc, v[u][q]);
                    }
                }
            }
        }
    }
}

// One lane per row (FP64): Cholesky, solve, psi, exit test (plain
// sequential order), 32 rows per warp.
template <int MC>
__global__ void __launch_bounds__(64) step_solve(StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TMC = MC * (MC + 1) / 2;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nwb = blockDim.x >> 5;
    // lane-interleaved per-warp area: element e of lane l at [e * 32 + l];
    // MC extra words per lane for the prepared pivot reciprocals
    double* Ms = reinterpret_cast<double*>(smem_raw) + static_cast<size_t>(warp) * (TMC + 2 * MC) * 32;
    double* gs = Ms + TMC * 32;
    uint64_t* vs = reinterpret_cast<uint64_t*>(gs + MC * 32);
#define MS(e) Ms[(e) * 32 + lane]
#define GS(e) gs[(e) * 32 + lane]
#define VS(e) vs[(e) * 32 + lane]
    const StepRows rows = step_rows(a);
    const int64_t ngroups = (rows.count + 31) / 32;
    for (int64_t grp = static_cast<int64_t>(blockIdx.x) * nwb + warp; grp < ngroups;
         grp += static_cast<int64_t>(gridDim.x) * nwb) {
        if (grp * 32 + lane >= rows.count) continue;
        const int64_t ii = rows.row(grp * 32 + lane);
        if (a.st[ii] != kStSolve) continue;
        const int m = a.m[ii];
        const int tm = tri(m);
        for (int t = 0; t < tm; ++t) MS(t) = a.M[ii * a.tmc + t];
        bool spd = true;
        // square roots and divisions on the integer pipes (rn::, the IEEE
        // results bit for bit); each pivot's reciprocal is prepared once and
        // kept (VS) for the back substitution
        for (int c = 0; c < m && spd; ++c) {
            const double piv = MS(tri(c) + c);
            if (!positive(piv)) {
                spd = false;
                break;
            }
            const double d = rn::sqrt_rn(piv);
            MS(tri(c) + c) = d;
            const rn::Divisor dv = rn::make_divisor(d);
            VS(c) = dv.v;
            for (int r = c + 1; r < m; ++r) MS(tri(r) + c) = rn::div_rn(MS(tri(r) + c), dv);
            for (int r = c + 1; r < m; ++r)
                for (int q = c + 1; q <= r; ++q) MS(tri(r) + q) = fma(-MS(tri(r) + c), MS(tri(q) + c), MS(tri(r) + q));
        }
        if (spd) {
            for (int r = 0; r < m; ++r) GS(r) = 0.0;
            GS(m - 1) = rn::div_rn(1.0, rn::divisor_from(MS(tri(m - 1) + m - 1), VS(m - 1)));
            for (int c = m - 1; c >= 0; --c) {
                const double gc = rn::div_rn(GS(c), rn::divisor_from(MS(tri(c) + c), VS(c)));
                GS(c) = gc;
                for (int r = 0; r < c; ++r) GS(r) = fma(-MS(tri(c) + r), gc, GS(r));
            }
        }
        if (!spd) {
            a.st[ii] = kRowNotSpd;
            continue;
        }
        const double psi = 1.0 / GS(m - 1);
        const double psi_prev = a.psi[ii];
        const bool stop = (a.exit_mode == 0) ? ((psi_prev - psi) < a.eps * psi_prev) : ((psi / a.psi0[ii]) <= a.eps);
        a.psi[ii] = psi;
        for (int r = 0; r < m; ++r) a.g[ii * a.mc + r] = GS(r);
        a.st[ii] = stop ? kStStop : kStActive;
    }
#undef MS
#undef GS
#undef VS
}

// LPR lanes per row, 32 / LPR rows per warp: Cholesky, solve, psi, exit
// test of larger systems (up to MC = 32 entries), whose lane-per-row
// workspace would not fit shared memory.  Each FP64 square root and each
// back-substitution division serves all rows of the warp in one warp
// instruction, and each column's divisions are spread over the row's lanes,
// so a row pays a few FP64 division/square-root warp operations per column
// instead of three.  Per element the operations and their order are those
// of the plain definition (right-looking; element (r, q) updated by the
// columns c < q in ascending order; lanes only split the elements).  Each
// row's triangle lives in shared memory with an odd stride so that the same
// element of the warp's rows falls in different banks.
//
// The divisions run on the integer pipes (rn::, the IEEE results bit for
// bit), which relieves the FP64 pipe; the one square root per column stays
// the IEEE FP64 operation (measured faster here: the integer version's
// instructions cost more issue slots than the FP64 pipe time it saves).
// Each pivot's reciprocal is prepared once and kept for the back
// substitution.
// GATHER: the row's system is gathered here from A (gather_rows_lower)
// instead of being read from the gather kernel's slot; the pattern is then
// kept in the row's area too.
// SQRT_INT: the per-column square root on the integer pipes too (rn::);
// with 16 rows per warp the FP64 pipe, not issue, binds the kernel.
template <int MC, int LPR, bool GATHER = false, bool SQRT_INT = false>
__global__ void __launch_bounds__(128) step_solve_wide(StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TMC = MC * (MC + 1) / 2;
    constexpr int RPW = 32 / LPR;            // rows per warp
    // doubles per row (odd): L, g, prepared reciprocals (+ the pattern)
    constexpr int RS = (TMC + 2 * MC + (GATHER ? (MC + 1) / 2 : 0)) | 1;
    constexpr size_t kPairBytes = (sizeof(uint16_t) * TMC + 15) / 16 * 16;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int grp = lane / LPR;
    const int sub = lane % LPR;
    const int nwb = blockDim.x >> 5;
    uint16_t* pairs = reinterpret_cast<uint16_t*>(smem_raw);
    for (int idx = threadIdx.x; idx < TMC; idx += blockDim.x) {
        int r = static_cast<int>((sqrtf(8.0f * static_cast<float>(idx) + 1.0f) - 1.0f) * 0.5f);
        if (tri(r + 1) <= idx) ++r;
        if (tri(r) > idx) --r;
        pairs[idx] = static_cast<uint16_t>((r << 8) | (idx - tri(r)));
    }
    __syncthreads();
    double* wbase = reinterpret_cast<double*>(smem_raw + kPairBytes) + static_cast<size_t>(warp) * RPW * RS;
    double* M = wbase + grp * RS;  // this row's packed lower triangle
    double* g = M + TMC;           // this row's solution
    uint64_t* V = reinterpret_cast<uint64_t*>(g + MC);  // prepared pivot reciprocals
    const int64_t nrw = static_cast<int64_t>(gridDim.x) * nwb * RPW;
    const StepRows rows = step_rows(a);
    for (int64_t r0 = (static_cast<int64_t>(blockIdx.x) * nwb + warp) * RPW; r0 < rows.count; r0 += nrw) {
        const int64_t ii = r0 + grp < rows.count ? rows.row(r0 + grp) : a.n;
        const bool row = ii < a.n && a.st[ii] == kStSolve;
        const int m = row ? a.m[ii] : 0;
        if constexpr (GATHER) {
            int32_t* Ps = reinterpret_cast<int32_t*>(V + MC);
            if (row) {
                for (int t = sub; t < m; t += LPR) Ps[t] = a.P[ii * a.mc + t];
                for (int t = sub; t < tri(m); t += LPR) M[t] = 0.0;
            }
            __syncwarp();
            if (row) gather_rows_lower<LPR, MC>(a, Ps, m, sub, [&](int idx, double v) { M[idx] = v; });
        } else {
            // load the warp's triangles, one row at a time with all lanes
            for (int q = 0; q < RPW; ++q) {
                const int mq = __shfl_sync(0xffffffffu, m, q * LPR);
                const int64_t iq = __shfl_sync(0xffffffffu, ii, q * LPR);
                const int tq = tri(mq);
                double* Mq = wbase + q * RS;
                for (int t = lane; t < tq; t += 32) Mq[t] = a.M[iq * a.tmc + t];
            }
        }
        int mmax = m;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mmax = max(mmax, __shfl_xor_sync(0xffffffffu, mmax, o));
        __syncwarp();
        bool spd = true;
        for (int c = 0; c < mmax; ++c) {
            const bool act = spd && c < m;
            const double piv = act ? M[tri(c) + c] : 1.0;
            if (act && !positive(piv)) spd = false;
            // one warp operation for all rows
            const double d = SQRT_INT ? rn::sqrt_rn(piv) : sqrt(piv);
            const rn::Divisor dv = rn::make_divisor(d);
            if (act && spd)
                for (int r = c + 1 + sub; r < m; r += LPR) M[tri(r) + c] = rn::div_rn(M[tri(r) + c], dv);
            __syncwarp();
            if (act && spd) {
                if (sub == 0) {
                    M[tri(c) + c] = d;
                    V[c] = dv.v;
                }
                const int w = m - c - 1;
                const int T_ = (w * (w + 1)) >> 1;
                for (int idx = sub; idx < T_; idx += LPR) {
                    const int pr = pairs[idx];
                    const int r = c + 1 + (pr >> 8), q = c + 1 + (pr & 0xff);
                    M[tri(r) + q] = fma(-M[tri(r) + c], M[tri(q) + c], M[tri(r) + q]);
                }
            }
            __syncwarp();
        }
        // z = e_m / L_mm, back substitution L^T g = z (column oriented)
        for (int t = sub; t < m; t += LPR) g[t] = 0.0;
        __syncwarp();
        {
            const bool ok = row && spd;
            const double z = ok ? rn::div_rn(1.0, rn::divisor_from(M[tri(m - 1) + m - 1], V[m - 1])) : 0.0;
            if (ok && sub == 0) g[m - 1] = z;
        }
        __syncwarp();
        for (int t = 0; t < mmax; ++t) {
            const int c = m - 1 - t;
            const bool act = row && spd && c >= 0;
            const double gc = act ? rn::div_rn(g[c], rn::divisor_from(M[tri(c) + c], V[c])) : 0.0;
            __syncwarp();
            if (act) {
                if (sub == 0) g[c] = gc;
                for (int r = sub; r < c; r += LPR) g[r] = fma(-M[tri(c) + r], gc, g[r]);
            }
            __syncwarp();
        }
        if (row) {
            if (!spd) {
                if (sub == 0) a.st[ii] = kRowNotSpd;
            } else {
                const double psi = 1.0 / g[m - 1];
                const double psi_prev = a.psi[ii];
                const bool stop =
                    (a.exit_mode == 0) ? ((psi_prev - psi) < a.eps * psi_prev) : ((psi / a.psi0[ii]) <= a.eps);
                for (int t = sub; t < m; t += LPR) a.g[ii * a.mc + t] = g[t];
                if (sub == 0) {
                    a.psi[ii] = psi;
                    a.st[ii] = stop ? kStStop : kStActive;
                }
            }
        }
        __syncwarp();
    }
}

// The precision form of step_solve_wide: FP32 Cholesky and triangular
// solves (the pivot's reciprocal square root r = rsqrt(piv) gives
// L_cc = piv r and L_rc = M_rc r; the diagonal slots keep r), then one FP64
// refinement step res = e_m - A[P,P] g (FP64, from the raw triangle),
// L L^T d = res (FP32), g += d (FP64).  Same lanes and layout as
// step_solve_wide; each row keeps its raw FP64 triangle for the residual.
template <int MC, int LPR, bool GATHER = false>
__global__ void __launch_bounds__(128) step_solve_wide32(StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TMC = MC * (MC + 1) / 2;
    constexpr int RPW = 32 / LPR;
    // per row: raw triangle (double) + g (double) (+ the pattern) | factor
    // (float) + x (float)
    constexpr int RSD = (TMC + MC + (GATHER ? (MC + 1) / 2 : 0)) | 1;  // doubles
    constexpr int RSF = ((TMC + MC) | 1) + 1;    // floats (even count keeps 8-byte alignment)
    constexpr size_t kRowBytes = RSD * sizeof(double) + RSF * sizeof(float);
    constexpr size_t kPairBytes = (sizeof(uint16_t) * TMC + 15) / 16 * 16;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int grp = lane / LPR;
    const int sub = lane % LPR;
    const int nwb = blockDim.x >> 5;
    uint16_t* pairs = reinterpret_cast<uint16_t*>(smem_raw);
    for (int idx = threadIdx.x; idx < TMC; idx += blockDim.x) {
        int r = static_cast<int>((sqrtf(8.0f * static_cast<float>(idx) + 1.0f) - 1.0f) * 0.5f);
        if (tri(r + 1) <= idx) ++r;
        if (tri(r) > idx) --r;
        pairs[idx] = static_cast<uint16_t>((r << 8) | (idx - tri(r)));
    }
    __syncthreads();
    unsigned char* wbase = smem_raw + kPairBytes + static_cast<size_t>(warp) * RPW * kRowBytes;
    double* M = reinterpret_cast<double*>(wbase + grp * kRowBytes);  // raw A[P,P], packed lower
    double* g = M + TMC;
    float* L = reinterpret_cast<float*>(reinterpret_cast<double*>(wbase + grp * kRowBytes) + RSD);
    float* x = L + TMC;
    const int64_t nrw = static_cast<int64_t>(gridDim.x) * nwb * RPW;
    const StepRows rows = step_rows(a);
    for (int64_t r0 = (static_cast<int64_t>(blockIdx.x) * nwb + warp) * RPW; r0 < rows.count; r0 += nrw) {
        const int64_t ii = r0 + grp < rows.count ? rows.row(r0 + grp) : a.n;
        const bool row = ii < a.n && a.st[ii] == kStSolve;
        const int m = row ? a.m[ii] : 0;
        if constexpr (GATHER) {
            int32_t* Ps = reinterpret_cast<int32_t*>(g + MC);
            if (row) {
                for (int t = sub; t < m; t += LPR) Ps[t] = a.P[ii * a.mc + t];
                for (int t = sub; t < tri(m); t += LPR) {
                    M[t] = 0.0;
                    L[t] = 0.0f;
                }
            }
            __syncwarp();
            if (row)
                gather_rows_lower<LPR, MC>(a, Ps, m, sub, [&](int idx, double v) {
                    M[idx] = v;
                    L[idx] = static_cast<float>(v);
                });
        } else {
            for (int q = 0; q < RPW; ++q) {
                const int mq = __shfl_sync(0xffffffffu, m, q * LPR);
                const int64_t iq = __shfl_sync(0xffffffffu, ii, q * LPR);
                const int tq = tri(mq);
                double* Mq = reinterpret_cast<double*>(wbase + q * kRowBytes);
                float* Lq = reinterpret_cast<float*>(Mq + RSD);
                for (int t = lane; t < tq; t += 32) {
                    const double v = a.M[iq * a.tmc + t];
                    Mq[t] = v;
                    Lq[t] = static_cast<float>(v);
                }
            }
        }
        int mmax = m;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mmax = max(mmax, __shfl_xor_sync(0xffffffffu, mmax, o));
        __syncwarp();
        bool spd = true;
        for (int c = 0; c < mmax; ++c) {
            const bool act = spd && c < m;
            const float piv = act ? L[tri(c) + c] : 1.0f;
            if (act && !positive(piv)) spd = false;
            const float rinv = rsqrtf(piv);
            if (act && spd)
                for (int r = c + 1 + sub; r < m; r += LPR) L[tri(r) + c] = L[tri(r) + c] * rinv;
            __syncwarp();
            if (act && spd) {
                if (sub == 0) L[tri(c) + c] = rinv;
                const int w = m - c - 1;
                const int T_ = (w * (w + 1)) >> 1;
                for (int idx = sub; idx < T_; idx += LPR) {
                    const int pr = pairs[idx];
                    const int r = c + 1 + (pr >> 8), q = c + 1 + (pr & 0xff);
                    L[tri(r) + q] = fmaf(-L[tri(r) + c], L[tri(q) + c], L[tri(r) + q]);
                }
            }
            __syncwarp();
        }
        const bool ok = row && spd;
        // x = L^{-T} L^{-1} e_m (FP32)
        for (int t = sub; t < m; t += LPR) x[t] = 0.0f;
        __syncwarp();
        if (ok && sub == 0) x[m - 1] = L[tri(m - 1) + m - 1];
        __syncwarp();
        for (int t = 0; t < mmax; ++t) {
            const int c = m - 1 - t;
            const bool act = ok && c >= 0;
            const float gc = act ? x[c] * L[tri(c) + c] : 0.0f;
            __syncwarp();
            if (act) {
                if (sub == 0) x[c] = gc;
                for (int r = sub; r < c; r += LPR) x[r] = fmaf(-L[tri(c) + r], gc, x[r]);
            }
            __syncwarp();
        }
        for (int t = sub; t < m; t += LPR) g[t] = static_cast<double>(x[t]);
        __syncwarp();
        // one FP64 refinement step: res = e_m - A[P,P] g
        if (ok)
            for (int r = sub; r < m; r += LPR) {
                double acc = (r == m - 1) ? 1.0 : 0.0;
                for (int q = 0; q < m; ++q) {
                    const double arq = (q <= r) ? M[tri(r) + q] : M[tri(q) + r];
                    acc = fma(-arq, g[q], acc);
                }
                x[r] = static_cast<float>(acc);
            }
        __syncwarp();
        // L z = res (forward), L^T d = z (back), in x
        for (int c = 0; c < mmax; ++c) {
            const bool act = ok && c < m;
            const float zc = act ? x[c] * L[tri(c) + c] : 0.0f;
            __syncwarp();
            if (act) {
                if (sub == 0) x[c] = zc;
                for (int r = c + 1 + sub; r < m; r += LPR) x[r] = fmaf(-L[tri(r) + c], zc, x[r]);
            }
            __syncwarp();
        }
        for (int t = 0; t < mmax; ++t) {
            const int c = m - 1 - t;
            const bool act = ok && c >= 0;
            const float gc = act ? x[c] * L[tri(c) + c] : 0.0f;
            __syncwarp();
            if (act) {
                if (sub == 0) x[c] = gc;
                for (int r = sub; r < c; r += LPR) x[r] = fmaf(-L[tri(c) + r], gc, x[r]);
            }
            __syncwarp();
        }
        for (int t = sub; t < m; t += LPR) g[t] = g[t] + static_cast<double>(x[t]);
        __syncwarp();
        if (row) {
            if (!spd) {
                if (sub == 0) a.st[ii] = kRowNotSpd;
            } else {
                const double psi = 1.0 / g[m - 1];
                const double psi_prev = a.psi[ii];
                const bool stop =
                    (a.exit_mode == 0) ? ((psi_prev - psi) < a.eps * psi_prev) : ((psi / a.psi0[ii]) <= a.eps);
                for (int t = sub; t < m; t += LPR) a.g[ii * a.mc + t] = g[t];
                if (sub == 0) {
                    a.psi[ii] = psi;
                    a.st[ii] = stop ? kStStop : kStActive;
                }
            }
        }
        __syncwarp();
    }
}

// Final scaling and output slots (same layout as the fused kernel).
__global__ void step_finish(StepArgs a, SetupArgs o) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t stv = a.st[i];
        if (stv == kStActive || stv == kStStop) {
            const int m = a.m[i];
            const double sq = sqrt(a.g[i * a.mc + m - 1]);
            // the row's divisions on the integer pipes (rn::, the IEEE
            // quotients bit for bit) with one prepared divisor: as FP64
            // divisions they kept this kernel FP64-pipe bound
            const rn::Divisor dv = rn::make_divisor(sq);
            for (int t = 0; t < m; ++t) {
                o.out_col[i * o.mcap + t] = a.P[i * a.mc + t];
                o.out_val[i * o.mcap + t] = rn::div_rn(a.g[i * a.mc + t], dv);
            }
            o.out_len[i] = m;
            o.psi[i] = a.psi[i];
            o.steps[i] = a.steps[i];
            o.status[i] = kRowOk;
        } else {
            o.out_len[i] = 0;
            o.status[i] = stv;
            if (stv == kRowOverflow) {
                const int32_t slot = atomicAdd(&o.counters[0], 1);
                o.retry_rows[slot] = static_cast<int32_t>(i);
            } else {
                atomicAdd(&o.counters[1], 1);
            }
        }
    }
}

// kiter = 0 (the diagonal pattern, G = diag(A)^{-1/2}: Jacobi): one thread
// per row, the same operations as the init and the final scaling of the
// other paths (g = 1 / a_ii, G_ii = g / sqrt(g), psi = a_ii).
__global__ void k_setup_diagonal(SetupArgs o) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double aii = 0.0;
        for (int32_t e = o.rowptr[i]; e < o.rowptr[i + 1]; ++e)
            if (o.col[e] == i) aii = o.val[e];
        if (positive(aii)) {
            // IEEE quotients on the integer pipes (rn::), as in the other paths
            const double g = rn::div_rn(1.0, rn::make_divisor(aii));
            o.out_col[i * o.mcap] = static_cast<int32_t>(i);
            o.out_val[i * o.mcap] = rn::div_rn(g, rn::make_divisor(sqrt(g)));
            o.out_len[i] = 1;
            o.psi[i] = aii;
            o.steps[i] = 0;
            o.status[i] = kRowOk;
        } else {
            o.out_len[i] = 0;
            o.status[i] = kRowNotSpd;
            atomicAdd(&o.counters[1], 1);
        }
    }
}

// After step k's solve: the rows still active become the work list of step
// k + 1 (two list buffers of n rows used in turn, counts[2]), so the later
// steps' kernels spend no lanes on finished rows.
afsai_status next_active_list(StepArgs& a, int32_t* lists, int32_t* counts, int32_t k, int blocks, cudaStream_t st) {
    int32_t* out = lists + static_cast<size_t>(k & 1) * static_cast<size_t>(a.n);
    int32_t* out_count = counts + (k & 1);
    AFSAI_CUDA_TRY(cudaMemsetAsync(out_count, 0, sizeof(int32_t), st));
    step_compact<<<blocks, 256, 0, st>>>(a.n, a.list, a.count, a.st, out, out_count);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    a.list = out;
    a.count = out_count;
    return AFSAI_OK;
}

// LPR = 0: lane-per-row solve kernel (step_solve); LPR > 0: step_solve_wide
// with LPR lanes per row (FP64 only).  INC: incremental gather.
template <int MC, int HT, bool CHOL32, bool INC = false, int LPR = 0, int GGL = 32>
afsai_status run_stepwise_t(const SetupArgs& o, int32_t kiter, cudaStream_t st) {
    const int32_t n = o.n;
    constexpr int TMC = MC * (MC + 1) / 2;
    DevBuf<int32_t> P, mm, steps, stt;
    DevBuf<double> g, M, psi, psi0;
    AFSAI_TRY(P.alloc(static_cast<size_t>(n) * MC, st));
    AFSAI_TRY(g.alloc(static_cast<size_t>(n) * MC, st));
    AFSAI_TRY(M.alloc(static_cast<size_t>(n) * TMC, st));
    AFSAI_TRY(mm.alloc(n, st));
    AFSAI_TRY(steps.alloc(n, st));
    AFSAI_TRY(stt.alloc(n, st));
    AFSAI_TRY(psi.alloc(n, st));
    AFSAI_TRY(psi0.alloc(n, st));
    StepArgs a{};
    a.n = n;
    a.rowptr = o.rowptr;
    a.col = o.col;
    a.val = o.val;
    a.s = o.s;
    a.exit_mode = o.exit_mode;
    a.eps = o.eps;
    a.mc = MC;
    a.tmc = TMC;
    a.P = P.p;
    a.g = g.p;
    a.M = M.p;
    a.m = mm.p;
    a.steps = steps.p;
    a.st = stt.p;
    a.psi = psi.p;
    a.psi0 = psi0.p;
    a.reach = o.reach;
    a.reach_words = o.reach_words;
    a.stripe_shift = o.stripe_shift;
    a.stripe_magic = o.stripe_magic;
    const int vec_blocks = std::max(1, std::min(ceil_div(n, 256), num_sms() * 8));
    step_init<<<vec_blocks, 256, 0, st>>>(a);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    // gather kernel: 8 warps per block, GGL lanes per row
    auto kg = step_gather<MC, HT, INC, GGL>;
    constexpr int kGroupsBlk = 256 / GGL;
    const size_t smem_g = sizeof(GatherWs<MC, HT>) * kGroupsBlk;
    AFSAI_CUDA_TRY(cudaFuncSetAttribute(kg, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_g)));
    int per_sm_g = 0;
    AFSAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_g, kg, 256, smem_g));
    const int blocks_g = std::max(1, std::min(per_sm_g * num_sms(), ceil_div(n, kGroupsBlk)));
    // solve kernel: lane-interleaved systems, 1 or 2 warps per block (or the
    // several-lanes-per-row kernel)
    static_assert(LPR > 0 || !CHOL32, "the one-lane-per-row solve is FP64 only");
    auto ks = [] {
        if constexpr (LPR > 0 && CHOL32)
            return step_solve_wide32<MC, LPR>;
        else if constexpr (LPR > 0)
            return step_solve_wide<MC, LPR>;
        else
            return step_solve<MC>;
    }();
    constexpr int RPW_S = LPR > 0 ? 32 / (LPR > 0 ? LPR : 1) : 32;
    const size_t per_warp =
        LPR > 0 ? (CHOL32 ? static_cast<size_t>(RPW_S) * (((TMC + MC) | 1) * sizeof(double) +
                                                         (((TMC + MC) | 1) + 1) * sizeof(float))
                          : static_cast<size_t>(RPW_S) * ((TMC + 2 * MC) | 1) * sizeof(double))
                : static_cast<size_t>(TMC + 2 * MC) * 32 * sizeof(double);
    const size_t pair_bytes = LPR > 0 ? (sizeof(uint16_t) * TMC + 15) / 16 * 16 : 0;
    // warps per block (1 to 4) that maximises resident warps per SM
    int wpb = 1, best_w = 0;
    for (int cand = 1; cand <= 4; ++cand) {
        const size_t blk = per_warp * cand + pair_bytes + 1024;
        if (blk > 200u * 1024u) break;
        const int warps = static_cast<int>((227u * 1024u) / blk) * cand;
        if (warps > best_w) {
            best_w = warps;
            wpb = cand;
        }
    }
    const size_t smem_s = per_warp * wpb + pair_bytes;
    AFSAI_CUDA_TRY(cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_s)));
    int per_sm_s = 0;
    AFSAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, ks, 32 * wpb, smem_s));
    if (per_sm_s < 1 || per_sm_g < 1) return fail(AFSAI_ENOTSUP, "stepwise set-up does not fit in shared memory");
    const int rows_per_warp_s = LPR > 0 ? 32 / (LPR > 0 ? LPR : 1) : 32;
    const int blocks_s = std::max(1, std::min(per_sm_s * num_sms(), ceil_div(ceil_div(n, rows_per_warp_s), wpb)));
    DevBuf<int32_t> lists, counts;
    if (kiter > 1) {
        AFSAI_TRY(lists.alloc(2 * static_cast<size_t>(n), st));
        AFSAI_TRY(counts.alloc(2, st));
    }
    for (int32_t k = 1; k <= kiter; ++k) {
        kg<<<blocks_g, 256, smem_g, st>>>(a);
        ks<<<blocks_s, 32 * wpb, smem_s, st>>>(a);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(2);
        if (k < kiter) AFSAI_TRY(next_active_list(a, lists.p, counts.p, k, vec_blocks, st));
    }
    step_finish<<<vec_blocks, 256, 0, st>>>(a, o);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFSAI_OK;
}

// Warps per block (1, 2 or 4) that maximise the resident warps per SM for a
// kernel using per_warp bytes of shared memory per warp plus fixed bytes.
int lane_best_wpb(size_t per_warp, size_t fixed) {
    int wpb = 1, best = 0;
    for (int cand = 1; cand <= 4; cand *= 2) {
        const size_t blk = per_warp * cand + fixed + 1024;
        if (blk > 200u * 1024u) break;
        const int warps = static_cast<int>((227u * 1024u) / blk) * cand;
        if (warps > best) {
            best = warps;
            wpb = cand;
        }
    }
    return wpb;
}

// Launch plan of the small-stencil solve kernel for patterns of at most MCS
// entries (its shared memory grows with MCS, so early steps, whose patterns
// are small, run with a smaller capacity and more resident warps).
template <int MCS, int LPR, bool CHOL32, bool SQRT_INT>
struct LaneSolvePlan {
    void (*k)(StepArgs) = nullptr;
    size_t smem = 0;
    int wpb = 1;
    int blocks = 1;
    afsai_status plan(int32_t n) {
        constexpr int TMC = MCS * (MCS + 1) / 2;
        if constexpr (CHOL32)
            k = step_solve_wide32<MCS, LPR, true>;
        else
            k = step_solve_wide<MCS, LPR, true, SQRT_INT>;
        constexpr int RPW = 32 / LPR;
        const size_t per_row = CHOL32 ? ((TMC + MCS + (MCS + 1) / 2) | 1) * sizeof(double) +
                                            (((TMC + MCS) | 1) + 1) * sizeof(float)
                                      : ((TMC + 2 * MCS + (MCS + 1) / 2) | 1) * sizeof(double);
        const size_t per_warp = per_row * RPW;
        const size_t pair_bytes = (sizeof(uint16_t) * TMC + 15) / 16 * 16;
        wpb = lane_best_wpb(per_warp, pair_bytes);
        smem = per_warp * wpb + pair_bytes;
        AFSAI_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
        int per_sm = 0;
        AFSAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * wpb, smem));
        if (per_sm < 1) return fail(AFSAI_ENOTSUP, "stepwise set-up does not fit in shared memory");
        blocks = std::max(1, std::min(per_sm * num_sms(), ceil_div(ceil_div(n, RPW), wpb)));
        return AFSAI_OK;
    }
    void launch(const StepArgs& a, cudaStream_t st) const { k<<<blocks, 32 * wpb, smem, st>>>(a); }
};

// Launch plan of the lane-per-row gather kernel with HTS table slots.
template <int MC, int HTS>
struct LaneGatherPlan {
    void (*k)(StepArgs) = nullptr;
    size_t smem = 0;
    int wpb = 1;
    int blocks = 1;
    afsai_status plan(int32_t n) {
        k = step_gather_lane<MC, HTS>;
        const size_t per_warp = static_cast<size_t>(HTS * 12 + MC * 4) * 32;
        wpb = lane_best_wpb(per_warp, 0);
        smem = per_warp * wpb;
        AFSAI_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
        int per_sm = 0;
        AFSAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * wpb, smem));
        if (per_sm < 1) return fail(AFSAI_ENOTSUP, "stepwise set-up does not fit in shared memory");
        blocks = std::max(1, std::min(per_sm * num_sms(), ceil_div(ceil_div(n, 32), wpb)));
        return AFSAI_OK;
    }
    void launch(const StepArgs& a, cudaStream_t st) const { k<<<blocks, 32 * wpb, smem, st>>>(a); }
};

// Small stencils (rows of A with at most kLaneRowMax entries, patterns of
// at most MC entries, s <= 4): the lane-per-row gather kernel and the
// LPR-lanes-per-row solve kernel that gathers its system from A.  No
// per-row system slot is allocated.  Steps below the full capacity run
// smaller kernels: the solve kernel compiled for 8 entries when the
// step's patterns hold at most 8 (1 + k s <= 8), then for 10 (of 12) or
// 12 (of 20); the gather kernel with 32-slot tables when the step's
// candidates cannot exceed 28 (|P_{k-1}| kLaneRowMax <= 28), then with
// 48-slot tables up to 42 below 96-slot ones.  Less shared memory per
// row, more resident warps, the same results (a row's arithmetic depends
// neither on its table size nor on the capacity above its pattern).
template <int MC, int LPR, bool CHOL32, int HT = kLaneHT, bool SQRT_INT = false>
afsai_status run_stepwise_lane(const SetupArgs& o, int32_t kiter, cudaStream_t st) {
    const int32_t n = o.n;
    DevBuf<int32_t> P, mm, steps, stt;
    DevBuf<double> g, psi, psi0;
    AFSAI_TRY(P.alloc(static_cast<size_t>(n) * MC, st));
    AFSAI_TRY(g.alloc(static_cast<size_t>(n) * MC, st));
    AFSAI_TRY(mm.alloc(n, st));
    AFSAI_TRY(steps.alloc(n, st));
    AFSAI_TRY(stt.alloc(n, st));
    AFSAI_TRY(psi.alloc(n, st));
    AFSAI_TRY(psi0.alloc(n, st));
    StepArgs a{};
    a.n = n;
    a.rowptr = o.rowptr;
    a.col = o.col;
    a.val = o.val;
    a.s = o.s;
    a.exit_mode = o.exit_mode;
    a.eps = o.eps;
    a.mc = MC;
    a.tmc = MC * (MC + 1) / 2;
    a.P = P.p;
    a.g = g.p;
    a.M = nullptr;
    a.m = mm.p;
    a.steps = steps.p;
    a.st = stt.p;
    a.psi = psi.p;
    a.psi0 = psi0.p;
    a.reach = o.reach;
    a.reach_words = o.reach_words;
    a.stripe_shift = o.stripe_shift;
    a.stripe_magic = o.stripe_magic;
    const int vec_blocks = std::max(1, std::min(ceil_div(n, 256), num_sms() * 8));
    step_init<<<vec_blocks, 256, 0, st>>>(a);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    LaneGatherPlan<MC, HT> gather;
    AFSAI_TRY(gather.plan(n));
    LaneSolvePlan<MC, LPR, CHOL32, SQRT_INT> solve;
    AFSAI_TRY(solve.plan(n));
    // the smaller variants (only when they are smaller): solve capacities 8
    // and 10 (patterns of up to 12) or 8 and 12 (up to 20)
    constexpr int kSmallMC = MC > 8 ? 8 : MC;
    constexpr int kMidMC = MC > 12 ? 12 : (MC > 10 ? 10 : MC);
    constexpr int kSmallHT = HT > 32 ? 32 : HT;
    constexpr int kMidHT = HT > 48 ? 48 : HT;
    LaneGatherPlan<MC, kSmallHT> gather_small;
    LaneGatherPlan<MC, kMidHT> gather_mid;
    LaneSolvePlan<kSmallMC, LPR, CHOL32, SQRT_INT> solve_small;
    LaneSolvePlan<kMidMC, LPR, CHOL32, SQRT_INT> solve_mid;
    if (kSmallHT < HT) AFSAI_TRY(gather_small.plan(n));
    if (kMidHT < HT && kMidHT > kSmallHT) AFSAI_TRY(gather_mid.plan(n));
    if (kSmallMC < MC) AFSAI_TRY(solve_small.plan(n));
    if (kMidMC < MC && kMidMC > kSmallMC) AFSAI_TRY(solve_mid.plan(n));
    DevBuf<int32_t> lists, counts;
    if (kiter > 1) {
        AFSAI_TRY(lists.alloc(2 * static_cast<size_t>(n), st));
        AFSAI_TRY(counts.alloc(2, st));
    }
    // AFSAI_LANE_SMALL: bit 0 the smaller gather tables, bit 1 the smaller
    // solve capacities.  Default (measured on the 256^3 diffusion set-up):
    // both for the FP64 Cholesky (107.9 -> 97.9 ms); the tables only for the
    // FP32 Cholesky of patterns up to 12 entries (93.9 -> 93.0 ms; with the
    // capacity of 8 too, 95.6 ms); both for patterns up to 20 (the uneven
    // batch: 495 -> 468 ms)
    static const int small_env = [] {
        const char* e = std::getenv("AFSAI_LANE_SMALL");
        return e ? std::atoi(e) : -1;
    }();
    const int small_mask = small_env >= 0 ? small_env : ((CHOL32 && MC <= 12) ? 1 : 3);
    for (int32_t k = 1; k <= kiter; ++k) {
        const int64_t prev = 1 + static_cast<int64_t>(k - 1) * o.s;  // |P_{k-1}| at most
        const int64_t next = prev + o.s;                              // |P_k| at most
        if ((small_mask & 1) && kSmallHT < HT && prev * kLaneRowMax <= kSmallHT - (kSmallHT >> 3))
            gather_small.launch(a, st);
        else if ((small_mask & 1) && kMidHT < HT && kMidHT > kSmallHT && prev * kLaneRowMax <= kMidHT - (kMidHT >> 3))
            gather_mid.launch(a, st);
        else
            gather.launch(a, st);
        if ((small_mask & 2) && kSmallMC < MC && next <= kSmallMC)
            solve_small.launch(a, st);
        else if ((small_mask & 2) && kMidMC < MC && kMidMC > kSmallMC && next <= kMidMC)
            solve_mid.launch(a, st);
        else
            solve.launch(a, st);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(2);
        if (k < kiter) AFSAI_TRY(next_active_list(a, lists.p, counts.p, k, vec_blocks, st));
    }
    step_finish<<<vec_blocks, 256, 0, st>>>(a, o);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFSAI_OK;
}

// Pattern capacities served by the small-pattern stepwise path (21 to 32
// entries: run_stepwise_wide).
bool stepwise_supported(int64_t mcap) { return mcap <= 20; }

// FP64 systems of 21 to 32 entries: incremental gather, LPR lanes per row
// in the solve.
afsai_status run_stepwise_wide(const SetupArgs& o, int ht, int lpr, int32_t kiter, bool chol32, cudaStream_t st) {
    if (chol32)
        return ht == 256 ? run_stepwise_t<32, 256, true, true, 8>(o, kiter, st)
                         : run_stepwise_t<32, 512, true, true, 8>(o, kiter, st);
    if (lpr == 8)
        return ht == 256 ? run_stepwise_t<32, 256, false, true, 8>(o, kiter, st)
                         : run_stepwise_t<32, 512, false, true, 8>(o, kiter, st);
    return ht == 256 ? run_stepwise_t<32, 256, false, true, 4>(o, kiter, st)
                     : run_stepwise_t<32, 512, false, true, 4>(o, kiter, st);
}

// Patterns of up to 12 entries whose candidates fit a 128-slot table
// (at most 112 keys): the gather kernel packs rows, GGL lanes per row.
template <int LPR>
afsai_status run_stepwise_packed(const SetupArgs& o, int ggl, int32_t kiter, cudaStream_t st) {
    switch (ggl) {
        case 4: return run_stepwise_t<12, 128, false, true, LPR, 4>(o, kiter, st);
        case 8: return run_stepwise_t<12, 128, false, true, LPR, 8>(o, kiter, st);
        case 16: return run_stepwise_t<12, 128, false, true, LPR, 16>(o, kiter, st);
        default: return run_stepwise_t<12, 128, false, true, LPR, 32>(o, kiter, st);
    }
}

// Whether the lane-per-row gather serves this set-up (AFSAI_GATHER_LANE=0
// turns it off).
bool lane_gather_applies(int64_t mcap, int32_t s, int32_t max_row_nnz) {
    static const bool on = [] {
        const char* e = std::getenv("AFSAI_GATHER_LANE");
        return !e || std::atoi(e) != 0;
    }();
    return on && mcap <= 20 && s <= 4 && max_row_nnz <= kLaneRowMax;
}

afsai_status run_stepwise(const SetupArgs& o, int64_t mcap, int ht, int32_t kiter, bool chol32, cudaStream_t st,
                          int64_t cand_bound) {
    // FP64: several lanes per row in the solve (measured best: 2 lanes for
    // patterns of up to 12 entries, 4 up to 20); AFSAI_STEPWISE_SMALL_LPR =
    // 1 selects the one-lane-per-row solve kernel, 2 or 4 force a width
    static const int small_lpr = [] {
        const char* e = std::getenv("AFSAI_STEPWISE_SMALL_LPR");
        return e ? std::atoi(e) : 0;
    }();
    // lanes per row of the gather kernel for small candidate sets
    // (AFSAI_GATHER_GL = 4, 8, 16 or 32)
    static const int gather_gl = [] {
        const char* e = std::getenv("AFSAI_GATHER_GL");
        return e ? std::atoi(e) : 32;
    }();
    const int lpr = small_lpr != 0 ? small_lpr : (mcap <= 12 ? 2 : 4);
    if (!chol32 && mcap <= 12 && cand_bound * 8 <= 128 * 7 && gather_gl != 32 && (lpr == 2 || lpr == 4))
        return lpr == 4 ? run_stepwise_packed<4>(o, gather_gl, kiter, st) : run_stepwise_packed<2>(o, gather_gl, kiter, st);
    if (!chol32 && mcap <= 20 && (lpr == 2 || lpr == 4)) {
        if (mcap <= 12)
            return lpr == 4 ? (ht == 256 ? run_stepwise_t<12, 256, false, true, 4>(o, kiter, st)
                                         : run_stepwise_t<12, 512, false, true, 4>(o, kiter, st))
                            : (ht == 256 ? run_stepwise_t<12, 256, false, true, 2>(o, kiter, st)
                                         : run_stepwise_t<12, 512, false, true, 2>(o, kiter, st));
        return lpr == 4 ? (ht == 256 ? run_stepwise_t<20, 256, false, true, 4>(o, kiter, st)
                                     : run_stepwise_t<20, 512, false, true, 4>(o, kiter, st))
                        : (ht == 256 ? run_stepwise_t<20, 256, false, true, 2>(o, kiter, st)
                                     : run_stepwise_t<20, 512, false, true, 2>(o, kiter, st));
    }
    // FP32 Cholesky + FP64 refinement (the mixed form): 4 lanes per row
    if (chol32 && mcap <= 20)
        return ht == 256 ? run_stepwise_t<20, 256, true, true, 4>(o, kiter, st)
                         : run_stepwise_t<20, 512, true, true, 4>(o, kiter, st);
    if (chol32) return fail(AFSAI_ENOTSUP, "small-pattern stepwise path: up to 20 entries");
    if (mcap <= 12)
        return ht == 256 ? run_stepwise_t<12, 256, false>(o, kiter, st) : run_stepwise_t<12, 512, false>(o, kiter, st);
    if (mcap <= 20)
        return ht == 256 ? run_stepwise_t<20, 256, false>(o, kiter, st) : run_stepwise_t<20, 512, false>(o, kiter, st);
    return fail(AFSAI_ENOTSUP, "small-pattern stepwise path: up to 20 entries");
}

// ---------------------------------------------------------------------------
// Locality bound (Section 4): stripe adjacency Ahat of A and its boolean
// powers, as bit rows of `words` 32-bit words per stripe.
// ---------------------------------------------------------------------------
constexpr int64_t kMaxStripes = 8192;

__device__ __forceinline__ uint32_t stripe_of(int32_t j, uint64_t magic, int shift) {
    return static_cast<uint32_t>((static_cast<uint64_t>(j) * magic) >> shift);
}

// bit (I, J) of ahat set iff block (I, J) of A holds a nonzero; one thread
// per row, a word is or-ed only when the stripe of the (sorted) columns
// changes
__global__ void k_stripe_adjacency(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   uint64_t magic, int shift, int32_t words, uint32_t* __restrict__ ahat) {
    for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
         r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint32_t* row = ahat + static_cast<size_t>(stripe_of(static_cast<int32_t>(r), magic, shift)) * words;
        uint32_t last = 0xffffffffu;
        for (int32_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            const uint32_t J = stripe_of(col[e], magic, shift);
            if (J != last) {
                atomicOr(&row[J >> 5], 1u << (J & 31u));
                last = J;
            }
        }
    }
}

__global__ void k_stripe_identity(int32_t nb, int32_t words, uint32_t* __restrict__ r) {
    for (int64_t I = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; I < nb;
         I += static_cast<int64_t>(gridDim.x) * blockDim.x)
        r[static_cast<size_t>(I) * words + (I >> 5)] = 1u << (I & 31);
}

// next[I] = OR over the stripes K set in cur[I] of ahat[K] (one boolean
// product); one block per stripe I, threads over the output words
__global__ void k_stripe_power(int32_t nb, int32_t words, const uint32_t* __restrict__ cur,
                               const uint32_t* __restrict__ ahat, uint32_t* __restrict__ next) {
    for (int32_t I = blockIdx.x; I < nb; I += gridDim.x) {
        const uint32_t* cr = cur + static_cast<size_t>(I) * words;
        for (int32_t w = threadIdx.x; w < words; w += blockDim.x) {
            uint32_t acc = 0u;
            for (int32_t wk = 0; wk < words; ++wk) {
                uint32_t bits = cr[wk];
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    acc |= ahat[static_cast<size_t>(wk * 32 + b) * words + w];
                }
            }
            next[static_cast<size_t>(I) * words + w] = acc;
        }
    }
}

// Fills the bound fields of `a`; `buf` holds the reach rows until the
// set-up ends.  No bound for block_rows = 0 or a single stripe.
afsai_status build_stripe_reach(const afsai_csr* A, const afsai_params* p, cudaStream_t st, SetupArgs* a,
                                DevBuf<uint32_t>* buf) {
    a->reach = nullptr;
    a->reach_words = 0;
    a->stripe_magic = 0;
    a->stripe_shift = 0;
    if (p->block_rows <= 0) return AFSAI_OK;
    const int64_t nb = (static_cast<int64_t>(A->n) + p->block_rows - 1) / p->block_rows;
    if (nb <= 1) return AFSAI_OK;
    if (nb > kMaxStripes) return fail(AFSAI_ENOTSUP, "more than 8192 stripes in the locality bound");
    const int32_t words = static_cast<int32_t>((nb + 31) / 32);
    // multiply-shift division by block_rows, exact for 0 <= j < 2^31
    int l = 0;
    while ((int64_t(1) << l) < p->block_rows) ++l;
    const uint64_t magic = ((uint64_t(1) << (31 + l)) / static_cast<uint64_t>(p->block_rows)) + 1u;
    const int shift = 31 + l;
    const size_t cells = static_cast<size_t>(nb) * words;
    DevBuf<uint32_t> ahat, tmp;
    AFSAI_TRY(ahat.alloc(cells, st));
    AFSAI_TRY(tmp.alloc(cells, st));
    AFSAI_TRY(buf->alloc(cells, st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(ahat.p, 0, cells * sizeof(uint32_t), st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(buf->p, 0, cells * sizeof(uint32_t), st));
    const int rb = std::max(1, std::min(ceil_div(A->n, 256), num_sms() * 8));
    k_stripe_adjacency<<<rb, 256, 0, st>>>(A->n, A->rowptr, A->col, magic, shift, words, ahat.p);
    const int ib = std::max(1, std::min(ceil_div(nb, 256), num_sms() * 8));
    k_stripe_identity<<<ib, 256, 0, st>>>(static_cast<int32_t>(nb), words, buf->p);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    uint32_t* cur = buf->p;
    uint32_t* nxt = tmp.p;
    for (int32_t t = 0; t < p->block_power; ++t) {
        const int pb = static_cast<int>(std::min<int64_t>(nb, static_cast<int64_t>(num_sms()) * 16));
        k_stripe_power<<<pb, 128, 0, st>>>(static_cast<int32_t>(nb), words, cur, ahat.p, nxt);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        std::swap(cur, nxt);
    }
    if (cur != buf->p)
        AFSAI_CUDA_TRY(cudaMemcpyAsync(buf->p, cur, cells * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    a->reach = buf->p;
    a->reach_words = words;
    a->stripe_magic = magic;
    a->stripe_shift = shift;
    // ahat and tmp are freed in stream order after the kernels that read them
    return AFSAI_OK;
}

int lanes_per_row(int mcap_t, bool chol32) {
    (void)mcap_t;
    (void)chol32;
    return 32;
}

}  // namespace

afsai_status setup_impl(const afsai_csr* A, const afsai_params* p, int32_t max_row_nnz, cudaStream_t st,
                        afsai_precond* M, bool sliced, const SetupTuning* tune) {
    const int32_t n = A->n;
    const int64_t mcap = 1 + static_cast<int64_t>(p->kiter) * p->s;
    if (mcap > 128) return fail(AFSAI_ENOTSUP, "1 + kiter*s must be <= 128");
    const int mcap_t = mcap <= 16 ? 16 : (mcap <= 20 ? 20 : (mcap <= 32 ? 32 : (mcap <= 64 ? 64 : 128)));
    // Shared table size: candidates are bounded by |P| * (longest row); the
    // table keeps a load factor <= 7/8 up to that bound, else it relies on
    // the overflow retry.  Only columns below the diagonal are candidates,
    // so with a symmetric pattern the rows of P offer about half their
    // entries: 256 slots serve while |P| times that half fits (27-point
    // rows, 17-entry patterns: at most 119 distinct candidates in the
    // oracle's patterns, no retry; set-up 5.39 -> 4.70 ms at 48^3 against
    // 512 slots, whose clearing and lower occupancy cost the difference).
    const int64_t cand_bound = mcap * static_cast<int64_t>(max_row_nnz);
    int ht = 512;
    if (mcap_t <= 32 && (cand_bound * 8 <= 256 * 7 || mcap * ((static_cast<int64_t>(max_row_nnz) + 1) / 2) <= 256))
        ht = 256;
    // (20-entry patterns use the 20-entry workspace template)
    const bool chol32 = p->chol_prec == 1;
    const int gl = lanes_per_row(mcap_t, chol32);

    cudaEvent_t ev0, ev1;
    AFSAI_CUDA_TRY(cudaEventCreate(&ev0));
    AFSAI_CUDA_TRY(cudaEventCreate(&ev1));
    AFSAI_CUDA_TRY(cudaEventRecord(ev0, st));

    DevBuf<int32_t> len, ocol, status, retry, counters;
    DevBuf<double> oval;
    AFSAI_TRY(len.alloc(n, st));
    AFSAI_TRY(ocol.alloc(static_cast<size_t>(n) * mcap, st));
    AFSAI_TRY(oval.alloc(static_cast<size_t>(n) * mcap, st));
    AFSAI_TRY(status.alloc(n, st));
    AFSAI_TRY(retry.alloc(n, st));
    AFSAI_TRY(counters.alloc(4, st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(counters.p, 0, 4 * sizeof(int32_t), st));
    AFSAI_CUDA_TRY(lib_malloc_async(reinterpret_cast<void**>(&M->psi), sizeof(double) * n, st));
    AFSAI_CUDA_TRY(lib_malloc_async(reinterpret_cast<void**>(&M->steps), sizeof(int32_t) * n, st));

    SetupArgs a{};
    a.n = n;
    a.rowptr = A->rowptr;
    a.col = A->col;
    a.val = A->val;
    a.kiter = p->kiter;
    a.s = p->s;
    a.exit_mode = p->exit_mode;
    a.eps = p->eps;
    a.mcap = mcap;
    a.out_len = len.p;
    a.out_col = ocol.p;
    a.out_val = oval.p;
    a.psi = M->psi;
    a.steps = M->steps;
    a.status = status.p;
    a.rows = nullptr;
    a.nrows = n;
    a.retry_rows = retry.p;
    a.counters = counters.p;
    DevBuf<uint32_t> reach;
    AFSAI_TRY(build_stripe_reach(A, p, st, &a, &reach));
    cudaEvent_t evk0, evk1;
    AFSAI_CUDA_TRY(cudaEventCreate(&evk0));
    AFSAI_CUDA_TRY(cudaEventCreate(&evk1));
    AFSAI_CUDA_TRY(cudaEventRecord(evk0, st));
    static const bool fused_only = [] {
        const char* e = std::getenv("AFSAI_SETUP_FUSED_ONLY");
        return e && std::atoi(e) != 0;
    }();
    // the stepwise path pays off where FP64 square roots and divisions
    // dominate: FP64 factorisation of small patterns
    // FP64 systems of 21 to 32 entries: incremental stepwise gather and the
    // several-lanes-per-row solve (8 lanes per row, 4 rows per warp);
    // AFSAI_STEPWISE_WIDE = 4 or 8 sets the lanes per row, 0 keeps the fused
    // kernel
    static const int wide_lpr = [] {
        const char* e = std::getenv("AFSAI_STEPWISE_WIDE");
        return e ? std::atoi(e) : 8;
    }();
    // the mixed form takes the same path (FP32 solve + FP64 refinement in
    // step_solve_wide32) unless AFSAI_STEPWISE_WIDE_MIXED = 0
    static const bool wide_mixed = [] {
        const char* e = std::getenv("AFSAI_STEPWISE_WIDE_MIXED");
        return !e || std::atoi(e) != 0;
    }();
    if (p->kiter == 0) {
        const int blocks = std::max(1, std::min(ceil_div(n, 256), num_sms() * 8));
        k_setup_diagonal<<<blocks, 256, 0, st>>>(a);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
    } else if (!fused_only && lane_gather_applies(mcap, p->s, max_row_nnz)) {
        // small stencils: lane-per-row gather, 2 lanes per row in the solve
        // (AFSAI_LANE_HT = 48 (default) or 64 table slots per row;
        // AFSAI_SOLVE_SQRT = 0 IEEE FP64 or 1 integer-pipe square roots)
        static const int lane_ht = [] {
            const char* e = std::getenv("AFSAI_LANE_HT");
            return e && std::atoi(e) == 64 ? 64 : kLaneHT;
        }();
        static const bool sqrt_int = [] {
            const char* e = std::getenv("AFSAI_SOLVE_SQRT");
            return e && std::atoi(e) == 1;
        }();
        // patterns of 13 to 20 entries (kiter 8, s 2 in the uneven batch):
        // up to ~60 distinct candidates (63 for an anisotropic 7-point
        // stencil), 96-slot tables (5 warps per SM; 128 slots: 4), 4 or 8
        // lanes per row
        // (no tuning given: 2 lanes per row for the FP64 Cholesky, 4 for the
        // FP32 one; 256^3 diffusion: FP64 103.8 ms with 2, 122.9 with 4;
        // FP32 Cholesky 94.6 ms with 2, 88.2 with 4)
        const int lpr = tune ? tune->lane_lpr : (chol32 ? 4 : 0);
        if (mcap > 12) {
            if (lpr == 8)
                AFSAI_TRY(chol32 ? (run_stepwise_lane<20, 8, true, 96>(a, p->kiter, st))
                                 : (run_stepwise_lane<20, 8, false, 96>(a, p->kiter, st)));
            else
                AFSAI_TRY(chol32 ? (run_stepwise_lane<20, 4, true, 96>(a, p->kiter, st))
                                 : (run_stepwise_lane<20, 4, false, 96>(a, p->kiter, st)));
        } else if (lpr == 4) {
            AFSAI_TRY(chol32 ? (run_stepwise_lane<12, 4, true>(a, p->kiter, st))
                             : (run_stepwise_lane<12, 4, false>(a, p->kiter, st)));
        } else if (chol32)
            AFSAI_TRY(lane_ht == 64 ? (run_stepwise_lane<12, 2, true, 64>(a, p->kiter, st))
                                    : (run_stepwise_lane<12, 2, true>(a, p->kiter, st)));
        else if (sqrt_int)
            AFSAI_TRY(lane_ht == 64 ? (run_stepwise_lane<12, 2, false, 64, true>(a, p->kiter, st))
                                    : (run_stepwise_lane<12, 2, false, kLaneHT, true>(a, p->kiter, st)));
        else
            AFSAI_TRY(lane_ht == 64 ? (run_stepwise_lane<12, 2, false, 64>(a, p->kiter, st))
                                    : (run_stepwise_lane<12, 2, false>(a, p->kiter, st)));
    } else if (!fused_only && stepwise_supported(mcap))
        AFSAI_TRY(run_stepwise(a, mcap, ht, p->kiter, chol32, st, cand_bound));
    else if (!fused_only && (wide_lpr == 4 || wide_lpr == 8) && mcap > 20 && mcap <= 32 && (!chol32 || wide_mixed))
        AFSAI_TRY(run_stepwise_wide(a, ht, wide_lpr, p->kiter, chol32, st));
    else
        AFSAI_TRY(dispatch(mcap_t, ht, gl, a, n, INT64_MAX, false, chol32, st));
    AFSAI_CUDA_TRY(cudaEventRecord(evk1, st));

    int32_t hc[4];
    AFSAI_CUDA_TRY(cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    float kms = 0.f;
    cudaEventElapsedTime(&kms, evk0, evk1);
    cudaEventDestroy(evk0);
    cudaEventDestroy(evk1);
    const int32_t nretry = hc[0];
    if (nretry > 0) {
        // redo the overflowed rows with a global-memory table per warp
        int log2 = 6;
        while ((int64_t(1) << log2) < 2 * cand_bound) ++log2;
        int64_t warps = std::min<int64_t>(nretry, static_cast<int64_t>(num_sms()) * 64);
        warps = (warps + 7) / 8 * 8;  // whole blocks of up to 8 warps
        const int64_t slots = warps << log2;
        DevBuf<int32_t> gkey, glist, rows2, counters2;
        DevBuf<double> gval;
        AFSAI_TRY(gkey.alloc(slots, st));
        AFSAI_TRY(glist.alloc(slots, st));
        AFSAI_TRY(gval.alloc(slots, st));
        AFSAI_TRY(rows2.alloc(nretry, st));
        AFSAI_TRY(counters2.alloc(4, st));
        AFSAI_CUDA_TRY(cudaMemcpyAsync(rows2.p, retry.p, sizeof(int32_t) * nretry, cudaMemcpyDeviceToDevice, st));
        AFSAI_CUDA_TRY(cudaMemsetAsync(counters2.p, 0, 4 * sizeof(int32_t), st));
        SetupArgs b = a;
        b.rows = rows2.p;
        b.nrows = nretry;
        b.counters = counters2.p;
        b.gkey = gkey.p;
        b.gval = gval.p;
        b.glist = glist.p;
        b.ght_log2 = log2;
        AFSAI_TRY(dispatch(mcap_t, ht, gl, b, nretry, warps, true, chol32, st));
        int32_t hc2[4];
        AFSAI_CUDA_TRY(cudaMemcpyAsync(hc2, counters2.p, sizeof(hc2), cudaMemcpyDeviceToHost, st));
        AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
        if (hc2[0] != 0) return fail(AFSAI_ENOTSUP, "candidate table overflow in the retry pass");
        hc[1] += hc2[1];
    }
    if (hc[1] > 0) {
        return fail(AFSAI_ENOTSPD, "non-positive pivot in " + std::to_string(hc[1]) + " row system(s)");
    }

    // CSR of G
    CsrDev& G = M->G;
    G.n = n;
    G.vtype = p->g_prec;
    AFSAI_CUDA_TRY(lib_malloc_async(reinterpret_cast<void**>(&G.rowptr), sizeof(int32_t) * (n + 1), st));
    int64_t nnz = 0;
    AFSAI_TRY(exclusive_scan_i32(len.p, G.rowptr, n, st, &nnz));
    G.nnz = nnz;
    AFSAI_CUDA_TRY(lib_malloc_async(reinterpret_cast<void**>(&G.col), sizeof(int32_t) * std::max<int64_t>(nnz, 1), st));
    AFSAI_CUDA_TRY(lib_malloc_async(&G.val, val_bytes(G.vtype) * std::max<int64_t>(nnz, 1), st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(counters.p, 0, sizeof(int32_t), st));
    {
        const int threads = 256;  // compact_rows_kernel's shared row starts assume 8 warps
        const int blocks = std::max(1, std::min(ceil_div(static_cast<int64_t>(n), threads), num_sms() * 16));
        if (G.vtype == VAL_F64)
            compact_rows_kernel<double><<<blocks, threads, 0, st>>>(n, mcap, len.p, ocol.p, oval.p, G.rowptr, G.col,
                                                                   static_cast<double*>(G.val), counters.p);
        else if (G.vtype == VAL_F32)
            compact_rows_kernel<float><<<blocks, threads, 0, st>>>(n, mcap, len.p, ocol.p, oval.p, G.rowptr, G.col,
                                                                  static_cast<float*>(G.val), counters.p);
        else
            compact_rows_kernel<__nv_bfloat16><<<blocks, threads, 0, st>>>(
                n, mcap, len.p, ocol.p, oval.p, G.rowptr, G.col, static_cast<__nv_bfloat16*>(G.val), counters.p);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
    }
    AFSAI_CUDA_TRY(cudaMemcpyAsync(&G.max_row, counters.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    AFSAI_TRY(build_transpose(G, &M->Gt, st));
    if (sliced) {
        // the sliced copies only serve the sliced SpMV engines: they are
        // built for a role whose engine is sliced or not chosen yet for this
        // shape; without room for them the CSR engines serve and the set-up
        // succeeds
        const std::string keep = afsai_last_error();
        const bool want_g = spmv_wants_sliced(ROLE_G, G), want_gt = spmv_wants_sliced(ROLE_GT, M->Gt);
        if ((want_g && build_sell(G, &G.sell, st, spmv_wants_order(ROLE_G, G)) != AFSAI_OK) ||
            (want_gt && build_sell(M->Gt, &M->Gt.sell, st, spmv_wants_order(ROLE_GT, M->Gt)) != AFSAI_OK)) {
            free_sell(&G.sell, st);
            free_sell(&M->Gt.sell, st);
            cudaGetLastError();
            set_error(keep);
        }
    }
    AFSAI_CUDA_TRY(cudaEventRecord(ev1, st));
    AFSAI_CUDA_TRY(cudaEventSynchronize(ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    M->info.n = n;
    M->info.nnz_G = nnz;
    M->info.max_row = G.max_row;
    M->info.g_prec = G.vtype;
    M->info.n_retry = nretry;
    M->info.setup_ms = ms;
    M->info.kernel_ms = kms;
    return AFSAI_OK;
}

}  // namespace afsai
