// TMA-staged CSR SpMV for sm_103a.
//
// A block owns tiles of ROWS = blockDim.x / TPR consecutive rows.  For each
// tile one thread issues bulk asynchronous copies (cp.async.bulk, completion
// counted on an mbarrier) of the tile's contiguous column and value spans
// into shared memory; the copies stream whole 16-byte-aligned windows of
// HBM.  Then TPR threads per row accumulate the row from shared memory, each
// over a contiguous part of the row in CSR order (TPR = 1: the plain
// sequential sum).  With one FP64 fma per entry and no cross-lane
// reductions for TPR = 1, the FP64 issue slots - the binding resource of
// GB300 FP64 SpMV - are all full.
//
// Alignment: a bulk copy needs 16-byte aligned source, destination and size.
// The copied window is the span rounded outwards to 16 bytes (never past
// the last whole 16-byte group of the array); the few trailing entries of
// the array beyond it are loaded with plain loads.  A tile whose span does
// not fit the stage buffer is computed straight from global memory with
// the same arithmetic.
//
// Every wait on the mbarrier is bounded (clock64 deadline); on expiry the
// block sets the error flag, waits once more (bounded) for its copies and
// returns without contributing to the grid reduction.
#pragma once

#include <functional>

#include "afsai_internal.cuh"

namespace afsai {
namespace tiled {

constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait for the given phase parity; false if `limit` cycles passed.
// The waits for a tile's copies take the caller's limit (the PCG passes a
// shorter one when asked to, so that the expiry path can be exercised);
// the second wait after an expiry, which lets the block's copies in flight
// land before it returns, always takes the full bound.  limit = 0 checks
// the phase once without waiting (mbarrier.try_wait may itself suspend the
// warp until the phase completes, so even a one-cycle limit need not run
// out).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, long long limit = kWaitCycles) {
    if (limit <= 0) return mbar_test_wait(bar, phase);
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

template <typename T>
struct Conv;
template <>
struct Conv<double> {
    __device__ static double f64(double v) { return v; }
    __device__ static float f32(double v) { return static_cast<float>(v); }
};
template <>
struct Conv<float> {
    __device__ static double f64(float v) { return static_cast<double>(v); }
    __device__ static float f32(float v) { return v; }
};
template <>
struct Conv<__nv_bfloat16> {
    __device__ static double f64(__nv_bfloat16 v) { return static_cast<double>(__bfloat162float(v)); }
    __device__ static float f32(__nv_bfloat16 v) { return __bfloat162float(v); }
};

template <typename ACC>
struct Mul;
template <>
struct Mul<double> {
    template <typename VT, typename XT>
    __device__ static double fma_(VT a, XT x, double acc) {
        return fma(Conv<VT>::f64(a), static_cast<double>(x), acc);
    }
};
template <>
struct Mul<float> {
    template <typename VT, typename XT>
    __device__ static float fma_(VT a, XT x, float acc) {
        return fmaf(Conv<VT>::f32(a), static_cast<float>(x), acc);
    }
};

// Shared-memory layout of a stage: [mbarrier (128 B)] [cols] [vals].
template <typename VT>
__host__ __device__ inline size_t stage_col_bytes(int cap) {
    return (static_cast<size_t>(cap) * 4 + 127) / 128 * 128;
}
template <typename VT>
__host__ __device__ inline size_t stage_bytes(int cap) {
    return 128 + stage_col_bytes<VT>(cap) + (static_cast<size_t>(cap) * sizeof(VT) + 127) / 128 * 128;
}

// Row loop of one tile.  Epi::row(i, acc) consumes the result of row i
// (called by the first thread of the row's group).  order (TPR = 1): the
// tile's rows by length, so that each warp takes rows of similar length.
template <int TPR, typename VT, typename XT, typename ACC, class Epi>
__device__ __forceinline__ void tile_rows(int64_t r0, int64_t r1, const int32_t* __restrict__ rowptr,
                                          const int32_t* __restrict__ col, const VT* __restrict__ val,
                                          const XT* __restrict__ x, const int32_t* scol, const VT* sval,
                                          int64_t c_lo, int64_t v_lo, bool staged, Epi& epi,
                                          const uint8_t* __restrict__ order = nullptr) {
    const int t = threadIdx.x;
    int64_t i = r0 + t / TPR;
    if (TPR == 1 && order != nullptr && i < r1) i = r0 + order[i];
    const int part = t % TPR;
    ACC acc = ACC(0);
    if (i < r1) {
        const int32_t b = rowptr[i], e = rowptr[i + 1];
        int32_t kb = b, ke = e;
        if (TPR > 1) {
            const int32_t len = e - b;
            kb = b + (len * part) / TPR;
            ke = b + (len * (part + 1)) / TPR;
        }
        if (staged) {
            const int32_t* sc = scol - c_lo;
            const VT* sv = sval - v_lo;
#pragma unroll 4
            for (int32_t k = kb; k < ke; ++k) acc = Mul<ACC>::fma_(sv[k], __ldg(&x[sc[k]]), acc);
        } else {
#pragma unroll 4
            for (int32_t k = kb; k < ke; ++k) acc = Mul<ACC>::fma_(__ldg(&val[k]), __ldg(&x[__ldg(&col[k])]), acc);
        }
    }
    if (TPR > 1) {
        // combine the parts in a fixed order (part 0 + part 1 (+ ...))
#pragma unroll
        for (int o = 1; o < TPR; o <<= 1) {
            const ACC other = __shfl_down_sync(0xffffffffu, acc, o, TPR);
            if ((part & ((o << 1) - 1)) == 0) acc += other;
        }
    }
    if (part == 0 && i < r1) epi.row(i, acc);
}

// Balanced variant of the tile's row loop (engine 103): the tile's entries
// are split evenly over the block's threads (each a contiguous run of
// C = ceil(T / threads) entries, T the tile's entry count), so every FP64
// fma instruction of the products is full whatever the row lengths (G^T
// rows: 1 to ~40 entries; one thread per row leaves about half of each
// warp idle in the FP64 pipe, the binding unit).  A run's thread only
// records sums in shared memory (no FP64 work in its divergent row-end
// branches): res[j] for a row j that lies inside its run, head[t] for the
// piece of a row begun in an earlier run, part[t] for the piece of a row
// that continues past the run.  Then thread j finishes row j with every
// lane active: res[j], or part over the runs the row starts in and
// crosses, then head of the run it ends in; the epilogue (store, fused
// dot product) runs once per row in row order.  Work area in shared
// memory after the stage: kBalancedTileBytes.
template <typename ACC>
struct BalancedTile {
    int32_t rp[257];  // row pointers of the tile's rows (blockDim.x <= 256)
    ACC res[256];     // sums of rows inside one run
    ACC part[256];    // each run's piece of the row continuing past its end
    ACC head[256];    // each run's piece of a row begun in an earlier run
};
constexpr size_t kBalancedTileBytes = sizeof(BalancedTile<double>);

template <typename VT, typename XT, typename ACC, class Epi>
__device__ __forceinline__ void tile_rows_balanced(int64_t r0, int64_t r1, const int32_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                   const XT* __restrict__ x, const int32_t* scol, const VT* sval,
                                                   int64_t c_lo, int64_t v_lo, bool staged, BalancedTile<ACC>& B,
                                                   Epi& epi) {
    const int t = threadIdx.x, nt = blockDim.x;
    const int nr = static_cast<int>(r1 - r0);
    for (int k = t; k <= nr; k += nt) B.rp[k] = rowptr[r0 + k];
    __syncthreads();
    const int32_t e0 = B.rp[0], e1 = B.rp[nr];
    const int32_t T = e1 - e0;
    const int32_t* __restrict__ cs = staged ? scol - c_lo : col;
    const VT* __restrict__ vs = staged ? sval - v_lo : val;
    const int32_t C = T > 0 ? (T + nt - 1) / nt : 1;
    const int32_t s = e0 + t * C;
    const int32_t e_end = s + C < e1 ? s + C : e1;
    if (s < e_end) {
        // the row holding entry s: the last row starting at or before s
        int k = 0, hi = nr - 1;
        while (k < hi) {
            const int mid = (k + hi + 1) >> 1;
            if (B.rp[mid] <= s)
                k = mid;
            else
                hi = mid - 1;
        }
        ACC acc = ACC(0);
        auto close_row = [&]() {
            if (B.rp[k] >= s)
                B.res[k] = acc;  // the whole row lies in this run
            else
                B.head[t] = acc;  // the row began in an earlier run
            ++k;
            acc = ACC(0);
        };
        int32_t e = s;
        for (; e + 4 <= e_end; e += 4) {
            int32_t c4[4];
            VT v4[4];
            XT x4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                c4[u] = cs[e + u];
                v4[u] = vs[e + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) x4[u] = __ldg(&x[c4[u]]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                while (B.rp[k + 1] <= e + u) close_row();
                acc = Mul<ACC>::fma_(v4[u], x4[u], acc);
            }
        }
        for (; e < e_end; ++e) {
            while (B.rp[k + 1] <= e) close_row();
            acc = Mul<ACC>::fma_(vs[e], __ldg(&x[cs[e]]), acc);
        }
        // the row of the last entry: it ends with the run or continues
        if (B.rp[k + 1] <= e_end)
            close_row();
        else
            B.part[t] = acc;
    }
    __syncthreads();
    if (t < nr) {
        const int32_t b = B.rp[t] - e0, e = B.rp[t + 1] - e0;
        ACC sum = ACC(0);
        if (e > b) {
            const int L0 = b / C, L1 = (e - 1) / C;
            if (L0 == L1) {
                sum = B.res[t];
            } else {
                sum = B.part[L0];
                for (int L = L0 + 1; L < L1; ++L) sum += B.part[L];
                sum += B.head[L1];
            }
        }
        epi.row(r0 + t, sum);
    }
}

// The tile loop.  Returns false if a bounded wait expired (error flag set).
// BAL: the balanced row loop (tile_rows_balanced; TPR must be 1).
template <int TPR, typename VT, typename XT, typename ACC, class Epi, bool BAL = false>
__device__ bool spmv_tiles(int32_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                           const int32_t* __restrict__ col, const VT* __restrict__ val, const XT* __restrict__ x,
                           int cap, int32_t* errflag, Epi& epi, long long wait,
                           const uint8_t* __restrict__ order = nullptr) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    int32_t* scol = reinterpret_cast<int32_t*>(smem + 128);
    VT* sval = reinterpret_cast<VT*>(smem + 128 + stage_col_bytes<VT>(cap));
    BalancedTile<ACC>& B = *reinterpret_cast<BalancedTile<ACC>*>(smem + stage_bytes<VT>(cap));
    const int rows_per_tile = blockDim.x / TPR;
    const int64_t ntiles = (static_cast<int64_t>(n) + rows_per_tile - 1) / rows_per_tile;
    constexpr int VPER = 16 / sizeof(VT);  // values per 16 bytes
    const int64_t c_end = nnz & ~int64_t(3);
    const int64_t v_end = nnz & ~int64_t(VPER - 1);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * rows_per_tile;
        const int64_t r1 = r0 + rows_per_tile < n ? r0 + rows_per_tile : n;
        const int64_t e0 = rowptr[r0], e1 = rowptr[r1];
        const int64_t c_lo = e0 & ~int64_t(3);
        const int64_t c_hi = ((e1 + 3) & ~int64_t(3)) < c_end ? ((e1 + 3) & ~int64_t(3)) : c_end;
        const int64_t v_lo = e0 & ~int64_t(VPER - 1);
        const int64_t v_hi = ((e1 + VPER - 1) & ~int64_t(VPER - 1)) < v_end ? ((e1 + VPER - 1) & ~int64_t(VPER - 1))
                                                                              : v_end;
        const bool fits = ((c_hi > e1 ? c_hi : e1) - c_lo) <= cap && ((v_hi > e1 ? v_hi : e1) - v_lo) <= cap;
        if (fits) {
            if (threadIdx.x == 0) {
                fence_proxy_async();
                const uint32_t cb = c_hi > c_lo ? static_cast<uint32_t>((c_hi - c_lo) * 4) : 0u;
                const uint32_t vb = v_hi > v_lo ? static_cast<uint32_t>((v_hi - v_lo) * sizeof(VT)) : 0u;
                mbar_arrive_expect_tx(bar, cb + vb);
                if (cb) bulk_g2s(scol, col + c_lo, cb, bar);
                if (vb) bulk_g2s(sval, val + v_lo, vb, bar);
            }
            // entries past the last whole 16-byte group of the arrays
            const int64_t ct = c_hi > c_lo ? c_hi : c_lo;
            for (int64_t e = ct + threadIdx.x; e < e1; e += blockDim.x) scol[e - c_lo] = col[e];
            const int64_t vt = v_hi > v_lo ? v_hi : v_lo;
            for (int64_t e = vt + threadIdx.x; e < e1; e += blockDim.x) sval[e - v_lo] = val[e];
            const bool ok = mbar_wait(bar, phase, wait);
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) {
                    if (errflag) atomicExch(errflag, 1);
                    mbar_wait(bar, phase);  // bounded: let this block's copies land
                }
                __syncthreads();
                return false;
            }
            phase ^= 1u;
            if constexpr (BAL)
                tile_rows_balanced<VT, XT, ACC>(r0, r1, rowptr, col, val, x, scol, sval, c_lo, v_lo, true, B, epi);
            else
                tile_rows<TPR, VT, XT, ACC>(r0, r1, rowptr, col, val, x, scol, sval, c_lo, v_lo, true, epi, order);
        } else {
            if constexpr (BAL)
                tile_rows_balanced<VT, XT, ACC>(r0, r1, rowptr, col, val, x, scol, sval, c_lo, v_lo, false, B, epi);
            else
                tile_rows<TPR, VT, XT, ACC>(r0, r1, rowptr, col, val, x, scol, sval, c_lo, v_lo, false, epi, order);
        }
        __syncthreads();  // the stage is reused by the next tile
    }
    return true;
}

// Strided rows: L lanes per row stride over the row (coalesced across the
// group), partial sums combined by a shuffle tree; a grid-stride loop with
// a uniform trip count keeps the shuffles convergent.
template <int L, typename VT, typename XT, typename ACC, class Epi>
__device__ __forceinline__ void spmv_strided(int32_t n, const int32_t* __restrict__ rowptr,
                                             const int32_t* __restrict__ col, const VT* __restrict__ val,
                                             const XT* __restrict__ x, Epi& epi) {
    const int sub = threadIdx.x & (L - 1);
    const int64_t g0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / L;
    const int64_t ng = (static_cast<int64_t>(gridDim.x) * blockDim.x) / L;
    const int64_t nloop = (n + ng - 1) / ng;
    for (int64_t it = 0; it < nloop; ++it) {
        const int64_t i = g0 + it * ng;
        ACC acc = ACC(0);
        if (i < n) {
            const int32_t b = rowptr[i], e = rowptr[i + 1];
            for (int32_t k = b + sub; k < e; k += L) acc = Mul<ACC>::fma_(__ldg(&val[k]), __ldg(&x[__ldg(&col[k])]), acc);
        }
        if (L > 1) {
#pragma unroll
            for (int o = L >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, L);
        }
        if (i < n && sub == 0) epi.row(i, acc);
    }
}

// Grouped rows: groups of L consecutive lanes (L not a power of two; the
// last 32 mod L lanes of a warp idle), each group strides one row, partial
// sums combined by a fixed tree of shuffles.  For rows whose length is a
// multiple of L (81 = 27 x 3 for 3-dof elasticity) every lane does the same
// number of fmas, so FP64 warp instructions stay full.
template <int L, typename VT, typename XT, typename ACC, class Epi>
__device__ __forceinline__ void spmv_grouped(int32_t n, const int32_t* __restrict__ rowptr,
                                             const int32_t* __restrict__ col, const VT* __restrict__ val,
                                             const XT* __restrict__ x, Epi& epi) {
    constexpr int G = 32 / L;  // groups per warp
    const int lane = threadIdx.x & 31;
    const int grp = lane / L;
    const int sub = lane - grp * L;
    const bool live = grp < G;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t nloop = (n + nwarp * G - 1) / (nwarp * G);
    for (int64_t it = 0; it < nloop; ++it) {
        const int64_t i = (warp + it * nwarp) * G + grp;
        ACC acc = ACC(0);
        if (live && i < n) {
            const int32_t b = rowptr[i], e = rowptr[i + 1];
            for (int32_t k = b + sub; k < e; k += L) acc = Mul<ACC>::fma_(__ldg(&val[k]), __ldg(&x[__ldg(&col[k])]), acc);
        }
#pragma unroll
        for (int o = 1; o < L; o <<= 1) {
            const ACC other = __shfl_down_sync(0xffffffffu, acc, o);
            if ((sub & ((o << 1) - 1)) == 0 && sub + o < L) acc += other;
        }
        if (live && i < n && sub == 0) epi.row(i, acc);
    }
}

// The sliced copy of a matrix as the kernels see it (SellDev).
struct SellView {
    int32_t nslices;
    int32_t nwin;  // sorting windows
    const int32_t* kptr;
    const int2* rowlen;
    const int32_t* col;
    const void* val;
    const uint8_t* order;  // row order of the CSR's tiles (SellDev::order)
};

inline SellView sell_view(const SellDev& S) {
    return SellView{S.nslices, (S.nslices + kSellWindowSlices - 1) / kSellWindowSlices, S.kptr, S.rowlen, S.col,
                    S.val, S.order};
}

// The engines sweep tasks (grid-stride).  In slice order (ILV = false) task
// t is slice t: neighbouring warps take neighbouring rows, whose gathers
// share lines of x.  Interleaved (ILV = true), tasks run over
// 0 .. nwin * 128 - 1 and task t is slice (t mod nwin) * 128 + t / nwin:
// the windows are taken in turn, so the slices that come first in their
// window, the longest ones, are handed out first and the short ones fill
// the end of the sweep (for matrices with uneven rows, such as G^T).  -1
// marks a position past the end of a partial last window.
template <bool ILV>
__device__ __forceinline__ int64_t slice_tasks(const SellView& S) {
    return ILV ? static_cast<int64_t>(S.nwin) * kSellWindowSlices : static_cast<int64_t>(S.nslices);
}
template <bool ILV>
__device__ __forceinline__ int64_t slice_of(const SellView& S, int64_t t) {
    if (!ILV) return t;
    const int64_t sl = (t % S.nwin) * kSellWindowSlices + t / S.nwin;
    return sl < S.nslices ? sl : -1;
}

// Sliced rows: one warp per slice of 32 rows, one lane per row, each row
// summed in CSR order (the plain sequential sum).  Four entries per lane
// are loaded before their fmas; lanes past their row's length skip both.
template <typename VT, typename XT, typename ACC, class Epi>
__device__ __forceinline__ void spmv_sliced(const SellView& S, const XT* __restrict__ x, Epi& epi) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const VT* __restrict__ sval = static_cast<const VT*>(S.val);
    const int64_t ntasks = slice_tasks<false>(S);
    for (int64_t t = w0; t < ntasks; t += nw) {
        const int64_t sl = slice_of<false>(S, t);
        if (sl < 0) continue;
        const int32_t k0 = __ldg(&S.kptr[sl]);
        const int32_t K = __ldg(&S.kptr[sl + 1]) - k0;
        const int2 rl = __ldg(&S.rowlen[sl * 32 + lane]);
        const int32_t* __restrict__ cp = S.col + static_cast<int64_t>(k0) * 32 + lane;
        const VT* __restrict__ vp = sval + static_cast<int64_t>(k0) * 32 + lane;
        ACC acc = ACC(0);
        int32_t k = 0;
        for (; k + 4 <= K; k += 4) {
            int32_t c[4];
            VT v[4];
            XT xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool on = k + u < rl.y;
                c[u] = on ? __ldg(cp + static_cast<int64_t>(k + u) * 32) : 0;
                v[u] = on ? __ldg(vp + static_cast<int64_t>(k + u) * 32) : VT(0.0f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = (k + u < rl.y) ? __ldg(&x[c[u]]) : XT(0);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (k + u < rl.y) acc = Mul<ACC>::fma_(v[u], xv[u], acc);
        }
        for (; k < K; ++k) {
            if (k < rl.y) {
                const int64_t o = static_cast<int64_t>(k) * 32;
                acc = Mul<ACC>::fma_(__ldg(vp + o), __ldg(&x[__ldg(cp + o)]), acc);
            }
        }
        if (rl.x >= 0) epi.row(rl.x, acc);
    }
}

// Sliced rows, software-pipelined: the columns and values of the next U
// entries are loaded while the current U are gathered and multiplied, so
// each warp keeps its next HBM loads in flight across the dependent gathers
// of x.  Same sums, in the same order, as spmv_sliced.
template <int U, bool ILV, typename VT, typename XT, typename ACC, class Epi>
__device__ __forceinline__ void spmv_sliced_pipe(const SellView& S, const XT* __restrict__ x, Epi& epi) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const VT* __restrict__ sval = static_cast<const VT*>(S.val);
    const int64_t ntasks = slice_tasks<ILV>(S);
    for (int64_t t = w0; t < ntasks; t += nw) {
        const int64_t sl = slice_of<ILV>(S, t);
        if (sl < 0) continue;
        const int32_t k0 = __ldg(&S.kptr[sl]);
        const int32_t K = __ldg(&S.kptr[sl + 1]) - k0;
        const int2 rl = __ldg(&S.rowlen[sl * 32 + lane]);
        const int32_t* __restrict__ cp = S.col + static_cast<int64_t>(k0) * 32 + lane;
        const VT* __restrict__ vp = sval + static_cast<int64_t>(k0) * 32 + lane;
        int32_t cn[U];
        VT vn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool on = u < rl.y;
            cn[u] = on ? __ldg(cp + static_cast<int64_t>(u) * 32) : 0;
            vn[u] = on ? __ldg(vp + static_cast<int64_t>(u) * 32) : VT(0.0f);
        }
        ACC acc = ACC(0);
        for (int32_t k = 0; k < K; k += U) {
            int32_t c[U];
            VT v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                c[u] = cn[u];
                v[u] = vn[u];
            }
            if (k + U < K) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool on = k + U + u < rl.y;
                    cn[u] = on ? __ldg(cp + static_cast<int64_t>(k + U + u) * 32) : 0;
                    vn[u] = on ? __ldg(vp + static_cast<int64_t>(k + U + u) * 32) : VT(0.0f);
                }
            }
            XT xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = (k + u < rl.y) ? __ldg(&x[c[u]]) : XT(0);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (k + u < rl.y) acc = Mul<ACC>::fma_(v[u], xv[u], acc);
        }
        if (rl.x >= 0) epi.row(rl.x, acc);
    }
}

// Sliced rows staged by bulk copies: each warp owns a ring of NST
// shared-memory stages, each holding CK k-steps of one slice (CK x 32
// columns, CK x 32 values: two contiguous runs of the sliced arrays, so
// two cp.async.bulk copies, completion counted on the stage's mbarrier).
// The warp walks its slices (grid-stride over the tasks) chunk by chunk; lane 0 refills a
// stage with the chunk NST ahead as soon as the warp has consumed it, so
// the HBM stream of the next chunks is in flight while the lanes gather x
// and run the fmas of the current one.  Same sums, in the same order, as
// spmv_sliced.  Every wait is bounded: on expiry the warp raises the error
// flag, waits once more (bounded) for each copy it still has in flight and
// stops; the block then returns false in every thread.
template <int CK, typename VT>
struct StagedShape {
    static constexpr uint32_t kColBytes = CK * 32 * 4;
    static constexpr uint32_t kValBytes = CK * 32 * sizeof(VT);
    static constexpr uint32_t kStage = kColBytes + kValBytes;
    static_assert(CK % 4 == 0 && kStage % 128 == 0, "stage layout");
};

template <int CK, int NST>
__host__ __device__ inline size_t staged_warp_bytes(size_t val_size) {
    return static_cast<size_t>(NST) * (CK * 32 * 4 + CK * 32 * val_size) + 128;
}

template <int CK, int NST, typename VT, typename XT, typename ACC, class Epi>
__device__ bool spmv_sliced_staged(const SellView& S, const XT* __restrict__ x, int32_t* errflag, Epi& epi,
                                   long long wait) {
    using SH = StagedShape<CK, VT>;
    static_assert(NST >= 1 && NST <= 16, "stages");
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    unsigned char* wbase = smem + static_cast<size_t>(threadIdx.x >> 5) * (NST * SH::kStage + 128);
    uint64_t* bars = reinterpret_cast<uint64_t*>(wbase + NST * SH::kStage);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NST; ++j) mbar_init(&bars[j], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const VT* __restrict__ sval = static_cast<const VT*>(S.val);

    // issue cursor: chunk ikb of the slice of task it (warp-uniform)
    const int64_t ntasks = slice_tasks<false>(S);
    int64_t it = w0;
    int32_t ikb = 0, ik0 = 0, iK = 0;
    auto load_task = [&]() {
        const int64_t is = it < ntasks ? slice_of<false>(S, it) : -1;
        ikb = 0;
        ik0 = is >= 0 ? __ldg(&S.kptr[is]) : 0;
        iK = is >= 0 ? __ldg(&S.kptr[is + 1]) - ik0 : 0;
    };
    load_task();
    auto issue = [&](int stage) -> bool {
        while (it < ntasks && ikb >= iK) {
            it += nw;
            load_task();
        }
        if (it >= ntasks) return false;
        const int32_t kn = iK - ikb < CK ? iK - ikb : CK;
        if (lane == 0) {
            const uint32_t cb = static_cast<uint32_t>(kn) * 128u;
            const uint32_t vb = static_cast<uint32_t>(kn) * 32u * static_cast<uint32_t>(sizeof(VT));
            unsigned char* st = wbase + stage * SH::kStage;
            const int64_t off = (static_cast<int64_t>(ik0) + ikb) * 32;
            fence_proxy_async();
            mbar_arrive_expect_tx(&bars[stage], cb + vb);
            bulk_g2s(st, S.col + off, cb, &bars[stage]);
            bulk_g2s(st + SH::kColBytes, sval + off, vb, &bars[stage]);
        }
        ikb += CK;
        return true;
    };

    int inflight = 0;
    for (int j = 0; j < NST; ++j)
        if (issue(j)) ++inflight;
    int stage = 0;
    uint32_t parity = 0;  // bit j: phase parity awaited on stage j
    bool ok_warp = true;
    for (int64_t t = w0; t < ntasks && ok_warp; t += nw) {
        const int64_t sl = slice_of<false>(S, t);
        if (sl < 0) continue;
        const int32_t K = __ldg(&S.kptr[sl + 1]) - __ldg(&S.kptr[sl]);
        const int2 rl = __ldg(&S.rowlen[sl * 32 + lane]);
        ACC acc = ACC(0);
        for (int32_t kb = 0; kb < K; kb += CK) {
            const bool ok = mbar_wait(&bars[stage], (parity >> stage) & 1u, wait);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0 && errflag) atomicExch(errflag, 1);
                // bounded second wait for every copy this warp has in flight
                for (int t = 0, j = stage; t < inflight; ++t, j = (j + 1) % NST)
                    mbar_wait(&bars[j], (parity >> j) & 1u);
                __syncwarp();
                ok_warp = false;
                break;
            }
            parity ^= 1u << stage;
            --inflight;
            const int32_t* sc = reinterpret_cast<const int32_t*>(wbase + stage * SH::kStage);
            const VT* sv = reinterpret_cast<const VT*>(wbase + stage * SH::kStage + SH::kColBytes);
#pragma unroll
            for (int g = 0; g < CK; g += 4) {
                int32_t c[4];
                VT v[4];
                XT xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool on = kb + g + u < rl.y;
                    c[u] = on ? sc[(g + u) * 32 + lane] : 0;
                    v[u] = on ? sv[(g + u) * 32 + lane] : VT(0.0f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) xv[u] = (kb + g + u < rl.y) ? __ldg(&x[c[u]]) : XT(0);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (kb + g + u < rl.y) acc = Mul<ACC>::fma_(v[u], xv[u], acc);
            }
            __syncwarp();  // every lane is done with the stage before it is refilled
            if (issue(stage)) ++inflight;
            stage = stage + 1 == NST ? 0 : stage + 1;
        }
        if (ok_warp && rl.x >= 0) epi.row(rl.x, acc);
    }
    // one block-uniform verdict (the callers' reductions use block barriers)
    return __syncthreads_and(ok_warp) != 0;
}

// Balanced rows: a warp takes 32 consecutive rows and splits their
// entries evenly over its lanes (each lane a contiguous run of
// ceil(T / 32) entries, T the rows' entry count), so every FP64 fma
// instruction of the warp is full whatever the row lengths (G^T: from 1 to
// ~40 entries per row, where one lane per row leaves about half the lanes
// idle).  A row inside one run is the sequential sum of its entries; a row
// cut by run boundaries is summed from its pieces in lane order by the lane
// that holds its last entry.  Shared memory per warp: kBalancedWarpBytes.
constexpr int kModeBalanced = 301;

template <typename ACC>
struct BalancedWarp {
    int32_t rp[33];   // row pointers of the warp's rows (rp[nr] = end)
    int32_t prow[32]; // row continued past the end of each lane's run (-1: none)
    ACC part[32];     // that row's partial sum over the lane's run
};

template <typename VT, typename XT, typename ACC, class Epi>
__device__ __forceinline__ void spmv_balanced(int32_t n, const int32_t* __restrict__ rowptr,
                                              const int32_t* __restrict__ col, const VT* __restrict__ val,
                                              const XT* __restrict__ x, Epi& epi) {
    extern __shared__ __align__(16) unsigned char smem[];
    BalancedWarp<ACC>& W = reinterpret_cast<BalancedWarp<ACC>*>(smem)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t r0 = w0 * 32; r0 < n; r0 += nw * 32) {
        const int nr = static_cast<int>(n - r0 < 32 ? n - r0 : 32);
        const int32_t e_all = __ldg(&rowptr[r0 + nr]);
        W.rp[lane] = lane < nr ? __ldg(&rowptr[r0 + lane]) : e_all;
        if (lane == 0) W.rp[32] = e_all;
        W.prow[lane] = -1;
        __syncwarp();
        const int32_t E0 = W.rp[0];
        const int32_t T = e_all - E0;
        const int32_t C = (T + 31) >> 5;
        const int32_t s = E0 + lane * C;
        const int32_t e_end = s + C < e_all ? s + C : e_all;
        ACC head = ACC(0);
        int head_row = -1;
        if (T == 0) {
            if (lane < nr) epi.row(r0 + lane, ACC(0));
        } else if (s < e_end) {
            // first row of the run: row 0 for lane 0 (empty leading rows
            // included), else the last row starting at or before s
            int k = 0;
            if (lane > 0) {
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (k + step < nr && W.rp[k + step] <= s) k += step;
            }
            ACC acc = ACC(0);
            auto close_row = [&]() {
                if (W.rp[k] >= s) {
                    epi.row(r0 + k, acc);  // the whole row lies in this run
                } else {
                    head = acc;            // the row began in an earlier run
                    head_row = k;
                }
                ++k;
                acc = ACC(0);
            };
            int32_t e = s;
            for (; e + 4 <= e_end; e += 4) {
                int32_t c4[4];
                VT v4[4];
                XT x4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    c4[u] = __ldg(&col[e + u]);
                    v4[u] = __ldg(&val[e + u]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) x4[u] = __ldg(&x[c4[u]]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    while (W.rp[k + 1] <= e + u) close_row();
                    acc = Mul<ACC>::fma_(v4[u], x4[u], acc);
                }
            }
            for (; e < e_end; ++e) {
                while (W.rp[k + 1] <= e) close_row();
                acc = Mul<ACC>::fma_(__ldg(&val[e]), __ldg(&x[__ldg(&col[e])]), acc);
            }
            // rows that end with this run (and empty rows right after it)
            while (k < nr && W.rp[k + 1] <= e_end) close_row();
            if (k < nr) {
                W.part[lane] = acc;
                W.prow[lane] = k;
            }
        }
        __syncwarp();
        if (head_row >= 0) {
            // pieces of the row from the lane of its first entry onwards
            const int L0 = (W.rp[head_row] - E0) / C;
            ACC sum = W.part[L0];
            for (int L = L0 + 1; L < lane; ++L) sum += W.part[L];
            sum += head;
            epi.row(r0 + head_row, sum);
        }
        __syncwarp();
    }
}

constexpr int kModeSliced = 200;
constexpr int kModeSlicedPipe = 201;
constexpr int kModeSlicedPipe8 = 202;
constexpr int kModeSlicedPipeIlv = 203;   // 201 with the windows interleaved
constexpr int kModeSlicedStaged8 = 210;   // 8 k-steps per stage, 3 stages
constexpr int kModeSlicedStaged16 = 211;  // 16 k-steps per stage, 2 stages
constexpr int kStagedWarps = 4;           // warps per block of the staged engines

// SpMV row engine.  MODE 1, 2, 4, 8: strided with MODE lanes per row;
// MODE 3, 6: grouped with MODE lanes per row; MODE 101, 102: TMA-staged
// tiles with MODE - 100 threads per row; MODE 103: TMA-staged tiles with the
// balanced row loop (tile_rows_balanced); MODE 104: as 101, each tile's rows
// taken longest first (SellDev::order, built with the sliced copy), so a
// warp's rows have similar lengths; MODE 200 - 203: the sliced copy,
// one lane per row (201, 202 software-pipelined by 4 and 8 entries, 203 as
// 201 with the windows interleaved);
// MODE 210, 211: the sliced copy staged through shared memory by bulk
// copies (8 k-steps x 3 stages, 16 k-steps x 2 stages per warp).
template <int MODE, typename VT, typename XT, typename ACC, class Epi>
__device__ __forceinline__ bool spmv_rows(int32_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                                          const int32_t* __restrict__ col, const VT* __restrict__ val,
                                          const XT* __restrict__ x, int cap, int32_t* errflag, Epi& epi,
                                          const SellView& sv, long long wait = kWaitCycles) {
    if constexpr (MODE == kModeSliced) {
        spmv_sliced<VT, XT, ACC>(sv, x, epi);
        return true;
    } else if constexpr (MODE == kModeSlicedPipe) {
        spmv_sliced_pipe<4, false, VT, XT, ACC>(sv, x, epi);
        return true;
    } else if constexpr (MODE == kModeSlicedPipe8) {
        spmv_sliced_pipe<8, false, VT, XT, ACC>(sv, x, epi);
        return true;
    } else if constexpr (MODE == kModeSlicedPipeIlv) {
        spmv_sliced_pipe<4, true, VT, XT, ACC>(sv, x, epi);
        return true;
    } else if constexpr (MODE == kModeSlicedStaged8) {
        return spmv_sliced_staged<8, 3, VT, XT, ACC>(sv, x, errflag, epi, wait);
    } else if constexpr (MODE == kModeSlicedStaged16) {
        return spmv_sliced_staged<16, 2, VT, XT, ACC>(sv, x, errflag, epi, wait);
    } else if constexpr (MODE == kModeBalanced) {
        spmv_balanced<VT, XT, ACC>(n, rowptr, col, val, x, epi);
        return true;
    } else if constexpr (MODE == 104) {
        // tiles of kTileOrderRows rows (the plan's block size), rows by length
        return spmv_tiles<1, VT, XT, ACC, Epi>(n, nnz, rowptr, col, val, x, cap, errflag, epi, wait, sv.order);
    } else if constexpr (MODE == 103) {
        return spmv_tiles<1, VT, XT, ACC, Epi, true>(n, nnz, rowptr, col, val, x, cap, errflag, epi, wait);
    } else if constexpr (MODE > 100) {
        return spmv_tiles<MODE - 100, VT, XT, ACC>(n, nnz, rowptr, col, val, x, cap, errflag, epi, wait);
    } else if constexpr (MODE == 3 || MODE == 6) {
        spmv_grouped<MODE, VT, XT, ACC>(n, rowptr, col, val, x, epi);
        return true;
    } else {
        spmv_strided<MODE, VT, XT, ACC>(n, rowptr, col, val, x, epi);
        return true;
    }
}

}  // namespace tiled

// Launch shape of one SpMV row engine.
struct SpmvMode {
    int mode = 4;       // see tiled::spmv_rows
    int threads = 256;
    int blocks = 1;
    size_t smem = 0;
    int cap = 0;
};

// Roles of the matrices whose engine choice is cached.
enum SpmvRole : int { ROLE_A = 0, ROLE_G = 1, ROLE_GT = 2 };

// How a solve launches a role's product (fused with its dot product or
// vector update): y = C x with engine m on a stream.  The engine timing
// runs this launch when given, so the engines are ranked by the kernel
// that will run (a fused kernel's registers, and so its resident blocks,
// differ from the plain product's).  x_float: x holds n floats.
struct RoleLaunch {
    bool x_float = false;
    std::function<afsai_status(const SpmvMode&, const void*, void*, cudaStream_t)> launch;
};

// Engine for a matrix: timed once per (role, shape, value type) among the
// candidate engines on the given stream (with `how`, else the plain
// product of the role), then cached.  Must not be called during stream
// capture.  With allow_tuning = false nothing is timed or allocated: the
// cached engine is used if there is one, else a default chosen from the
// average row length.
afsai_status spmv_mode_for(int role, const CsrDev& C, cudaStream_t st, SpmvMode* out, bool allow_tuning = true,
                           const RoleLaunch* how = nullptr);

// n values with full significands and both signs, +-(1 + f) (doubles, or
// floats with as_float), to time products on the data they see.
void fill_tune_vector(void* x, int32_t n, bool as_float, cudaStream_t st);

// Whether a sliced copy of C (and the tile row order built with it) would
// serve `role`: the engine is pinned to one that reads them, or it has not
// been chosen yet for this shape with a sliced copy, or such an engine was
// chosen.
bool spmv_wants_sliced(int role, const CsrDev& C);

// Whether the tile row order (engine 104) would serve `role`: the engine is
// pinned to 104, or not chosen yet for this shape with a sliced copy, or
// 104 was chosen.
bool spmv_wants_order(int role, const CsrDev& C);

// y = C x with the engine `m` and the value/vector types of `role`.
afsai_status spmv_launch_role(int role, const SpmvMode& m, const CsrDev& C, const void* x, void* y, cudaStream_t st);

// Host-side launch plan of a tiled SpMV.
struct TiledPlan {
    int threads = 128;  // block size
    int tpr = 1;        // threads per row
    int cap = 0;        // stage capacity in entries
    size_t smem = 0;    // dynamic shared memory per block
    int blocks = 1;     // persistent grid
    bool ok = false;    // false: use the untiled kernels
};

// Plans a tiled SpMV for a CSR with the given shape and value size.
TiledPlan plan_tiled(int32_t n, int64_t nnz, int32_t max_row, size_t val_size, const void* col, const void* val,
                     int tpr = 0, size_t extra_smem = 0);

}  // namespace afsai
