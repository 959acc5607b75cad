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

// Bounded wait for the given phase parity; false if the deadline passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase)) {
        if (clock64() - t0 > kWaitCycles) return false;
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
// (called by the first thread of the row's group).
template <int TPR, typename VT, typename XT, typename ACC, class Epi>
__device__ __forceinline__ void tile_rows(int64_t r0, int64_t r1, const int32_t* __restrict__ rowptr,
                                          const int32_t* __restrict__ col, const VT* __restrict__ val,
                                          const XT* __restrict__ x, const int32_t* scol, const VT* sval,
                                          int64_t c_lo, int64_t v_lo, bool staged, Epi& epi) {
    const int t = threadIdx.x;
    const int64_t i = r0 + t / TPR;
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

// The tile loop.  Returns false if a bounded wait expired (error flag set).
template <int TPR, typename VT, typename XT, typename ACC, class Epi>
__device__ bool spmv_tiles(int32_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                           const int32_t* __restrict__ col, const VT* __restrict__ val, const XT* __restrict__ x,
                           int cap, int32_t* errflag, Epi& epi) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    int32_t* scol = reinterpret_cast<int32_t*>(smem + 128);
    VT* sval = reinterpret_cast<VT*>(smem + 128 + stage_col_bytes<VT>(cap));
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
            const bool ok = mbar_wait(bar, phase);
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) {
                    if (errflag) atomicExch(errflag, 1);
                    mbar_wait(bar, phase);  // bounded: let this block's copies land
                }
                __syncthreads();
                return false;
            }
            phase ^= 1u;
            tile_rows<TPR, VT, XT, ACC>(r0, r1, rowptr, col, val, x, scol, sval, c_lo, v_lo, true, epi);
        } else {
            tile_rows<TPR, VT, XT, ACC>(r0, r1, rowptr, col, val, x, scol, sval, c_lo, v_lo, false, epi);
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

// SpMV row engine.  MODE 1, 2, 4, 8: strided with MODE lanes per row;
// MODE 3, 6: grouped with MODE lanes per row; MODE 101, 102: TMA-staged
// tiles with MODE - 100 threads per row.
template <int MODE, typename VT, typename XT, typename ACC, class Epi>
__device__ __forceinline__ bool spmv_rows(int32_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                                          const int32_t* __restrict__ col, const VT* __restrict__ val,
                                          const XT* __restrict__ x, int cap, int32_t* errflag, Epi& epi) {
    if constexpr (MODE > 100) {
        return spmv_tiles<MODE - 100, VT, XT, ACC>(n, nnz, rowptr, col, val, x, cap, errflag, epi);
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

// Engine for a matrix: timed once per (role, shape, value type) among the
// candidate engines on the given stream, then cached.  Must not be called
// during stream capture.  With allow_tuning = false nothing is timed or
// allocated: the cached engine is used if there is one, else a default
// chosen from the average row length.
afsai_status spmv_mode_for(int role, const CsrDev& C, cudaStream_t st, SpmvMode* out, bool allow_tuning = true);

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
                     int tpr = 0);

}  // namespace afsai
