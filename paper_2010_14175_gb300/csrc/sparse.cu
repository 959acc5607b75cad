// Sparse building blocks: exclusive scan, G -> G^T transpose, CSR SpMV and
// the preconditioner application z = G^T (G r) (Eq. "prec").
//
// SpMV (Section 3, "miniwarp"): a group of L lanes owns one row, L chosen
// from the average row length.  On GB300 an FP64 warp instruction costs the
// same whatever the number of active lanes, so the group size trades FP64
// issue slots (L = 1: one fma per entry, no shuffle reduction) against
// memory coalescing (larger L): short rows (7-point stencils, rows of G) use
// one lane per row, long rows (elasticity, 81 per row) use small groups.
#include <algorithm>
#include <climits>
#include <cstdlib>

#include "afsai_internal.cuh"

namespace afsai {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// exclusive scan of int32 counts (three passes, int64 block sums)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t* sh, int64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int64_t w = (lane < (kScanThreads >> 5)) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += t;
        }
        if (lane < (kScanThreads >> 5)) sh[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v += sh[warp - 1];
    if (total) *total = sh[(kScanThreads >> 5) - 1];
    __syncthreads();
    return v;
}

__global__ void scan_tile_sums(const int32_t* __restrict__ in, int32_t n, int64_t* __restrict__ sums) {
    __shared__ int64_t sh[32];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
    int64_t v = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t idx = base + threadIdx.x * kScanItems + k;
        if (idx < n) v += in[idx];
    }
    int64_t tot;
    block_incl_scan(v, sh, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_sums_single(int64_t* __restrict__ sums, int32_t nb) {
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int32_t base = 0; base < nb; base += kScanThreads) {
        const int32_t idx = base + threadIdx.x;
        const int64_t v = idx < nb ? sums[idx] : 0;
        int64_t tot;
        const int64_t inc = block_incl_scan(v, sh, &tot);
        if (idx < nb) sums[idx] = carry + inc - v;  // exclusive
        carry += tot;
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void scan_tiles(const int32_t* __restrict__ in, int32_t n, const int64_t* __restrict__ offs,
                           int32_t* __restrict__ out, int32_t* __restrict__ overflow) {
    __shared__ int64_t sh[32];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
    int64_t loc[kScanItems];
    int64_t v = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t idx = base + threadIdx.x * kScanItems + k;
        loc[k] = (idx < n) ? in[idx] : 0;
        v += loc[k];
    }
    const int64_t inc = block_incl_scan(v, sh, nullptr);
    int64_t run = offs[blockIdx.x] + inc - v;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t idx = base + threadIdx.x * kScanItems + k;
        if (idx < n) {
            if (run > INT_MAX) *overflow = 1;
            out[idx] = static_cast<int32_t>(run);
        }
        run += loc[k];
    }
}

__global__ void scan_write_total(int32_t* __restrict__ out, int32_t n, const int64_t* __restrict__ sums, int32_t nb,
                                 int32_t* __restrict__ overflow) {
    const int64_t t = sums[nb];
    if (t > INT_MAX) *overflow = 1;
    out[n] = static_cast<int32_t>(t);
}

// ---------------------------------------------------------------------------
// transpose G -> G^T (counting sort by column, then per-row sort by row)
// ---------------------------------------------------------------------------
__global__ void count_cols(const int32_t* __restrict__ col, int64_t nnz, int32_t* __restrict__ cnt) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < nnz;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        atomicAdd(&cnt[col[e]], 1);
}

template <typename VT>
__global__ void scatter_transpose(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const VT* __restrict__ val, const int32_t* __restrict__ trowptr,
                                  int32_t* __restrict__ fill, int32_t* __restrict__ tcol, VT* __restrict__ tval) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = gw; i < n; i += nw) {
        for (int32_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
            const int32_t j = col[e];
            const int32_t pos = trowptr[j] + atomicAdd(&fill[j], 1);
            tcol[pos] = static_cast<int32_t>(i);
            tval[pos] = val[e];
        }
    }
}

// Rows of G^T are written in arrival order; sort each by column (the row
// index of G) so that every G^T row is sorted and the SpMV order is fixed.
// Rank sort: an entry's position is the number of smaller keys in its row
// (keys are distinct).  Reads from the unsorted copy, writes the final.
template <typename VT>
__global__ void sort_rows_rank(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ ucol,
                               const VT* __restrict__ uval, int32_t* __restrict__ col, VT* __restrict__ val) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t j = gw; j < n; j += nw) {
        const int32_t b = rowptr[j], e = rowptr[j + 1], len = e - b;
        if (len <= 32) {
            const int32_t k = lane < len ? ucol[b + lane] : INT_MAX;
            int rank = 0;
            for (int t = 0; t < len; ++t) {
                const int32_t o = __shfl_sync(kFull, k, t);
                rank += (o < k);
            }
            if (lane < len) {
                col[b + rank] = k;
                val[b + rank] = uval[b + lane];
            }
        } else {
            for (int32_t u = lane; u < len; u += 32) {
                const int32_t k = ucol[b + u];
                int rank = 0;
                for (int32_t t = 0; t < len; ++t) rank += (ucol[b + t] < k);
                col[b + rank] = k;
                val[b + rank] = uval[b + u];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// SpMV kernels
// ---------------------------------------------------------------------------
template <typename VT>
__device__ __forceinline__ double as_f64(VT v) {
    return static_cast<double>(v);
}
template <>
__device__ __forceinline__ double as_f64<__nv_bfloat16>(__nv_bfloat16 v) {
    return static_cast<double>(__bfloat162float(v));
}
template <typename VT>
__device__ __forceinline__ float as_f32(VT v) {
    return static_cast<float>(v);
}
template <>
__device__ __forceinline__ float as_f32<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

// FP64 values and vectors: one lane per row, fma in CSR order.
__global__ void spmv_f64_scalar(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t b = rowptr[i], e = rowptr[i + 1];
        double acc = 0.0;
        for (int32_t k = b; k < e; ++k) acc = fma(__ldg(&val[k]), __ldg(&x[__ldg(&col[k])]), acc);
        y[i] = acc;
    }
}

// FP64: L lanes per row, lanes stride the row, shuffle reduction.
template <int L>
__global__ void spmv_f64_group(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
    const int sub = threadIdx.x & (L - 1);
    const int64_t g0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / L;
    const int64_t ng = (static_cast<int64_t>(gridDim.x) * blockDim.x) / L;
    const int64_t nloop = (n + ng - 1) / ng;  // uniform trip count keeps the shuffles convergent
    for (int64_t it = 0; it < nloop; ++it) {
        const int64_t i = g0 + it * ng;
        double acc = 0.0;
        if (i < n) {
            const int32_t b = rowptr[i], e = rowptr[i + 1];
            for (int32_t k = b + sub; k < e; k += L) acc = fma(__ldg(&val[k]), __ldg(&x[__ldg(&col[k])]), acc);
        }
#pragma unroll
        for (int o = L >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o, L);
        if (i < n && sub == 0) y[i] = acc;
    }
}

// Reduced-precision G / G^T (fp32 or bf16 values): fp32 arithmetic, x read
// as XT (double or float), y written as YT.
template <typename VT, typename XT, typename YT>
__global__ void spmv_lowp_scalar(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const VT* __restrict__ val, const XT* __restrict__ x, YT* __restrict__ y) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t b = rowptr[i], e = rowptr[i + 1];
        float acc = 0.0f;
        for (int32_t k = b; k < e; ++k)
            acc = fmaf(as_f32<VT>(__ldg(&val[k])), static_cast<float>(__ldg(&x[__ldg(&col[k])])), acc);
        y[i] = static_cast<YT>(acc);
    }
}

int spmv_group_for(int64_t n, int64_t nnz) {
    static int forced = [] {
        const char* s = std::getenv("AFSAI_SPMV_GROUP");
        return s ? std::atoi(s) : 0;
    }();
    if (forced == 1 || forced == 2 || forced == 4 || forced == 8 || forced == 16 || forced == 32) return forced;
    const double avg = n > 0 ? static_cast<double>(nnz) / n : 0.0;
    if (avg <= 16.0) return 1;
    if (avg <= 48.0) return 2;
    return 4;
}

int grid_for(int64_t work_items, int threads) {
    const int64_t need = (work_items + threads - 1) / threads;
    const int64_t cap = static_cast<int64_t>(num_sms()) * (2048 / threads) * 4;
    return static_cast<int>(std::max<int64_t>(1, std::min(need, cap)));
}

}  // namespace

int num_sms() {
    static int sms = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return sms;
}

afsai_status exclusive_scan_i32(const int32_t* in, int32_t* out, int32_t n, cudaStream_t st, int64_t* total_host) {
    const int32_t nb = (n + kScanTile - 1) / kScanTile;
    DevBuf<int64_t> sums;
    DevBuf<int32_t> ovf;
    AFSAI_TRY(sums.alloc(static_cast<size_t>(nb) + 1, st));
    AFSAI_TRY(ovf.alloc(1, st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(ovf.p, 0, sizeof(int32_t), st));
    if (nb > 0) {
        scan_tile_sums<<<nb, kScanThreads, 0, st>>>(in, n, sums.p);
        scan_sums_single<<<1, kScanThreads, 0, st>>>(sums.p, nb);
        scan_tiles<<<nb, kScanThreads, 0, st>>>(in, n, sums.p, out, ovf.p);
        count_launches(3);
    } else {
        AFSAI_CUDA_TRY(cudaMemsetAsync(sums.p, 0, sizeof(int64_t), st));
    }
    scan_write_total<<<1, 1, 0, st>>>(out, n, sums.p, nb, ovf.p);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    int64_t tot = 0;
    int32_t of = 0;
    AFSAI_CUDA_TRY(cudaMemcpyAsync(&tot, sums.p + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    AFSAI_CUDA_TRY(cudaMemcpyAsync(&of, ovf.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    if (of) return fail(AFSAI_ENOTSUP, "more than 2^31-1 entries in a CSR matrix");
    if (total_host) *total_host = tot;
    return AFSAI_OK;
}

template <typename VT>
static afsai_status transpose_typed(const CsrDev& G, CsrDev* Gt, cudaStream_t st) {
    const int32_t n = G.n;
    DevBuf<int32_t> cnt, ucol;
    DevBuf<VT> uval;
    AFSAI_TRY(cnt.alloc(static_cast<size_t>(n) + 1, st));
    AFSAI_TRY(ucol.alloc(std::max<int64_t>(G.nnz, 1), st));
    AFSAI_TRY(uval.alloc(std::max<int64_t>(G.nnz, 1), st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (n + 1), st));
    const int threads = 256;
    count_cols<<<grid_for(G.nnz, threads), threads, 0, st>>>(G.col, G.nnz, cnt.p);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    Gt->n = n;
    Gt->nnz = G.nnz;
    Gt->vtype = G.vtype;
    AFSAI_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&Gt->rowptr), sizeof(int32_t) * (n + 1), st));
    AFSAI_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&Gt->col), sizeof(int32_t) * std::max<int64_t>(G.nnz, 1), st));
    AFSAI_CUDA_TRY(cudaMallocAsync(&Gt->val, sizeof(VT) * std::max<int64_t>(G.nnz, 1), st));
    int64_t tot = 0;
    AFSAI_TRY(exclusive_scan_i32(cnt.p, Gt->rowptr, n, st, &tot));
    AFSAI_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (n + 1), st));
    scatter_transpose<VT><<<grid_for(static_cast<int64_t>(n) * 32, threads), threads, 0, st>>>(
        n, G.rowptr, G.col, static_cast<const VT*>(G.val), Gt->rowptr, cnt.p, ucol.p, uval.p);
    AFSAI_CUDA_TRY(cudaGetLastError());
    sort_rows_rank<VT><<<grid_for(static_cast<int64_t>(n) * 32, threads), threads, 0, st>>>(
        n, Gt->rowptr, ucol.p, uval.p, Gt->col, static_cast<VT*>(Gt->val));
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return AFSAI_OK;
}

afsai_status build_transpose(const CsrDev& G, CsrDev* Gt, cudaStream_t st) {
    afsai_status s;
    if (G.vtype == VAL_F64)
        s = transpose_typed<double>(G, Gt, st);
    else if (G.vtype == VAL_F32)
        s = transpose_typed<float>(G, Gt, st);
    else
        s = transpose_typed<__nv_bfloat16>(G, Gt, st);
    if (s != AFSAI_OK) return s;
    // longest row of G^T (host needs it only for reporting)
    Gt->max_row = 0;
    return AFSAI_OK;
}

afsai_status spmv_csr(const CsrDev& A, const double* x, double* y, cudaStream_t st) {
    if (A.vtype != VAL_F64) return fail(AFSAI_EINVAL, "spmv_csr expects FP64 values");
    const int threads = 256;
    const int L = spmv_group_for(A.n, A.nnz);
    const auto* v = static_cast<const double*>(A.val);
    switch (L) {
        case 1:
            spmv_f64_scalar<<<grid_for(A.n, threads), threads, 0, st>>>(A.n, A.rowptr, A.col, v, x, y);
            break;
        case 2:
            spmv_f64_group<2><<<grid_for(int64_t(A.n) * 2, threads), threads, 0, st>>>(A.n, A.rowptr, A.col, v, x, y);
            break;
        case 4:
            spmv_f64_group<4><<<grid_for(int64_t(A.n) * 4, threads), threads, 0, st>>>(A.n, A.rowptr, A.col, v, x, y);
            break;
        case 8:
            spmv_f64_group<8><<<grid_for(int64_t(A.n) * 8, threads), threads, 0, st>>>(A.n, A.rowptr, A.col, v, x, y);
            break;
        case 16:
            spmv_f64_group<16><<<grid_for(int64_t(A.n) * 16, threads), threads, 0, st>>>(A.n, A.rowptr, A.col, v, x, y);
            break;
        default:
            spmv_f64_group<32><<<grid_for(int64_t(A.n) * 32, threads), threads, 0, st>>>(A.n, A.rowptr, A.col, v, x, y);
            break;
    }
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFSAI_OK;
}

// t = G r ; z = G^T t.  For fp32/bf16 G the intermediate t is fp32 (t
// points to n doubles of scratch, used as n floats).
afsai_status apply_precond(const afsai_precond* M, const double* r, double* t, double* z, cudaStream_t st) {
    const CsrDev& G = M->G;
    const CsrDev& Gt = M->Gt;
    if (G.vtype == VAL_F64) {
        AFSAI_TRY(spmv_csr(G, r, t, st));
        AFSAI_TRY(spmv_csr(Gt, t, z, st));
        return AFSAI_OK;
    }
    const int threads = 256;
    float* tf = reinterpret_cast<float*>(t);
    if (G.vtype == VAL_F32) {
        spmv_lowp_scalar<float, double, float><<<grid_for(G.n, threads), threads, 0, st>>>(
            G.n, G.rowptr, G.col, static_cast<const float*>(G.val), r, tf);
        spmv_lowp_scalar<float, float, double><<<grid_for(G.n, threads), threads, 0, st>>>(
            Gt.n, Gt.rowptr, Gt.col, static_cast<const float*>(Gt.val), tf, z);
    } else {
        spmv_lowp_scalar<__nv_bfloat16, double, float><<<grid_for(G.n, threads), threads, 0, st>>>(
            G.n, G.rowptr, G.col, static_cast<const __nv_bfloat16*>(G.val), r, tf);
        spmv_lowp_scalar<__nv_bfloat16, float, double><<<grid_for(G.n, threads), threads, 0, st>>>(
            Gt.n, Gt.rowptr, Gt.col, static_cast<const __nv_bfloat16*>(Gt.val), tf, z);
    }
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return AFSAI_OK;
}

void free_csr(CsrDev* A, cudaStream_t st) {
    if (A->rowptr) cudaFreeAsync(A->rowptr, st);
    if (A->col) cudaFreeAsync(A->col, st);
    if (A->val) cudaFreeAsync(A->val, st);
    A->rowptr = nullptr;
    A->col = nullptr;
    A->val = nullptr;
}

}  // namespace afsai
