// Preconditioned conjugate gradients with M^{-1} = G^T G (Eq. "prec"),
// stopping at ||r_k|| <= rtol ||b|| (Section 5.2: an 8-order reduction).
//
// Standard (Hestenes-Stiefel) PCG, one iteration =
//   q = A p,            pq = p.q,  alpha = rz / pq           [spmv_dot]
//   x += alpha p, r -= alpha q,    rr = r.r, convergence test [update_xr]
//   t = G r                                                   [spmv_G]
//   z = G^T t,          rz' = r.z, beta = rz' / rz            [spmv_Gt_dot]
//   p = z + beta p                                            [update_p]
// All scalars live in device memory.  Each reduction is deterministic: every
// block writes one partial, and the last block to finish (atomic ticket)
// sums the partials in a fixed order and derives alpha, beta or the
// convergence flag.  Once converged, every kernel returns at entry, so
// iterations can be enqueued ahead in a CUDA graph of several iterations
// and the host only polls the flag between graph launches.
//
// Residual, dot products, alpha and beta are FP64 whatever the precision of
// G; with an FP32/BF16 G the two triangular products run in FP32.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <type_traits>
#include <vector>

#include "afsai_internal.cuh"

namespace afsai {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

struct Scalars {
    double rz;
    double alpha;
    double beta;
    double rr;
    double bb;
    double tol2;
    int32_t done;   // 0 running, 1 converged, 2 maxit reached
    int32_t iters;
    int32_t maxit;
    int32_t pad;
    unsigned ticket[8];
};

// Block sum of one or two values (fixed shuffle tree, then warp 0).
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double (*sh)[32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], o);
        if (lane == 0) sh[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double w = lane < (kThreads >> 5) ? sh[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
            v[k] = w;
        }
    }
}

// Writes this block's partial(s); returns true in the last block to
// arrive, which then holds the grid totals in v (thread 0).
template <int K>
__device__ bool grid_sum(double (&v)[K], double* partials, unsigned* ticket) {
    __shared__ double sh[K][32];
    __shared__ bool last;
    block_sum<K>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) partials[k * gridDim.x + blockIdx.x] = v[k];
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        acc[k] = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            acc[k] += reinterpret_cast<volatile double*>(partials)[k * gridDim.x + b];
    }
    __syncthreads();
    block_sum<K>(acc, sh);
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = acc[k];
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

template <typename VT>
__device__ __forceinline__ double ld_f64(const VT* p) {
    return static_cast<double>(__ldg(p));
}
__device__ __forceinline__ float ld_f32(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_f32(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Row i of an FP64 CSR times x, by a group of L lanes (L = 1: sequential).
template <int L>
__device__ __forceinline__ double row_dot_f64(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                              const double* __restrict__ val, const double* __restrict__ x, int64_t i,
                                              int64_t n, int sub) {
    double acc = 0.0;
    if (i < n) {
        const int32_t b = rowptr[i], e = rowptr[i + 1];
        for (int32_t k = b + sub; k < e; k += L) acc = fma(__ldg(&val[k]), __ldg(&x[__ldg(&col[k])]), acc);
    }
    if (L > 1) {
#pragma unroll
        for (int o = L >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o, L);
    }
    return acc;
}

// ---- init: r = b - q (q = A x), rr = r.r, bb = b.b ----------------------
__global__ void k_init_residual(int32_t n, const double* __restrict__ b, const double* __restrict__ q,
                                double* __restrict__ r, Scalars* s, double* partials, double rtol) {
    double v[2] = {0.0, 0.0};
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double ri = b[i] - q[i];
        r[i] = ri;
        v[0] = fma(ri, ri, v[0]);
        v[1] = fma(b[i], b[i], v[1]);
    }
    if (grid_sum<2>(v, partials, &s->ticket[0]) && threadIdx.x == 0) {
        s->rr = v[0];
        s->bb = v[1];
        s->tol2 = rtol * rtol * v[1];
        s->iters = 0;
        s->done = (v[0] <= s->tol2) ? 1 : 0;
    }
}

// ---- p = z, rz = r.z ------------------------------------------------------
__global__ void k_init_p(int32_t n, const double* __restrict__ r, const double* __restrict__ z, double* __restrict__ p,
                         Scalars* s, double* partials) {
    double v[1] = {0.0};
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        p[i] = z[i];
        v[0] = fma(r[i], z[i], v[0]);
    }
    if (grid_sum<1>(v, partials, &s->ticket[1]) && threadIdx.x == 0) s->rz = v[0];
}

// ---- q = A p, pq = p.q, alpha = rz / pq ----------------------------------
template <int L>
__global__ void k_spmv_A_dot(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ p, double* __restrict__ q,
                             Scalars* s, double* partials) {
    if (s->done) return;
    const int sub = threadIdx.x & (L - 1);
    const int64_t g0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / L;
    const int64_t ng = (static_cast<int64_t>(gridDim.x) * blockDim.x) / L;
    const int64_t nloop = (n + ng - 1) / ng;
    double v[1] = {0.0};
    for (int64_t it = 0; it < nloop; ++it) {
        const int64_t i = g0 + it * ng;
        const double qi = row_dot_f64<L>(rowptr, col, val, p, i, n, sub);
        if (i < n && sub == 0) {
            q[i] = qi;
            v[0] = fma(p[i], qi, v[0]);
        }
    }
    if (grid_sum<1>(v, partials, &s->ticket[2]) && threadIdx.x == 0) s->alpha = s->rz / v[0];
}

// ---- x += alpha p, r -= alpha q, rr = r.r, convergence --------------------
__global__ void k_update_xr(int32_t n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, Scalars* s, double* partials) {
    if (s->done) return;
    const double alpha = s->alpha;
    double v[1] = {0.0};
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        v[0] = fma(ri, ri, v[0]);
    }
    if (grid_sum<1>(v, partials, &s->ticket[3]) && threadIdx.x == 0) {
        s->rr = v[0];
        s->iters += 1;
        if (v[0] <= s->tol2)
            s->done = 1;
        else if (s->iters >= s->maxit)
            s->done = 2;
    }
}

// ---- t = G r (FP64 G) ------------------------------------------------------
template <int L>
__global__ void k_spmv_G_f64(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ r, double* __restrict__ t,
                             const Scalars* s, int init) {
    if (!init && s->done) return;
    const int sub = threadIdx.x & (L - 1);
    const int64_t g0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / L;
    const int64_t ng = (static_cast<int64_t>(gridDim.x) * blockDim.x) / L;
    const int64_t nloop = (n + ng - 1) / ng;
    for (int64_t it = 0; it < nloop; ++it) {
        const int64_t i = g0 + it * ng;
        const double ti = row_dot_f64<L>(rowptr, col, val, r, i, n, sub);
        if (i < n && sub == 0) t[i] = ti;
    }
}

// ---- z = G^T t, rz' = r.z, beta (FP64 G) -----------------------------------
template <int L>
__global__ void k_spmv_Gt_dot_f64(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, const double* __restrict__ t,
                                  const double* __restrict__ r, double* __restrict__ z, Scalars* s, double* partials,
                                  int init) {
    if (!init && s->done) return;
    const int sub = threadIdx.x & (L - 1);
    const int64_t g0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / L;
    const int64_t ng = (static_cast<int64_t>(gridDim.x) * blockDim.x) / L;
    const int64_t nloop = (n + ng - 1) / ng;
    double v[1] = {0.0};
    for (int64_t it = 0; it < nloop; ++it) {
        const int64_t i = g0 + it * ng;
        const double zi = row_dot_f64<L>(rowptr, col, val, t, i, n, sub);
        if (i < n && sub == 0) {
            z[i] = zi;
            v[0] = fma(r[i], zi, v[0]);
        }
    }
    if (grid_sum<1>(v, partials, &s->ticket[4]) && threadIdx.x == 0) {
        if (init) {
            s->rz = v[0];
        } else {
            s->beta = v[0] / s->rz;
            s->rz = v[0];
        }
    }
}

// ---- reduced-precision G: t = G r (fp32 out), z = G^T t (fp64 out) ---------
template <typename VT>
__global__ void k_spmv_G_lowp(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const VT* __restrict__ val, const double* __restrict__ r, float* __restrict__ t,
                              const Scalars* s, int init) {
    if (!init && s->done) return;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t b = rowptr[i], e = rowptr[i + 1];
        float acc = 0.0f;
        for (int32_t k = b; k < e; ++k) acc = fmaf(ld_f32(&val[k]), static_cast<float>(__ldg(&r[__ldg(&col[k])])), acc);
        t[i] = acc;
    }
}

template <typename VT>
__global__ void k_spmv_Gt_dot_lowp(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   const VT* __restrict__ val, const float* __restrict__ t,
                                   const double* __restrict__ r, double* __restrict__ z, Scalars* s,
                                   double* partials, int init) {
    if (!init && s->done) return;
    double v[1] = {0.0};
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t b = rowptr[i], e = rowptr[i + 1];
        float acc = 0.0f;
        for (int32_t k = b; k < e; ++k) acc = fmaf(ld_f32(&val[k]), __ldg(&t[__ldg(&col[k])]), acc);
        const double zi = static_cast<double>(acc);
        z[i] = zi;
        v[0] = fma(r[i], zi, v[0]);
    }
    if (grid_sum<1>(v, partials, &s->ticket[4]) && threadIdx.x == 0) {
        if (init) {
            s->rz = v[0];
        } else {
            s->beta = v[0] / s->rz;
            s->rz = v[0];
        }
    }
}

// ---- p = z + beta p ---------------------------------------------------------
__global__ void k_update_p(int32_t n, const double* __restrict__ z, double* __restrict__ p, const Scalars* s) {
    if (s->done) return;
    const double beta = s->beta;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

// ---- identity preconditioner (M = NULL): z = r, rz' = r.r ------------------
__global__ void k_copy_dot(int32_t n, const double* __restrict__ r, double* __restrict__ z, Scalars* s,
                           double* partials, int init) {
    if (!init && s->done) return;
    double v[1] = {0.0};
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        z[i] = r[i];
        v[0] = fma(r[i], r[i], v[0]);
    }
    if (grid_sum<1>(v, partials, &s->ticket[4]) && threadIdx.x == 0) {
        if (init) {
            s->rz = v[0];
        } else {
            s->beta = v[0] / s->rz;
            s->rz = v[0];
        }
    }
}

// ---- true residual ||b - A x||^2 -----------------------------------------
__global__ void k_true_residual(int32_t n, const double* __restrict__ b, const double* __restrict__ q, Scalars* s,
                                double* partials, double* out) {
    double v[1] = {0.0};
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double d = b[i] - q[i];
        v[0] = fma(d, d, v[0]);
    }
    if (grid_sum<1>(v, partials, &s->ticket[5]) && threadIdx.x == 0) *out = v[0];
}

int group_for(int64_t n, int64_t nnz) {
    static int forced = [] {
        const char* e = std::getenv("AFSAI_SPMV_GROUP");
        return e ? std::atoi(e) : 0;
    }();
    if (forced == 1 || forced == 2 || forced == 4 || forced == 8) return forced;
    const double avg = n > 0 ? static_cast<double>(nnz) / n : 0.0;
    if (avg <= 16.0) return 1;
    if (avg <= 48.0) return 2;
    return 4;
}

int blocks_for(int64_t items) {
    const int64_t need = (items + kThreads - 1) / kThreads;
    const int64_t cap = static_cast<int64_t>(num_sms()) * (2048 / kThreads) * 2;
    return static_cast<int>(std::max<int64_t>(1, std::min(need, cap)));
}

struct Launcher {
    int32_t n;
    const CsrDev* A;
    const afsai_precond* M;
    double *x, *r, *p, *q, *z, *t;
    const double* b;
    Scalars* s;
    double* partials;
    cudaStream_t st;

    template <typename F>
    afsai_status by_group(int L, F f) {
        switch (L) {
            case 1: f(std::integral_constant<int, 1>{}); break;
            case 2: f(std::integral_constant<int, 2>{}); break;
            case 4: f(std::integral_constant<int, 4>{}); break;
            default: f(std::integral_constant<int, 8>{}); break;
        }
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        return AFSAI_OK;
    }

    // z = M r and rz (init: rz only; else beta too)
    afsai_status precond_dot(int init) {
        if (!M) {
            k_copy_dot<<<blocks_for(n), kThreads, 0, st>>>(n, r, z, s, partials, init);
            AFSAI_CUDA_TRY(cudaGetLastError());
            count_launches(1);
            return AFSAI_OK;
        }
        const CsrDev& G = M->G;
        const CsrDev& Gt = M->Gt;
        if (G.vtype == VAL_F64) {
            const int LG = group_for(G.n, G.nnz), LT = group_for(Gt.n, Gt.nnz);
            AFSAI_TRY(by_group(LG, [&](auto Lc) {
                constexpr int L = decltype(Lc)::value;
                k_spmv_G_f64<L><<<blocks_for(int64_t(n) * L), kThreads, 0, st>>>(
                    n, G.rowptr, G.col, static_cast<const double*>(G.val), r, t, s, init);
            }));
            return by_group(LT, [&](auto Lc) {
                constexpr int L = decltype(Lc)::value;
                k_spmv_Gt_dot_f64<L><<<blocks_for(int64_t(n) * L), kThreads, 0, st>>>(
                    n, Gt.rowptr, Gt.col, static_cast<const double*>(Gt.val), t, r, z, s, partials, init);
            });
        }
        float* tf = reinterpret_cast<float*>(t);
        if (G.vtype == VAL_F32) {
            k_spmv_G_lowp<float><<<blocks_for(n), kThreads, 0, st>>>(n, G.rowptr, G.col,
                                                                     static_cast<const float*>(G.val), r, tf, s, init);
            k_spmv_Gt_dot_lowp<float><<<blocks_for(n), kThreads, 0, st>>>(
                n, Gt.rowptr, Gt.col, static_cast<const float*>(Gt.val), tf, r, z, s, partials, init);
        } else {
            k_spmv_G_lowp<__nv_bfloat16><<<blocks_for(n), kThreads, 0, st>>>(
                n, G.rowptr, G.col, static_cast<const __nv_bfloat16*>(G.val), r, tf, s, init);
            k_spmv_Gt_dot_lowp<__nv_bfloat16><<<blocks_for(n), kThreads, 0, st>>>(
                n, Gt.rowptr, Gt.col, static_cast<const __nv_bfloat16*>(Gt.val), tf, r, z, s, partials, init);
        }
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(2);
        return AFSAI_OK;
    }

    afsai_status iteration() {
        const int LA = group_for(A->n, A->nnz);
        AFSAI_TRY(by_group(LA, [&](auto Lc) {
            constexpr int L = decltype(Lc)::value;
            k_spmv_A_dot<L><<<blocks_for(int64_t(n) * L), kThreads, 0, st>>>(
                n, A->rowptr, A->col, static_cast<const double*>(A->val), p, q, s, partials);
        }));
        k_update_xr<<<blocks_for(n), kThreads, 0, st>>>(n, x, r, p, q, s, partials);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        AFSAI_TRY(precond_dot(0));
        k_update_p<<<blocks_for(n), kThreads, 0, st>>>(n, z, p, s);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        return AFSAI_OK;
    }
};

int iters_per_graph() {
    static int v = [] {
        const char* e = std::getenv("AFSAI_PCG_GRAPH_ITERS");
        const int k = e ? std::atoi(e) : 0;
        return k > 0 ? k : 8;
    }();
    return v;
}

}  // namespace

namespace {

afsai_status pcg_body(const CsrDev& A, const afsai_precond* M, const double* b, double* x, double rtol,
                      int32_t maxit, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1, pcg_info* info) {
    const int32_t n = A.n;
    DevBuf<double> vec, partials, trueres;
    DevBuf<Scalars> sc;
    AFSAI_TRY(vec.alloc(static_cast<size_t>(n) * 5, st));
    AFSAI_TRY(partials.alloc(static_cast<size_t>(num_sms()) * 64, st));
    AFSAI_TRY(sc.alloc(1, st));
    AFSAI_TRY(trueres.alloc(1, st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(sc.p, 0, sizeof(Scalars), st));
    Scalars init_s{};
    init_s.maxit = maxit;
    AFSAI_CUDA_TRY(cudaMemcpyAsync(sc.p, &init_s, sizeof(Scalars), cudaMemcpyHostToDevice, st));
    Launcher L{};
    L.n = n;
    L.A = &A;
    L.M = M;
    L.x = x;
    L.b = b;
    L.r = vec.p;
    L.p = vec.p + n;
    L.q = vec.p + 2 * static_cast<size_t>(n);
    L.z = vec.p + 3 * static_cast<size_t>(n);
    L.t = vec.p + 4 * static_cast<size_t>(n);
    L.s = sc.p;
    L.partials = partials.p;
    L.st = st;

    AFSAI_CUDA_TRY(cudaEventRecord(ev0, st));
    // r = b - A x ; z = M r ; p = z
    AFSAI_TRY(spmv_csr(A, x, L.q, st));
    k_init_residual<<<blocks_for(n), kThreads, 0, st>>>(n, b, L.q, L.r, sc.p, partials.p, rtol);
    AFSAI_CUDA_TRY(cudaGetLastError());
    AFSAI_TRY(L.precond_dot(1));
    k_init_p<<<blocks_for(n), kThreads, 0, st>>>(n, L.r, L.z, L.p, sc.p, partials.p);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(2);

    // a CUDA graph of K iterations, relaunched until the flag is set
    const int K = iters_per_graph();
    cudaGraph_t graph = nullptr;
    AFSAI_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int64_t before_capture = launches_so_far();
    afsai_status cap = AFSAI_OK;
    for (int k = 0; k < K && cap == AFSAI_OK; ++k) cap = L.iteration();
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    const int64_t per_graph = launches_so_far() - before_capture;  // kernel nodes of one graph
    set_launches(before_capture);
    if (cap != AFSAI_OK) {
        if (graph) cudaGraphDestroy(graph);
        return cap;
    }
    AFSAI_CUDA_TRY(ce);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    AFSAI_CUDA_TRY(ie);
    int32_t* done_host = nullptr;
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&done_host), sizeof(int32_t));
    if (e == cudaSuccess) {
        *done_host = 0;
        const int64_t max_launches = maxit > 0 ? (static_cast<int64_t>(maxit) + K - 1) / K + 1 : 0;
        for (int64_t l = 0; l < max_launches && e == cudaSuccess; ++l) {
            e = cudaGraphLaunch(exec, st);
            if (e == cudaSuccess) count_launches(per_graph);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(done_host, &sc.p->done, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess && *done_host) break;
        }
        cudaFreeHost(done_host);
    }
    cudaGraphExecDestroy(exec);
    AFSAI_CUDA_TRY(e);
    AFSAI_CUDA_TRY(cudaEventRecord(ev1, st));
    // true residual
    AFSAI_TRY(spmv_csr(A, x, L.q, st));
    k_true_residual<<<blocks_for(n), kThreads, 0, st>>>(n, b, L.q, sc.p, partials.p, trueres.p);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    Scalars hs{};
    double tr2 = 0.0;
    AFSAI_CUDA_TRY(cudaMemcpyAsync(&hs, sc.p, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
    AFSAI_CUDA_TRY(cudaMemcpyAsync(&tr2, trueres.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    const double bn = std::sqrt(hs.bb);
    if (info) {
        info->iters = hs.iters;
        info->converged = (hs.done == 1 || (hs.done == 0 && hs.iters == 0)) ? 1 : 0;
        info->relres_rec = bn > 0 ? std::sqrt(hs.rr) / bn : 0.0;
        info->relres_true = bn > 0 ? std::sqrt(tr2) / bn : 0.0;
        info->solve_ms = ms;
    }
    if (hs.done == 2) return fail(AFSAI_ENOCONV, "PCG reached maxit without convergence");
    return AFSAI_OK;
}

}  // namespace

afsai_status pcg_impl(const afsai_csr* Ain, const afsai_precond* M, const double* b, double* x, double rtol,
                      int32_t maxit, cudaStream_t user_st, pcg_info* info) {
    const CsrDev A = view_of(Ain);
    // The iteration is captured into a CUDA graph, which needs a stream that
    // is not the legacy default stream: work runs on a private stream
    // ordered after the caller's stream and joined back at the end.
    cudaStream_t st;
    AFSAI_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaEvent_t join = nullptr, ev0 = nullptr, ev1 = nullptr;
    cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    afsai_status result = AFSAI_OK;
    if (!join || !ev0 || !ev1) {
        result = fail(AFSAI_ECUDA, "cudaEventCreate failed");
    } else {
        cudaEventRecord(join, user_st);
        cudaStreamWaitEvent(st, join, 0);
        result = pcg_body(A, M, b, x, rtol, maxit, st, ev0, ev1, info);
        cudaEventRecord(join, st);
        cudaStreamWaitEvent(user_st, join, 0);
    }
    cudaStreamSynchronize(st);
    if (join) cudaEventDestroy(join);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    cudaStreamDestroy(st);
    return result;
}

}  // namespace afsai
