// Preconditioned conjugate gradients with M^{-1} = G^T G (Eq. "prec"),
// stopping at ||r_k|| <= rtol ||b|| (Section 5.2: an 8-order reduction).
//
// Standard (Hestenes-Stiefel) PCG, one iteration =
//   q = A p,            pq = p.q,  alpha = rz / pq           [spmv A + dot]
//   x += alpha p, r -= alpha q,    rr = r.r, convergence test [update_xr]
//   t = G r                                                   [spmv G]
//   z = G^T t,          rz' = r.z, beta = rz' / rz            [spmv G^T + dot]
//   p = z + beta p                                            [update_p]
// The three SpMVs are the TMA-staged kernels of spmv_tiled.cuh with the
// dot product fused into their epilogue.  All scalars live in device
// memory.  Each reduction is deterministic: every block writes one partial,
// and the last block to finish (atomic ticket) sums the partials in a fixed
// order and derives alpha, beta or the convergence flag.  Once converged,
// every kernel returns at entry, so iterations are enqueued ahead in a CUDA
// graph of several iterations and the host only polls the flag between
// graph launches.
//
// Residual, dot products, alpha and beta are FP64 whatever the precision of
// G; with an FP32/BF16 G the two triangular products run in FP32.
//
// Stopping rule (Section 5.2, an 8-order reduction): the loop stops when
// the recursive residual meets ||r_k|| <= rtol ||b|| (the same comparison
// of square roots as the plain definition); the host then computes the
// true residual ||b - A x_k||; if that is above rtol ||b|| the recurrence
// continues one iteration at a time, with the true residual checked after
// each, until it meets the tolerance or maxit is reached.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <type_traits>

#include "afsai_internal.cuh"
#include "spmv_tiled.cuh"

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
    double tolr;  // rtol ||b||
    int32_t done;  // 0 running, 1 converged, 2 maxit reached, 3 device wait expired
    int32_t iters;
    int32_t maxit;
    int32_t err;   // set by a bounded wait that ran out
    unsigned ticket[8];
};

// Block sum of K values (fixed shuffle tree, then warp 0).  blockDim.x is
// a multiple of 32 and at most 1024.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double (*sh)[32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
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
            double w = lane < nwarps ? sh[k][lane] : 0.0;
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

__device__ __forceinline__ void abort_solve(Scalars* s) {
    if (threadIdx.x == 0) atomicExch(&s->done, 3);
}

// ---- init: r = b - q (q = A x), rr = r.r, bb = b.b ----------------------
__global__ void k_init_residual(int32_t n, const double* __restrict__ b, const double* __restrict__ q,
                                double* __restrict__ r, float* __restrict__ r32, Scalars* s, double* partials,
                                double rtol) {
    double v[2] = {0.0, 0.0};
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double ri = b[i] - q[i];
        r[i] = ri;
        if (r32) r32[i] = static_cast<float>(ri);
        v[0] = fma(ri, ri, v[0]);
        v[1] = fma(b[i], b[i], v[1]);
    }
    if (grid_sum<2>(v, partials, &s->ticket[0]) && threadIdx.x == 0) {
        s->rr = v[0];
        s->bb = v[1];
        s->tolr = rtol * sqrt(v[1]);
        s->iters = 0;
        s->done = (sqrt(v[0]) <= s->tolr) ? 1 : 0;
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

// Epilogues of the tiled SpMVs.
template <typename ACC, typename YT>
struct EpiStore {
    YT* y;
    __device__ void row(int64_t i, ACC a) { y[i] = static_cast<YT>(a); }
};
template <typename ACC>
struct EpiStoreDot {
    double* y;
    const double* w;
    double dot;
    __device__ void row(int64_t i, ACC a) {
        const double d = static_cast<double>(a);
        y[i] = d;
        dot = fma(w[i], d, dot);
    }
};

// ---- q = A p, pq = p.q, alpha = rz / pq ----------------------------------
template <int MODE>
__global__ void k_spmv_A_dot(int32_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                             const int32_t* __restrict__ col, const double* __restrict__ val,
                             const double* __restrict__ p, double* __restrict__ q, Scalars* s, double* partials,
                             int cap, tiled::SellView sv, long long wait) {
    if (s->done) return;
    EpiStoreDot<double> epi{q, p, 0.0};
    if (!tiled::spmv_rows<MODE, double, double, double>(n, nnz, rowptr, col, val, p, cap, &s->err, epi, sv, wait)) {
        abort_solve(s);
        return;
    }
    double v[1] = {epi.dot};
    if (grid_sum<1>(v, partials, &s->ticket[2]) && threadIdx.x == 0) s->alpha = s->rz / v[0];
}

// ---- x += alpha p, r -= alpha q, rr = r.r, convergence --------------------
// Pairs of elements per load (16-byte aligned vectors), several pairs per
// thread in flight; the per-thread dot partial runs over its elements in
// index order.
__global__ void k_update_xr(int32_t n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, float* __restrict__ r32, Scalars* s, double* partials) {
    if (s->done) return;
    const double alpha = s->alpha;
    double v[1] = {0.0};
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const bool aligned = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(r) |
                           reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q)) & 15u) == 0;
    if (aligned) {
        const int64_t n2 = n / 2;
        auto* x2 = reinterpret_cast<double2*>(x);
        auto* r2 = reinterpret_cast<double2*>(r);
        const auto* p2 = reinterpret_cast<const double2*>(p);
        const auto* q2 = reinterpret_cast<const double2*>(q);
#pragma unroll 4
        for (int64_t k = tid; k < n2; k += nth) {
            double2 xv = x2[k], rv = r2[k];
            const double2 pv = p2[k], qv = q2[k];
            xv.x = fma(alpha, pv.x, xv.x);
            xv.y = fma(alpha, pv.y, xv.y);
            rv.x = fma(-alpha, qv.x, rv.x);
            rv.y = fma(-alpha, qv.y, rv.y);
            x2[k] = xv;
            r2[k] = rv;
            if (r32)
                reinterpret_cast<float2*>(r32)[k] = make_float2(static_cast<float>(rv.x), static_cast<float>(rv.y));
            v[0] = fma(rv.x, rv.x, v[0]);
            v[0] = fma(rv.y, rv.y, v[0]);
        }
        if ((n & 1) && tid == 0) {
            const int64_t i = n - 1;
            x[i] = fma(alpha, p[i], x[i]);
            const double ri = fma(-alpha, q[i], r[i]);
            r[i] = ri;
            if (r32) r32[i] = static_cast<float>(ri);
            v[0] = fma(ri, ri, v[0]);
        }
    } else {
        for (int64_t i = tid; i < n; i += nth) {
            x[i] = fma(alpha, p[i], x[i]);
            const double ri = fma(-alpha, q[i], r[i]);
            r[i] = ri;
            if (r32) r32[i] = static_cast<float>(ri);
            v[0] = fma(ri, ri, v[0]);
        }
    }
    if (grid_sum<1>(v, partials, &s->ticket[3]) && threadIdx.x == 0) {
        s->rr = v[0];
        s->iters += 1;
        if (sqrt(v[0]) <= s->tolr)
            s->done = 1;
        else if (s->iters >= s->maxit)
            s->done = 2;
    }
}

// ---- t = G r (ACC: double for an FP64 G, float otherwise; r in ACC too:
// with FP32 accumulation the solve keeps an FP32 copy of r, rounded once
// per element where the residual is written, instead of rounding each
// gathered double in the product: a double-to-float conversion runs on
// the FP64 pipe, and one per entry of G kept that pipe 85% busy) ----------
template <int MODE, typename VT, typename ACC>
__global__ void k_spmv_G(int32_t n, int64_t nnz, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                         const VT* __restrict__ val, const ACC* __restrict__ r, ACC* __restrict__ t, Scalars* s,
                         int cap, int init, tiled::SellView sv, long long wait) {
    if (!init && s->done) return;
    EpiStore<ACC, ACC> epi{t};
    if (!tiled::spmv_rows<MODE, VT, ACC, ACC>(n, nnz, rowptr, col, val, r, cap, &s->err, epi, sv, wait))
        abort_solve(s);
}

// ---- z = G^T t, rz' = r.z, beta -------------------------------------------
template <int MODE, typename VT, typename ACC>
__global__ void k_spmv_Gt_dot(int32_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                              const int32_t* __restrict__ col, const VT* __restrict__ val, const ACC* __restrict__ t,
                              const double* __restrict__ r, double* __restrict__ z, Scalars* s, double* partials,
                              int cap, int init, tiled::SellView sv, long long wait) {
    if (!init && s->done) return;
    EpiStoreDot<ACC> epi{z, r, 0.0};
    if (!tiled::spmv_rows<MODE, VT, ACC, ACC>(n, nnz, rowptr, col, val, t, cap, &s->err, epi, sv, wait)) {
        abort_solve(s);
        return;
    }
    double v[1] = {epi.dot};
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
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = static_cast<int64_t>(gridDim.x) * blockDim.x;
    if (((reinterpret_cast<uintptr_t>(z) | reinterpret_cast<uintptr_t>(p)) & 15u) == 0) {
        const int64_t n2 = n / 2;
        auto* p2 = reinterpret_cast<double2*>(p);
        const auto* z2 = reinterpret_cast<const double2*>(z);
#pragma unroll 4
        for (int64_t k = tid; k < n2; k += nth) {
            double2 pv = p2[k];
            const double2 zv = z2[k];
            pv.x = fma(beta, pv.x, zv.x);
            pv.y = fma(beta, pv.y, zv.y);
            p2[k] = pv;
        }
        if ((n & 1) && tid == 0) p[n - 1] = fma(beta, p[n - 1], z[n - 1]);
    } else {
        for (int64_t i = tid; i < n; i += nth) p[i] = fma(beta, p[i], z[i]);
    }
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

// Vector kernels: a small persistent grid, so that each thread sums many
// elements before the (FP64) block reduction.
int vec_blocks(int64_t n) {
    const int64_t need = (n + kThreads - 1) / kThreads;
    const int64_t cap = static_cast<int64_t>(num_sms()) * 2;
    return static_cast<int>(std::max<int64_t>(1, std::min(need, cap)));
}

// Shared-memory limit of a product kernel, and its grid trimmed to one
// resident wave of that kernel.
template <typename K>
void fit(K kern, SpmvMode& m) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    m.blocks = resident_grid(kern, m.blocks, m.threads, m.smem);
}

// Calls f(std::integral_constant<int, MODE>) for the engine mode.
template <typename F>
bool with_mode(int mode, F f) {
    switch (mode) {
        case 1: f(std::integral_constant<int, 1>{}); return true;
        case 2: f(std::integral_constant<int, 2>{}); return true;
        case 4: f(std::integral_constant<int, 4>{}); return true;
        case 8: f(std::integral_constant<int, 8>{}); return true;
        case 3: f(std::integral_constant<int, 3>{}); return true;
        case 6: f(std::integral_constant<int, 6>{}); return true;
        case 101: f(std::integral_constant<int, 101>{}); return true;
        case 102: f(std::integral_constant<int, 102>{}); return true;
        case 103: f(std::integral_constant<int, 103>{}); return true;
        case 104: f(std::integral_constant<int, 104>{}); return true;
        case tiled::kModeSliced: f(std::integral_constant<int, tiled::kModeSliced>{}); return true;
        case tiled::kModeSlicedPipe: f(std::integral_constant<int, tiled::kModeSlicedPipe>{}); return true;
        case tiled::kModeSlicedPipe8: f(std::integral_constant<int, tiled::kModeSlicedPipe8>{}); return true;
        case tiled::kModeSlicedPipeIlv: f(std::integral_constant<int, tiled::kModeSlicedPipeIlv>{}); return true;
        case tiled::kModeSlicedStaged8: f(std::integral_constant<int, tiled::kModeSlicedStaged8>{}); return true;
        case tiled::kModeSlicedStaged16: f(std::integral_constant<int, tiled::kModeSlicedStaged16>{}); return true;
        case tiled::kModeBalanced: f(std::integral_constant<int, tiled::kModeBalanced>{}); return true;
        default: return false;
    }
}

// Accumulation of the G and G^T products of an FP32/BF16 G: FP32
// (default) or FP64 (AFSAI_G_ACC64=1).
bool acc64() {
    static const bool v = [] {
        const char* e = std::getenv("AFSAI_G_ACC64");
        return e && std::atoi(e) != 0;
    }();
    return v;
}

struct Launcher {
    int32_t n;
    const CsrDev* A;
    const afsai_precond* M;
    double *x, *r, *p, *q, *z, *t;
    float* r32 = nullptr;  // FP32 copy of r for an FP32-accumulated G product (in t's slot)
    const double* b;
    Scalars* s;
    double* partials;
    cudaStream_t st;
    SpmvMode ma, mg, mt;
    long long wait;  // cycles a tile's copies may take before the solve gives up
    // timestamps between the kernels of one iteration (6 events, recorded as
    // event nodes of the captured graph), or nullptr
    cudaEvent_t* marks = nullptr;
    void mark(int k) {
        if (marks) cudaEventRecordWithFlags(marks[k], st, cudaEventRecordExternal);
    }

    // fused product kernels launched with engine m0 for the engine timing
    // (on scratch scalars ts; y = C x; x_float: t is FP32)
    afsai_status tune_A(const SpmvMode& m0, const void* x, void* y, cudaStream_t s2, Scalars* ts) {
        SpmvMode m = m0;
        const auto* v = static_cast<const double*>(A->val);
        if (!with_mode(m.mode, [&](auto Mc) {
                constexpr int MD = decltype(Mc)::value;
                fit(k_spmv_A_dot<MD>, m);
                k_spmv_A_dot<MD><<<m.blocks, m.threads, m.smem, s2>>>(
                    A->n, A->nnz, A->rowptr, A->col, v, static_cast<const double*>(x), static_cast<double*>(y), ts,
                    partials, m.cap, tiled::sell_view(A->sell), tiled::kWaitCycles);
            }))
            return fail(AFSAI_EINVAL, "unknown SpMV mode");
        AFSAI_CUDA_TRY(cudaGetLastError());
        return AFSAI_OK;
    }
    template <typename VT, typename ACC>
    afsai_status tune_G(const SpmvMode& m0, const void* x, void* y, cudaStream_t s2, Scalars* ts) {
        SpmvMode m = m0;
        const CsrDev& G = M->G;
        if (!with_mode(m.mode, [&](auto Mc) {
                constexpr int MD = decltype(Mc)::value;
                fit(k_spmv_G<MD, VT, ACC>, m);
                k_spmv_G<MD, VT, ACC><<<m.blocks, m.threads, m.smem, s2>>>(
                    G.n, G.nnz, G.rowptr, G.col, static_cast<const VT*>(G.val), static_cast<const ACC*>(x),
                    static_cast<ACC*>(y), ts, m.cap, 1, tiled::sell_view(G.sell), tiled::kWaitCycles);
            }))
            return fail(AFSAI_EINVAL, "unknown SpMV mode");
        AFSAI_CUDA_TRY(cudaGetLastError());
        return AFSAI_OK;
    }
    template <typename VT, typename ACC>
    afsai_status tune_Gt(const SpmvMode& m0, const void* x, void* y, cudaStream_t s2, Scalars* ts) {
        SpmvMode m = m0;
        const CsrDev& Gt = M->Gt;
        if (!with_mode(m.mode, [&](auto Mc) {
                constexpr int MD = decltype(Mc)::value;
                fit(k_spmv_Gt_dot<MD, VT, ACC>, m);
                k_spmv_Gt_dot<MD, VT, ACC><<<m.blocks, m.threads, m.smem, s2>>>(
                    Gt.n, Gt.nnz, Gt.rowptr, Gt.col, static_cast<const VT*>(Gt.val), static_cast<const ACC*>(x), r,
                    static_cast<double*>(y), ts, partials, m.cap, 1, tiled::sell_view(Gt.sell), tiled::kWaitCycles);
            }))
            return fail(AFSAI_EINVAL, "unknown SpMV mode");
        AFSAI_CUDA_TRY(cudaGetLastError());
        return AFSAI_OK;
    }
    template <typename VT, typename ACC>
    afsai_status plan_G(Scalars* ts) {
        RoleLaunch lg, lt;
        lg.x_float = sizeof(ACC) == sizeof(float);
        lg.launch = [&](const SpmvMode& m, const void* x, void* y, cudaStream_t s2) {
            return tune_G<VT, ACC>(m, x, y, s2, ts);
        };
        lt.x_float = sizeof(ACC) == sizeof(float);
        lt.launch = [&](const SpmvMode& m, const void* x, void* y, cudaStream_t s2) {
            return tune_Gt<VT, ACC>(m, x, y, s2, ts);
        };
        AFSAI_TRY(spmv_mode_for(ROLE_G, M->G, st, &mg, true, &lg));
        return spmv_mode_for(ROLE_GT, M->Gt, st, &mt, true, &lt);
    }

    // engine choice (timed on the fused kernels of the solve) and
    // shared-memory limits, before any stream capture
    afsai_status plan() {
        DevBuf<Scalars> ts;
        AFSAI_TRY(ts.alloc(1, st));
        AFSAI_CUDA_TRY(cudaMemsetAsync(ts.p, 0, sizeof(Scalars), st));
        // r (set by the solve's first kernel) serves the timed dot products
        fill_tune_vector(r, n, false, st);
        RoleLaunch la;
        la.launch = [&](const SpmvMode& m, const void* x, void* y, cudaStream_t s2) {
            return tune_A(m, x, y, s2, ts.p);
        };
        AFSAI_TRY(spmv_mode_for(ROLE_A, *A, st, &ma, true, &la));
        if (M) {
            const int vt = M->G.vtype;
            if (vt == VAL_F64)
                AFSAI_TRY((plan_G<double, double>(ts.p)));
            else if (vt == VAL_F32)
                AFSAI_TRY((acc64() ? plan_G<float, double>(ts.p) : plan_G<float, float>(ts.p)));
            else
                AFSAI_TRY((acc64() ? plan_G<__nv_bfloat16, double>(ts.p)
                                   : plan_G<__nv_bfloat16, float>(ts.p)));
        }
        with_mode(ma.mode, [&](auto Mc) { fit(k_spmv_A_dot<decltype(Mc)::value>, ma); });
        if (M) {
            const int vt = M->G.vtype;
            const bool a64 = acc64();
            with_mode(mg.mode, [&](auto Mc) {
                constexpr int MD = decltype(Mc)::value;
                if (vt == VAL_F64)
                    fit(k_spmv_G<MD, double, double>, mg);
                else if (vt == VAL_F32)
                    a64 ? fit(k_spmv_G<MD, float, double>, mg) : fit(k_spmv_G<MD, float, float>, mg);
                else
                    a64 ? fit(k_spmv_G<MD, __nv_bfloat16, double>, mg) : fit(k_spmv_G<MD, __nv_bfloat16, float>, mg);
            });
            with_mode(mt.mode, [&](auto Mc) {
                constexpr int MD = decltype(Mc)::value;
                if (vt == VAL_F64)
                    fit(k_spmv_Gt_dot<MD, double, double>, mt);
                else if (vt == VAL_F32)
                    a64 ? fit(k_spmv_Gt_dot<MD, float, double>, mt) : fit(k_spmv_Gt_dot<MD, float, float>, mt);
                else
                    a64 ? fit(k_spmv_Gt_dot<MD, __nv_bfloat16, double>, mt)
                        : fit(k_spmv_Gt_dot<MD, __nv_bfloat16, float>, mt);
            });
        }
        return AFSAI_OK;
    }

    afsai_status spmv_A_dot() {
        mark(0);
        const auto* v = static_cast<const double*>(A->val);
        with_mode(ma.mode, [&](auto Mc) {
            k_spmv_A_dot<decltype(Mc)::value><<<ma.blocks, ma.threads, ma.smem, st>>>(
                A->n, A->nnz, A->rowptr, A->col, v, p, q, s, partials, ma.cap, tiled::sell_view(A->sell), wait);
        });
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        return AFSAI_OK;
    }

    template <typename VT, typename ACC>
    void launch_G_pair(const CsrDev& G, const CsrDev& Gt, int init) {
        ACC* tt = reinterpret_cast<ACC*>(t);
        const ACC* rin;
        if constexpr (sizeof(ACC) == sizeof(float))
            rin = r32;
        else
            rin = r;
        with_mode(mg.mode, [&](auto Mc) {
            k_spmv_G<decltype(Mc)::value, VT, ACC><<<mg.blocks, mg.threads, mg.smem, st>>>(
                G.n, G.nnz, G.rowptr, G.col, static_cast<const VT*>(G.val), rin, tt, s, mg.cap, init,
                tiled::sell_view(G.sell), wait);
        });
        mark(3);
        with_mode(mt.mode, [&](auto Mc) {
            k_spmv_Gt_dot<decltype(Mc)::value, VT, ACC><<<mt.blocks, mt.threads, mt.smem, st>>>(
                Gt.n, Gt.nnz, Gt.rowptr, Gt.col, static_cast<const VT*>(Gt.val), tt, r, z, s, partials, mt.cap, init,
                tiled::sell_view(Gt.sell), wait);
        });
    }

    // z = M r and rz (init: rz only; else beta too)
    afsai_status precond_dot(int init) {
        if (!M) {
            k_copy_dot<<<vec_blocks(n), kThreads, 0, st>>>(n, r, z, s, partials, init);
            AFSAI_CUDA_TRY(cudaGetLastError());
            count_launches(1);
            return AFSAI_OK;
        }
        const CsrDev& G = M->G;
        const CsrDev& Gt = M->Gt;
        if (G.vtype == VAL_F64)
            launch_G_pair<double, double>(G, Gt, init);
        else if (G.vtype == VAL_F32)
            acc64() ? launch_G_pair<float, double>(G, Gt, init) : launch_G_pair<float, float>(G, Gt, init);
        else
            acc64() ? launch_G_pair<__nv_bfloat16, double>(G, Gt, init)
                    : launch_G_pair<__nv_bfloat16, float>(G, Gt, init);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(2);
        return AFSAI_OK;
    }

    // first half of an iteration: q = A p, alpha, x and r, the recursive test
    afsai_status head() {
        AFSAI_TRY(spmv_A_dot());
        mark(1);
        k_update_xr<<<vec_blocks(n), kThreads, 0, st>>>(n, x, r, p, q, r32, s, partials);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        mark(2);
        return AFSAI_OK;
    }
    // second half: z = M r, beta, p
    afsai_status tail() {
        AFSAI_TRY(precond_dot(0));
        mark(4);
        k_update_p<<<vec_blocks(n), kThreads, 0, st>>>(n, z, p, s);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        mark(5);
        return AFSAI_OK;
    }
    afsai_status iteration() {
        AFSAI_TRY(head());
        return tail();
    }
};

// Cycle limit of the first wait for a tile's bulk copies in the staged SpMV
// engines of the PCG (AFSAI_WAIT_CYCLES, default ~2 s at 2 GHz; 0: a single
// check without waiting); a wait that runs out ends the solve with
// AFSAI_ETIMEOUT.  The wait that lets a block's copies in flight land after
// an expiry keeps the full bound.
long long first_wait_cycles() {
    static const long long v = [] {
        const char* e = std::getenv("AFSAI_WAIT_CYCLES");
        if (!e || !*e) return tiled::kWaitCycles;
        const long long k = std::atoll(e);
        return k >= 0 ? k : tiled::kWaitCycles;
    }();
    return v;
}

int iters_per_graph() {
    static int v = [] {
        const char* e = std::getenv("AFSAI_PCG_GRAPH_ITERS");
        const int k = e ? std::atoi(e) : 0;
        return k > 0 ? k : 8;
    }();
    return v;
}

// A sliced copy of A for one solve, freed when the solve ends.
struct SlicedA {
    CsrDev view;
    cudaStream_t st;
    ~SlicedA() { free_sell(&view.sell, st); }
};

afsai_status pcg_body(const CsrDev& Ain, const afsai_precond* M, const double* b, double* x, double rtol,
                      int32_t maxit, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1, pcg_info* info) {
    const int32_t n = Ain.n;
    // The matrix may change between solves, so its sliced copy is rebuilt
    // for each solve (one pass over A) unless a CSR engine was chosen for
    // this shape.  Without room for the copy the CSR engines serve.
    SlicedA sa{Ain, st};
    if (spmv_wants_sliced(ROLE_A, Ain)) {
        const std::string keep = afsai_last_error();
        if (build_sell(Ain, &sa.view.sell, st, spmv_wants_order(ROLE_A, Ain)) != AFSAI_OK) {
            cudaGetLastError();  // a failed allocation is not an error of the solve
            set_error(keep);
        }
    }
    const CsrDev& A = sa.view;
    DevBuf<double> vec, partials, trueres;
    DevBuf<Scalars> sc;
    const size_t vs = (static_cast<size_t>(n) + 31) / 32 * 32;  // 256-byte aligned vector stride
    AFSAI_TRY(vec.alloc(vs * 5, st));
    AFSAI_TRY(partials.alloc(static_cast<size_t>(num_sms()) * 64, st));
    AFSAI_TRY(sc.alloc(1, st));
    AFSAI_TRY(trueres.alloc(1, st));
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
    L.p = vec.p + vs;
    L.q = vec.p + 2 * vs;
    L.z = vec.p + 3 * vs;
    L.t = vec.p + 4 * vs;
    // t's slot holds vs doubles; with an FP32-accumulated G product t uses
    // its first n floats and the FP32 copy of r starts at float vs
    if (M && M->G.vtype != VAL_F64 && !acc64()) L.r32 = reinterpret_cast<float*>(L.t) + vs;
    L.s = sc.p;
    L.partials = partials.p;
    L.st = st;
    L.wait = first_wait_cycles();
    AFSAI_TRY(L.plan());
    // partials hold one value per block of the largest grid (2 per block for K = 2)
    if (std::max({L.ma.blocks, L.mg.blocks, L.mt.blocks, vec_blocks(n)}) * 2 > num_sms() * 64)
        return fail(AFSAI_ENOTSUP, "reduction grid larger than the partials buffer");

    AFSAI_CUDA_TRY(cudaEventRecord(ev0, st));
    // r = b - A x ; z = M r ; p = z
    AFSAI_TRY(spmv_csr(A, x, L.q, st));
    k_init_residual<<<vec_blocks(n), kThreads, 0, st>>>(n, b, L.q, L.r, L.r32, sc.p, partials.p, rtol);
    AFSAI_CUDA_TRY(cudaGetLastError());
    AFSAI_TRY(L.precond_dot(1));
    k_init_p<<<vec_blocks(n), kThreads, 0, st>>>(n, L.r, L.z, L.p, sc.p, partials.p);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(2);

    // a CUDA graph of K iterations, relaunched until the flag is set
    const int K = iters_per_graph();
    cudaGraph_t graph = nullptr;
    AFSAI_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int64_t before_capture = launches_so_far();
    afsai_status cap = AFSAI_OK;
    // the kernels of the graph's first iteration are timed (event nodes)
    cudaEvent_t marks[6] = {};
    bool have_marks = info != nullptr && M != nullptr;
    for (int k = 0; k < 6 && have_marks; ++k)
        if (cudaEventCreate(&marks[k]) != cudaSuccess) have_marks = false;
    if (!have_marks) cudaGetLastError();
    for (int k = 0; k < K && cap == AFSAI_OK; ++k) {
        L.marks = (k == 0 && have_marks) ? marks : nullptr;
        cap = L.iteration();
    }
    L.marks = nullptr;
    struct MarkGuard {
        cudaEvent_t* m;
        ~MarkGuard() {
            for (int k = 0; k < 6; ++k)
                if (m[k]) cudaEventDestroy(m[k]);
        }
    } mark_guard{marks};
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
    double kernel_ms[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    Scalars* hs_pinned = nullptr;
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&hs_pinned), sizeof(Scalars));
    bool true_ok = false;
    double tr2 = 0.0;
    if (e == cudaSuccess) {
        // the scalars after the initial residual (done = 1: x0 already meets the tolerance)
        e = cudaMemcpyAsync(hs_pinned, sc.p, sizeof(Scalars), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        const int64_t max_launches = maxit > 0 ? (static_cast<int64_t>(maxit) + K - 1) / K + 1 : 0;
        // graph launches until the recursive test (or maxit, or a wait) ends the loop
        for (int64_t l = 0; l < max_launches && e == cudaSuccess && hs_pinned->done == 0; ++l) {
            e = cudaGraphLaunch(exec, st);
            if (e == cudaSuccess) count_launches(per_graph);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hs_pinned, sc.p, sizeof(Scalars), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess && l == 0 && have_marks)
                for (int k = 0; k < 5; ++k) {
                    float km = 0.f;
                    if (cudaEventElapsedTime(&km, marks[k], marks[k + 1]) == cudaSuccess) kernel_ms[k] = km;
                }
            if (e == cudaSuccess && hs_pinned->done) break;
        }
        // the recursive residual met the tolerance: check the true one, and
        // continue the recurrence one iteration at a time while it is above
        while (e == cudaSuccess && hs_pinned->done == 1) {
            afsai_status ts = spmv_csr(A, x, L.q, st);
            if (ts == AFSAI_OK) {
                k_true_residual<<<vec_blocks(n), kThreads, 0, st>>>(n, b, L.q, sc.p, partials.p, trueres.p);
                count_launches(1);
                e = cudaMemcpyAsync(&tr2, trueres.p, sizeof(double), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            } else {
                e = cudaErrorUnknown;
            }
            if (e != cudaSuccess) break;
            if (std::sqrt(tr2) <= hs_pinned->tolr) {
                true_ok = true;
                break;
            }
            if (hs_pinned->iters >= maxit) {
                hs_pinned->done = 2;
                break;
            }
            const int32_t zero = 0;
            e = cudaMemcpyAsync(&sc.p->done, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) break;
            if (L.tail() != AFSAI_OK || L.head() != AFSAI_OK) {
                e = cudaErrorUnknown;
                break;
            }
            e = cudaMemcpyAsync(hs_pinned, sc.p, sizeof(Scalars), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            // a recursive residual above the tolerance again: back to the graph
            if (e == cudaSuccess && hs_pinned->done == 0) {
                for (int64_t l = 0; l < max_launches && e == cudaSuccess; ++l) {
                    e = cudaGraphLaunch(exec, st);
                    if (e == cudaSuccess) count_launches(per_graph);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(hs_pinned, sc.p, sizeof(Scalars), cudaMemcpyDeviceToHost, st);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                    if (e == cudaSuccess && hs_pinned->done) break;
                }
            }
        }
    }
    Scalars hs{};
    if (hs_pinned) {
        hs = *hs_pinned;
        cudaFreeHost(hs_pinned);
    }
    cudaGraphExecDestroy(exec);
    AFSAI_CUDA_TRY(e);
    AFSAI_CUDA_TRY(cudaEventRecord(ev1, st));
    if (!true_ok) {
        // true residual at exit (maxit, an expired wait, or no iterations)
        AFSAI_TRY(spmv_csr(A, x, L.q, st));
        k_true_residual<<<vec_blocks(n), kThreads, 0, st>>>(n, b, L.q, sc.p, partials.p, trueres.p);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        AFSAI_CUDA_TRY(cudaMemcpyAsync(&tr2, trueres.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    const double bn = std::sqrt(hs.bb);
    const bool converged = true_ok || (hs.done == 1 && std::sqrt(tr2) <= hs.tolr);
    if (info) {
        info->iters = hs.iters;
        info->converged = converged ? 1 : 0;
        info->relres_rec = bn > 0 ? std::sqrt(hs.rr) / bn : 0.0;
        info->relres_true = bn > 0 ? std::sqrt(tr2) / bn : 0.0;
        info->solve_ms = ms;
        for (int k = 0; k < 5; ++k) info->kernel_ms[k] = kernel_ms[k];
    }
    if (hs.done == 3 || hs.err) return fail(AFSAI_ETIMEOUT, "a bounded device wait ran out during PCG");
    if (!converged) return fail(AFSAI_ENOCONV, "PCG reached maxit without convergence");
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
