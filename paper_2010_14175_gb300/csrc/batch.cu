// Batched aFSAI-PCG: many independent SPD systems of uneven size solved
// with one set-up pass per bucket of systems and one graph launch of PCG.
//
// Set-up.  The systems are grouped by the longest row of their matrix
// (small stencils: the lane-per-row path; longer rows: the warp-per-row
// path); each bucket's CSRs are packed into one block-diagonal matrix and
// set up in one pass over all its rows, with a solve tile chosen per
// bucket by timing a sample.  Rows are independent and a row only sees
// columns of its own block, so each system's G is exactly the G of that
// system alone.  G and G^T stay packed; their column indices are made
// local to each system afterwards.
//
// PCG.  Every system keeps its own vectors and scalars (rz, alpha, beta,
// rr, convergence).  Work is cut into chunks of up to kChunk rows of one
// system; a block handles one chunk at a time, one thread per row.  The SpMV
// of a row is the plain sequential sum in CSR order, and every per-system
// dot product is reduced over the system's own chunks in a fixed order
// (fixed tree inside a chunk, chunks in table order), so the result of a
// system does not depend on which other systems share the batch.  The
// iteration kernels visit the chunks of running systems only (a list built
// again after every body in which a system finished).  The whole loop is
// one launch of a graph with a device-side while loop that ends when no
// system runs or a body budget is spent.
//
// The descriptor and chunk tables live in device memory with a fixed
// capacity and their counts are read on the device, so a captured graph
// stays valid when the tables are rewritten between launches (the solve
// server relies on this).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>
#include <tuple>
#include <mutex>
#include <map>

#include "afsai_batch.cuh"

namespace afsai {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Sum over the block of one value per thread (fixed tree); result in
// thread 0.  blockDim.x == kChunk.
__device__ __forceinline__ double chunk_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (kChunk >> 5) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    }
    __syncthreads();
    return t;
}

// Records the chunk partial; returns true in the block that completes the
// system's last chunk, which then holds the system total in `total`
// (thread 0): the chunk partials of the system summed in chunk order.
__device__ bool system_sum(double part, const BSys& sy, int32_t c, double* partials, unsigned* ticket,
                           double* total) {
    __shared__ bool last;
    __shared__ double sh[32];
    if (threadIdx.x == 0) {
        partials[c] = part;
        __threadfence();
        last = atomicAdd(ticket, 1u) == static_cast<unsigned>(sy.nchunks - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc = 0.0;
    for (int32_t k = threadIdx.x; k < sy.nchunks; k += blockDim.x)
        acc += reinterpret_cast<volatile double*>(partials)[sy.chunk0 + k];
    const double t = chunk_sum(acc, sh);
    if (threadIdx.x == 0) {
        *total = t;
        *ticket = 0u;
    }
    return true;
}

template <typename VT>
__device__ __forceinline__ float vf(VT v) {
    return static_cast<float>(v);
}
template <>
__device__ __forceinline__ float vf<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

// Row i of a CSR times x, sequential in CSR order (FP64).
__device__ __forceinline__ double row_f64(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                          const double* __restrict__ val, const double* __restrict__ x, int32_t i) {
    double acc = 0.0;
    const int32_t e = rp[i + 1];
    for (int32_t k = rp[i]; k < e; ++k) acc = fma(__ldg(&val[k]), __ldg(&x[__ldg(&col[k])]), acc);
    return acc;
}

// ---- init: r = b - A x, bb, rr ------------------------------------------
// r32: the G product accumulates in FP32 and reads an FP32 copy of r, kept
// in the second half of the system's t slot (n doubles; t itself takes the
// first n floats): rounded once per element here instead of once per entry
// of G in the product (a double-to-float conversion runs on the FP64 pipe).
__device__ __forceinline__ float* r32_of(const BSys& sy) { return static_cast<float*>(sy.t) + sy.n; }

__global__ void kb_init(const BSys* __restrict__ sys, BScal* sc, const BChunk* __restrict__ chunks,
                        ChunkList L, double* partials, double* partials2, int r32) {
    __shared__ double sh[32];
    for (int32_t k = blockIdx.x; k < *L.count; k += gridDim.x) {
        const int32_t c = L.act ? L.act[k] : k;
        const BChunk ch = chunks[c];
        BScal* s = &sc[ch.sys];
        if (!s->fresh) continue;
        const BSys& sy = sys[ch.sys];
        const int32_t i = ch.row0 + threadIdx.x;
        double rr = 0.0, bb = 0.0;
        if (i < ch.row1) {
            const double ri = sy.b[i] - row_f64(sy.Arp, sy.Acol, sy.Aval, sy.x, i);
            sy.r[i] = ri;
            if (r32) r32_of(sy)[i] = static_cast<float>(ri);
            rr = ri * ri;
            bb = sy.b[i] * sy.b[i];
        }
        const double trr = chunk_sum(rr, sh);
        const double tbb = chunk_sum(bb, sh);
        if (threadIdx.x == 0) partials2[c] = tbb;
        double tot;
        if (system_sum(trr, sy, c, partials, &s->ticket[0], &tot) && threadIdx.x == 0) {
            double b2 = 0.0;
            for (int32_t k = 0; k < sy.nchunks; ++k) b2 += reinterpret_cast<volatile double*>(partials2)[sy.chunk0 + k];
            s->rr = tot;
            s->bb = b2;
            s->tolr = s->rtol * sqrt(b2);
            s->iters = 0;
            if (sqrt(tot) <= s->tolr) {  // r = b - A x0 is the true residual here
                s->done = 1;
                atomicSub(s->active, 1);
                atomicAdd(s->active + 3, 1);
            }
        }
        __syncthreads();
    }
}

// ---- t = G r --------------------------------------------------------------
template <typename VT, typename TT>
__device__ __forceinline__ TT row_G(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const VT* __restrict__ val, const TT* __restrict__ x, int32_t i) {
    if constexpr (sizeof(TT) == 8) {
        double acc = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
            acc = fma(static_cast<double>(__ldg(&val[k])), __ldg(&x[__ldg(&col[k])]), acc);
        return acc;
    } else {
        float acc = 0.0f;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) acc = fmaf(vf<VT>(val[k]), __ldg(&x[__ldg(&col[k])]), acc);
        return acc;
    }
}

template <typename VT, typename TT>
__device__ __forceinline__ TT row_Gt(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                     const VT* __restrict__ val, const TT* __restrict__ t, int32_t i) {
    TT acc = TT(0);
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        if constexpr (sizeof(TT) == 8)
            acc = fma(static_cast<double>(__ldg(&val[k])), __ldg(&t[__ldg(&col[k])]), acc);
        else
            acc = fmaf(vf<VT>(val[k]), __ldg(&t[__ldg(&col[k])]), acc);
    }
    return acc;
}

template <typename VT, typename TT>
__global__ void kb_G(const BSys* __restrict__ sys, const BScal* sc, const BChunk* __restrict__ chunks,
                     ChunkList L, int init) {
    for (int32_t k = blockIdx.x; k < *L.count; k += gridDim.x) {
        const int32_t c = L.act ? L.act[k] : k;
        const BChunk ch = chunks[c];
        if (init ? !sc[ch.sys].fresh : (sc[ch.sys].done != 0)) continue;
        const BSys& sy = sys[ch.sys];
        const int32_t i = ch.row0 + threadIdx.x;
        if (i < ch.row1) {
            const TT* rin;
            if constexpr (sizeof(TT) == sizeof(float))
                rin = r32_of(sy);
            else
                rin = sy.r;
            static_cast<TT*>(sy.t)[i] = row_G<VT, TT>(sy.Grp, sy.Gcol, static_cast<const VT*>(sy.Gval), rin, i);
        }
    }
}

// ---- z = G^T t, rz' = r.z, beta -------------------------------------------
template <typename VT, typename TT>
__global__ void kb_Gt_dot(const BSys* __restrict__ sys, BScal* sc, const BChunk* __restrict__ chunks,
                          ChunkList L, double* partials, int init) {
    __shared__ double sh[32];
    for (int32_t k = blockIdx.x; k < *L.count; k += gridDim.x) {
        const int32_t c = L.act ? L.act[k] : k;
        const BChunk ch = chunks[c];
        BScal* s = &sc[ch.sys];
        if (init ? !s->fresh : (s->done != 0)) continue;
        const BSys& sy = sys[ch.sys];
        const int32_t i = ch.row0 + threadIdx.x;
        double part = 0.0;
        if (i < ch.row1) {
            const double zi = static_cast<double>(
                row_Gt<VT, TT>(sy.Trp, sy.Tcol, static_cast<const VT*>(sy.Tval), static_cast<const TT*>(sy.t), i));
            sy.z[i] = zi;
            part = sy.r[i] * zi;
        }
        const double tp = chunk_sum(part, sh);
        double tot;
        if (system_sum(tp, sy, c, partials, &s->ticket[1], &tot) && threadIdx.x == 0) {
            if (init) {
                s->rz = tot;
            } else {
                s->beta = tot / s->rz;
                s->rz = tot;
            }
        }
        __syncthreads();
    }
}

// ---- p = z (init) ---------------------------------------------------------
__global__ void kb_init_p(const BSys* __restrict__ sys, const BScal* sc, const BChunk* __restrict__ chunks,
                          ChunkList L) {
    for (int32_t k = blockIdx.x; k < *L.count; k += gridDim.x) {
        const int32_t c = L.act ? L.act[k] : k;
        const BChunk ch = chunks[c];
        if (!sc[ch.sys].fresh) continue;
        const BSys& sy = sys[ch.sys];
        const int32_t i = ch.row0 + threadIdx.x;
        if (i < ch.row1) sy.p[i] = sy.z[i];
    }
}

// ---- end of the start sequence: systems are no longer fresh ---------------
__global__ void kb_clear_fresh(BScal* sc, int32_t nslots) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nslots; k += gridDim.x * blockDim.x) sc[k].fresh = 0;
}

// ---- q = A p, pq, alpha ---------------------------------------------------
__global__ void kb_A_dot(const BSys* __restrict__ sys, BScal* sc, const BChunk* __restrict__ chunks,
                         ChunkList L, double* partials) {
    __shared__ double sh[32];
    for (int32_t k = blockIdx.x; k < *L.count; k += gridDim.x) {
        const int32_t c = L.act ? L.act[k] : k;
        const BChunk ch = chunks[c];
        BScal* s = &sc[ch.sys];
        if (s->done || s->fresh) continue;
        const BSys& sy = sys[ch.sys];
        const int32_t i = ch.row0 + threadIdx.x;
        double part = 0.0;
        if (i < ch.row1) {
            const double qi = row_f64(sy.Arp, sy.Acol, sy.Aval, sy.p, i);
            sy.q[i] = qi;
            part = sy.p[i] * qi;
        }
        const double tp = chunk_sum(part, sh);
        double tot;
        if (system_sum(tp, sy, c, partials, &s->ticket[2], &tot) && threadIdx.x == 0) s->alpha = s->rz / tot;
        __syncthreads();
    }
}

// ---- x += alpha p, r -= alpha q, rr, convergence --------------------------
__global__ void kb_update_xr(const BSys* __restrict__ sys, BScal* sc, const BChunk* __restrict__ chunks,
                             ChunkList L, double* partials, int r32) {
    __shared__ double sh[32];
    for (int32_t k = blockIdx.x; k < *L.count; k += gridDim.x) {
        const int32_t c = L.act ? L.act[k] : k;
        const BChunk ch = chunks[c];
        BScal* s = &sc[ch.sys];
        if (s->done || s->fresh) continue;
        const BSys& sy = sys[ch.sys];
        const double alpha = s->alpha;
        const int32_t i = ch.row0 + threadIdx.x;
        double part = 0.0;
        if (i < ch.row1) {
            sy.x[i] = fma(alpha, sy.p[i], sy.x[i]);
            const double ri = fma(-alpha, sy.q[i], sy.r[i]);
            sy.r[i] = ri;
            if (r32) r32_of(sy)[i] = static_cast<float>(ri);
            part = ri * ri;
        }
        const double tp = chunk_sum(part, sh);
        double tot;
        if (system_sum(tp, sy, c, partials, &s->ticket[3], &tot) && threadIdx.x == 0) {
            s->rr = tot;
            s->iters += 1;
            if (sqrt(tot) <= s->tolr) {
                s->done = 3;  // the true residual decides (kb_true_check)
            } else if (s->iters >= s->maxit) {
                s->done = 2;
                atomicSub(s->active, 1);
                atomicAdd(s->active + 3, 1);
            }
        }
        __syncthreads();
    }
}

// ---- the stopping rule's second half (Section 5.2, 8 orders of reduction):
// a system whose recursive residual met rtol ||b|| ends only if its true
// residual ||b - A x|| does too; otherwise its recurrence continues (the
// rest of this iteration runs for it) ------------------------------------
__global__ void kb_true_check(const BSys* __restrict__ sys, BScal* sc, const BChunk* __restrict__ chunks,
                              ChunkList L, double* partials) {
    __shared__ double sh[32];
    for (int32_t k = blockIdx.x; k < *L.count; k += gridDim.x) {
        const int32_t c = L.act ? L.act[k] : k;
        const BChunk ch = chunks[c];
        BScal* s = &sc[ch.sys];
        if (s->done != 3) continue;
        const BSys& sy = sys[ch.sys];
        const int32_t i = ch.row0 + threadIdx.x;
        double part = 0.0;
        if (i < ch.row1) {
            const double d = sy.b[i] - row_f64(sy.Arp, sy.Acol, sy.Aval, sy.x, i);
            part = d * d;
        }
        const double tp = chunk_sum(part, sh);
        double tot;
        if (system_sum(tp, sy, c, partials, &s->ticket[5], &tot) && threadIdx.x == 0) {
            s->true_rr = tot;
            if (sqrt(tot) <= s->tolr) {
                s->done = 1;
                atomicSub(s->active, 1);
                atomicAdd(s->active + 3, 1);
            } else if (s->iters >= s->maxit) {
                s->done = 2;
                atomicSub(s->active, 1);
                atomicAdd(s->active + 3, 1);
            } else {
                s->done = 0;
            }
        }
        __syncthreads();
    }
}

// ---- loop condition of the one-graph PCG: continue while systems run and
// the body budget lasts (counts[2], set by the host before the launch) -----
__global__ void kb_loop_cond(int32_t* counts, cudaGraphConditionalHandle h, int stop_on_retire,
                             const volatile int32_t* host_flag) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int32_t left = counts[2] - 1;
        counts[2] = left;
        bool go = counts[0] > 0 && left > 0;
        if (stop_on_retire && counts[3] > 0) go = false;
        if (host_flag && *host_flag != 0) go = false;
        cudaGraphSetConditional(h, go ? 1u : 0u);
    }
}

// ---- the running systems' chunks (d_act), listed again when forced or when
// a system finished since the last listing (counts[3] moved) ---------------
__global__ void kb_act_begin(int32_t* counts, int force) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const bool go = force || counts[3] != counts[5];
        counts[5] = counts[3];
        counts[6] = go ? 1 : 0;
        if (go) counts[4] = 0;
    }
}

// Warps append their chunks of running systems (one atomic per warp); the
// order of the list changes no result: each chunk keeps its partial slot
// (its index in the table) and a system's partials are summed in table
// order.
__global__ void kb_act_build(const BScal* __restrict__ sc, const BChunk* __restrict__ chunks, int32_t* counts,
                             int32_t* __restrict__ act) {
    if (counts[6] == 0) return;
    const int32_t n = counts[1];
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t w = w0; w * 32 < n; w += nw) {
        const int64_t c = w * 32 + lane;
        const bool keep = c < n && sc[chunks[c].sys].done == 0;
        const unsigned mask = __ballot_sync(kFull, keep);
        if (mask == 0u) continue;
        int32_t base = 0;
        if (lane == 0) base = atomicAdd(counts + 4, __popc(mask));
        base = __shfl_sync(kFull, base, 0);
        if (keep) act[base + __popc(mask & ((1u << lane) - 1u))] = static_cast<int32_t>(c);
    }
}

// ---- p = z + beta p --------------------------------------------------------
__global__ void kb_update_p(const BSys* __restrict__ sys, const BScal* sc, const BChunk* __restrict__ chunks,
                            ChunkList L) {
    for (int32_t k = blockIdx.x; k < *L.count; k += gridDim.x) {
        const int32_t c = L.act ? L.act[k] : k;
        const BChunk ch = chunks[c];
        const BScal* s = &sc[ch.sys];
        if (s->done || s->fresh) continue;
        const BSys& sy = sys[ch.sys];
        const int32_t i = ch.row0 + threadIdx.x;
        if (i < ch.row1) sy.p[i] = fma(s->beta, sy.p[i], sy.z[i]);
    }
}

// ---- true residual ||b - A x||^2 per system -------------------------------
__global__ void kb_true_residual(const BSys* __restrict__ sys, BScal* sc, const BChunk* __restrict__ chunks,
                                 ChunkList L, double* partials, int only_done) {
    __shared__ double sh[32];
    for (int32_t k = blockIdx.x; k < *L.count; k += gridDim.x) {
        const int32_t c = L.act ? L.act[k] : k;
        const BChunk ch = chunks[c];
        BScal* s = &sc[ch.sys];
        if (only_done && s->done == 0) continue;
        const BSys& sy = sys[ch.sys];
        const int32_t i = ch.row0 + threadIdx.x;
        double part = 0.0;
        if (i < ch.row1) {
            const double d = sy.b[i] - row_f64(sy.Arp, sy.Acol, sy.Aval, sy.x, i);
            part = d * d;
        }
        const double tp = chunk_sum(part, sh);
        double tot;
        if (system_sum(tp, sy, c, partials, &s->ticket[4], &tot) && threadIdx.x == 0) s->true_rr = tot;
        __syncthreads();
    }
}

// ---- packing of many CSRs into one block-diagonal CSR ---------------------
__global__ void kb_pack(int32_t nsys, const PackSrc* __restrict__ src, const int64_t* __restrict__ row_off,
                        int64_t nrows, int32_t* __restrict__ rowptr, int32_t* __restrict__ col,
                        double* __restrict__ val, int32_t* __restrict__ bad) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t g = gw; g < nrows; g += nw) {
        int lo = 0, hi = nsys - 1;  // system of row g: last s with row_off[s] <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_off[mid] <= g)
                lo = mid;
            else
                hi = mid - 1;
        }
        const PackSrc& s = src[lo];
        const int32_t i = static_cast<int32_t>(g - row_off[lo]);
        const int32_t b = s.rowptr[i], e = s.rowptr[i + 1];
        if (b < 0 || e < b || e > s.nnz) {
            if (lane == 0) atomicOr(bad, 1);
            if (lane == 0) rowptr[g] = static_cast<int32_t>(s.nnz_off);
            continue;
        }
        if (lane == 0) rowptr[g] = static_cast<int32_t>(s.nnz_off + b);
        for (int32_t k = b + lane; k < e; k += 32) {
            const int32_t c = s.col[k];
            col[s.nnz_off + k] = (c >= 0 && c < s.n) ? c + static_cast<int32_t>(row_off[lo]) : -1;
            val[s.nnz_off + k] = s.val[k];
        }
    }
}

// columns of the packed G / G^T back to system-local indices
__global__ void kb_localize(int32_t nsys, const int64_t* __restrict__ row_off, const int32_t* __restrict__ rowptr,
                            int64_t nrows, int32_t* __restrict__ col) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t g = gw; g < nrows; g += nw) {
        int lo = 0, hi = nsys - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_off[mid] <= g)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int32_t off = static_cast<int32_t>(row_off[lo]);
        for (int32_t k = rowptr[g] + lane; k < rowptr[g + 1]; k += 32) col[k] -= off;
    }
}

int grid_blocks() { return num_sms() * (2048 / kChunk); }

}  // namespace

// ---------------------------------------------------------------------------
// BatchEngine
// ---------------------------------------------------------------------------
afsai_status BatchEngine::reserve(int32_t max_sys, int64_t max_chunks, cudaStream_t st) {
    if (max_sys <= cap_sys && max_chunks <= cap_chunks) return AFSAI_OK;
    release(st);
    cap_sys = std::max<int32_t>(max_sys, 1);
    cap_chunks = std::max<int64_t>(max_chunks, 1);
    AFSAI_CUDA_TRY(lib_malloc_async(reinterpret_cast<void**>(&d_sys), sizeof(BSys) * cap_sys, st));
    AFSAI_CUDA_TRY(lib_malloc_async(reinterpret_cast<void**>(&d_sc), sizeof(BScal) * cap_sys, st));
    AFSAI_CUDA_TRY(lib_malloc_async(reinterpret_cast<void**>(&d_chunks), sizeof(BChunk) * cap_chunks, st));
    AFSAI_CUDA_TRY(lib_malloc_async(reinterpret_cast<void**>(&d_partials), sizeof(double) * cap_chunks, st));
    AFSAI_CUDA_TRY(lib_malloc_async(reinterpret_cast<void**>(&d_partials2), sizeof(double) * cap_chunks, st));
    AFSAI_CUDA_TRY(lib_malloc_async(reinterpret_cast<void**>(&d_act), sizeof(int32_t) * cap_chunks, st));
    AFSAI_CUDA_TRY(lib_malloc_async(reinterpret_cast<void**>(&d_counts), sizeof(int32_t) * 8, st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(d_counts, 0, sizeof(int32_t) * 8, st));
    AFSAI_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&h_counts), sizeof(int32_t) * 4));
    return AFSAI_OK;
}

void BatchEngine::release(cudaStream_t st) {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    if (d_sys) cudaFreeAsync(d_sys, st);
    if (d_sc) cudaFreeAsync(d_sc, st);
    if (d_chunks) cudaFreeAsync(d_chunks, st);
    if (d_partials) cudaFreeAsync(d_partials, st);
    if (d_partials2) cudaFreeAsync(d_partials2, st);
    if (d_counts) cudaFreeAsync(d_counts, st);
    if (d_act) cudaFreeAsync(d_act, st);
    if (h_counts) cudaFreeHost(h_counts);
    d_sys = nullptr;
    d_sc = nullptr;
    d_chunks = nullptr;
    d_partials = nullptr;
    d_partials2 = nullptr;
    d_counts = nullptr;
    d_act = nullptr;
    h_counts = nullptr;
    cap_sys = 0;
    cap_chunks = 0;
}

// Host tables -> device.  Systems get consecutive chunk ranges.
afsai_status BatchEngine::upload(const std::vector<BSys>& sys_in, const std::vector<BScal>& sc_in, cudaStream_t st) {
    std::vector<BSys> sys = sys_in;
    chunks_h.clear();
    for (size_t s = 0; s < sys.size(); ++s) {
        sys[s].chunk0 = static_cast<int32_t>(chunks_h.size());
        const int32_t nc = (sys[s].n + kChunk - 1) / kChunk;
        sys[s].nchunks = nc;
        for (int32_t c = 0; c < nc; ++c)
            chunks_h.push_back(BChunk{static_cast<int32_t>(s), c * kChunk, std::min(sys[s].n, (c + 1) * kChunk)});
    }
    AFSAI_TRY(reserve(static_cast<int32_t>(sys.size()), static_cast<int64_t>(chunks_h.size()), st));
    std::vector<BScal> sc = sc_in;
    for (auto& v : sc) {
        v.active = d_counts;
        v.fresh = 1;
    }
    if (!sys.empty()) {
        AFSAI_CUDA_TRY(cudaMemcpyAsync(d_sys, sys.data(), sizeof(BSys) * sys.size(), cudaMemcpyHostToDevice, st));
        AFSAI_CUDA_TRY(cudaMemcpyAsync(d_sc, sc.data(), sizeof(BScal) * sc.size(), cudaMemcpyHostToDevice, st));
        AFSAI_CUDA_TRY(cudaMemcpyAsync(d_chunks, chunks_h.data(), sizeof(BChunk) * chunks_h.size(),
                                       cudaMemcpyHostToDevice, st));
    }
    int32_t counts[4] = {static_cast<int32_t>(sys.size()), static_cast<int32_t>(chunks_h.size()), 0, 0};
    AFSAI_CUDA_TRY(cudaMemcpyAsync(d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, st));
    // the host array is pageable: wait for the copies before it goes away
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    return AFSAI_OK;
}

template <typename VT, typename TT>
afsai_status launch_precond(BatchEngine& E, int init, cudaStream_t st) {
    const int gb = grid_blocks();
    kb_G<VT, TT><<<gb, kChunk, 0, st>>>(E.d_sys, E.d_sc, E.d_chunks, init ? E.all() : E.active(), init);
    kb_Gt_dot<VT, TT><<<gb, kChunk, 0, st>>>(E.d_sys, E.d_sc, E.d_chunks, init ? E.all() : E.active(),
                                             E.d_partials, init);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return AFSAI_OK;
}

afsai_status BatchEngine::precond(int init, cudaStream_t st) {
    if (vtype == VAL_F64) return launch_precond<double, double>(*this, init, st);
    if (vtype == VAL_F32) return launch_precond<float, float>(*this, init, st);
    return launch_precond<__nv_bfloat16, float>(*this, init, st);
}

afsai_status BatchEngine::start(cudaStream_t st) {
    const int gb = grid_blocks();
    kb_init<<<gb, kChunk, 0, st>>>(d_sys, d_sc, d_chunks, all(), d_partials, d_partials2, vtype != VAL_F64);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    AFSAI_TRY(precond(1, st));
    kb_init_p<<<gb, kChunk, 0, st>>>(d_sys, d_sc, d_chunks, all());
    kb_clear_fresh<<<std::max(1, std::min(ceil_div(cap_sys, 256), 64)), 256, 0, st>>>(d_sc, cap_sys);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return AFSAI_OK;
}

afsai_status BatchEngine::set_tables(const std::vector<BSys>& sys_in, const std::vector<char>& running,
                                     int32_t nrunning, cudaStream_t st) {
    std::vector<BSys> sys = sys_in;
    chunks_h.clear();
    for (size_t s = 0; s < sys.size(); ++s) {
        sys[s].chunk0 = static_cast<int32_t>(chunks_h.size());
        sys[s].nchunks = 0;
        if (!running[s] || sys[s].n <= 0) continue;
        const int32_t nc = (sys[s].n + kChunk - 1) / kChunk;
        sys[s].nchunks = nc;
        for (int32_t c = 0; c < nc; ++c)
            chunks_h.push_back(BChunk{static_cast<int32_t>(s), c * kChunk, std::min(sys[s].n, (c + 1) * kChunk)});
    }
    if (static_cast<int32_t>(sys.size()) > cap_sys || static_cast<int64_t>(chunks_h.size()) > cap_chunks)
        return fail(AFSAI_ENOTSUP, "batch tables above their reserved capacity");
    if (!sys.empty())
        AFSAI_CUDA_TRY(cudaMemcpyAsync(d_sys, sys.data(), sizeof(BSys) * sys.size(), cudaMemcpyHostToDevice, st));
    if (!chunks_h.empty())
        AFSAI_CUDA_TRY(cudaMemcpyAsync(d_chunks, chunks_h.data(), sizeof(BChunk) * chunks_h.size(),
                                       cudaMemcpyHostToDevice, st));
    h_counts[0] = nrunning;
    h_counts[1] = static_cast<int32_t>(chunks_h.size());
    AFSAI_CUDA_TRY(cudaMemcpyAsync(d_counts, h_counts, sizeof(int32_t) * 2, cudaMemcpyHostToDevice, st));
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    return AFSAI_OK;
}

afsai_status BatchEngine::set_scalars(int32_t slot, const BScal& sc_in, cudaStream_t st) {
    if (slot < 0 || slot >= cap_sys) return fail(AFSAI_EINVAL, "slot out of range");
    BScal sc = sc_in;
    sc.active = d_counts;
    AFSAI_CUDA_TRY(cudaMemcpyAsync(d_sc + slot, &sc, sizeof(BScal), cudaMemcpyHostToDevice, st));
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    return AFSAI_OK;
}

afsai_status BatchEngine::iteration(cudaStream_t st) {
    const int gb = grid_blocks();
    kb_A_dot<<<gb, kChunk, 0, st>>>(d_sys, d_sc, d_chunks, active(), d_partials);
    kb_update_xr<<<gb, kChunk, 0, st>>>(d_sys, d_sc, d_chunks, active(), d_partials, vtype != VAL_F64);
    kb_true_check<<<gb, kChunk, 0, st>>>(d_sys, d_sc, d_chunks, active(), d_partials);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(3);
    AFSAI_TRY(precond(0, st));
    kb_update_p<<<gb, kChunk, 0, st>>>(d_sys, d_sc, d_chunks, active());
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFSAI_OK;
}

afsai_status BatchEngine::capture(int iters_per_graph, cudaStream_t st) {
    if (exec) {
        cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
    graph_iters = iters_per_graph;
    cudaGraph_t graph = nullptr;
    AFSAI_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int64_t before = launches_so_far();
    afsai_status cap = AFSAI_OK;
    for (int k = 0; k < iters_per_graph && cap == AFSAI_OK; ++k) cap = iteration(st);
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    per_graph = launches_so_far() - before;
    set_launches(before);
    if (cap != AFSAI_OK) {
        if (graph) cudaGraphDestroy(graph);
        return cap;
    }
    AFSAI_CUDA_TRY(ce);
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    AFSAI_CUDA_TRY(ie);
    return AFSAI_OK;
}

afsai_status BatchEngine::refresh_active(cudaStream_t st, bool force) {
    kb_act_begin<<<1, 32, 0, st>>>(d_counts, force ? 1 : 0);
    kb_act_build<<<grid_blocks(), kChunk, 0, st>>>(d_sc, d_chunks, d_counts, d_act);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return AFSAI_OK;
}

afsai_status BatchEngine::arm_loop(cudaStream_t st) {
    h_counts[2] = loop_bodies;
    h_counts[3] = 0;
    AFSAI_CUDA_TRY(cudaMemcpyAsync(d_counts + 2, h_counts + 2, 2 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    return AFSAI_OK;
}

afsai_status BatchEngine::capture_loop(int iters_per_body, int32_t max_bodies, cudaStream_t st, bool stop_on_retire,
                                       const volatile int32_t* host_flag) {
    if (exec) {
        cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
    graph_iters = iters_per_body;
    loop_bodies = std::max<int32_t>(max_bodies, 1);
    cudaGraph_t graph = nullptr;
    AFSAI_CUDA_TRY(cudaGraphCreate(&graph, 0));
    struct GraphGuard {
        cudaGraph_t g;
        ~GraphGuard() {
            if (g) cudaGraphDestroy(g);
        }
    } guard{graph};
    cudaGraphConditionalHandle handle;
    AFSAI_CUDA_TRY(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    AFSAI_CUDA_TRY(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    AFSAI_CUDA_TRY(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const int64_t before = launches_so_far();
    afsai_status cap = AFSAI_OK;
    for (int k = 0; k < iters_per_body && cap == AFSAI_OK; ++k) cap = iteration(st);
    if (cap == AFSAI_OK && use_act) cap = refresh_active(st, false);
    if (cap == AFSAI_OK) {
        kb_loop_cond<<<1, 32, 0, st>>>(d_counts, handle, stop_on_retire ? 1 : 0, host_flag);
        count_launches(1);
    }
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &captured);
    per_graph = launches_so_far() - before;  // kernels of one body
    set_launches(before);
    AFSAI_TRY(cap);
    AFSAI_CUDA_TRY(ce);
    AFSAI_CUDA_TRY(cudaGetLastError());
    AFSAI_CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
    return AFSAI_OK;
}

afsai_status BatchEngine::launch_graph(cudaStream_t st) {
    if (use_act) AFSAI_TRY(refresh_active(st, true));
    AFSAI_CUDA_TRY(cudaGraphLaunch(exec, st));
    count_launches(per_graph);
    return AFSAI_OK;
}

afsai_status BatchEngine::read_active(cudaStream_t st, int32_t* active) {
    AFSAI_CUDA_TRY(cudaMemcpyAsync(h_counts, d_counts, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, st));
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    *active = h_counts[0];
    return AFSAI_OK;
}

afsai_status BatchEngine::finish(cudaStream_t st, int only_done) {
    kb_true_residual<<<grid_blocks(), kChunk, 0, st>>>(d_sys, d_sc, d_chunks, all(), d_partials, only_done);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFSAI_OK;
}

// ---------------------------------------------------------------------------
// Packed set-up of many systems, by buckets
// ---------------------------------------------------------------------------
namespace {

// Longest row of each system's A (one block per system).
__global__ void kb_max_row(int32_t nsys, const PackSrc* __restrict__ src, int32_t* __restrict__ out) {
    __shared__ int32_t sh[32];
    for (int32_t s = blockIdx.x; s < nsys; s += gridDim.x) {
        const PackSrc p = src[s];
        int32_t mx = 0;
        for (int32_t i = threadIdx.x; i < p.n; i += blockDim.x) mx = max(mx, p.rowptr[i + 1] - p.rowptr[i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x < 32) {
            int32_t v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
            if (threadIdx.x == 0) out[s] = v;
        }
        __syncthreads();
    }
}

// Packs the members of a bucket into one block-diagonal CSR and runs the
// set-up on it; G and G^T come back with system-local column indices.
afsai_status setup_packed(const std::vector<PackSrc>& all, const std::vector<int32_t>& members,
                          const afsai_params* p, const SetupTuning* tune, cudaStream_t st, afsai_precond** out,
                          std::vector<int64_t>* row_off_h) {
    const int32_t nm = static_cast<int32_t>(members.size());
    row_off_h->assign(nm + 1, 0);
    std::vector<PackSrc> src(nm);
    int64_t nnz_total = 0;
    for (int32_t k = 0; k < nm; ++k) {
        src[k] = all[members[k]];
        src[k].nnz_off = nnz_total;
        (*row_off_h)[k + 1] = (*row_off_h)[k] + src[k].n;
        nnz_total += src[k].nnz;
    }
    const int64_t nrows = (*row_off_h)[nm];
    if (nrows >= INT32_MAX || nnz_total >= INT32_MAX) return fail(AFSAI_ENOTSUP, "batch larger than 2^31 rows/entries");
    DevBuf<PackSrc> dsrc;
    DevBuf<int64_t> droff;
    DevBuf<int32_t> bad, prp, pcol;
    DevBuf<double> pval;
    AFSAI_TRY(dsrc.alloc(nm, st));
    AFSAI_TRY(droff.alloc(nm + 1, st));
    AFSAI_TRY(bad.alloc(1, st));
    AFSAI_TRY(prp.alloc(nrows + 1, st));
    AFSAI_TRY(pcol.alloc(nnz_total, st));
    AFSAI_TRY(pval.alloc(nnz_total, st));
    AFSAI_CUDA_TRY(cudaMemcpyAsync(dsrc.p, src.data(), sizeof(PackSrc) * nm, cudaMemcpyHostToDevice, st));
    AFSAI_CUDA_TRY(cudaMemcpyAsync(droff.p, row_off_h->data(), sizeof(int64_t) * (nm + 1), cudaMemcpyHostToDevice, st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int32_t), st));
    const int32_t tot32 = static_cast<int32_t>(nnz_total);
    AFSAI_CUDA_TRY(cudaMemcpyAsync(prp.p + nrows, &tot32, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const int blocks = std::max(1, std::min(ceil_div(nrows * 32, 256), num_sms() * 16));
    kb_pack<<<blocks, 256, 0, st>>>(nm, dsrc.p, droff.p, nrows, prp.p, pcol.p, pval.p, bad.p);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    int32_t hbad = 0;
    AFSAI_CUDA_TRY(cudaMemcpyAsync(&hbad, bad.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    if (hbad) return fail(AFSAI_EINVAL, "a system has malformed row pointers");
    afsai_csr packed{static_cast<int32_t>(nrows), nnz_total, prp.p, pcol.p, pval.p};
    afsai_precond* M = nullptr;
    AFSAI_TRY(setup_precond(&packed, p, st, false, &M, tune));
    kb_localize<<<blocks, 256, 0, st>>>(nm, droff.p, M->G.rowptr, nrows, M->G.col);
    kb_localize<<<blocks, 256, 0, st>>>(nm, droff.p, M->Gt.rowptr, nrows, M->Gt.col);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    *out = M;
    return AFSAI_OK;
}

// Set-up autotuner: the solve kernel's tile (lanes per row, hence rows per
// warp) of the lane-per-row path, per bucket shape (pattern capacity,
// Cholesky precision), timed once per process on a sample of the bucket
// (members in order up to ~120k rows, each candidate twice, best time) and
// cached.  AFSAI_BATCH_LPR pins the choice.
struct TuneKey {
    int dev;
    int64_t mcap;
    int chol;
    bool operator<(const TuneKey& o) const {
        return std::tie(dev, mcap, chol) < std::tie(o.dev, o.mcap, o.chol);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune_cache;

afsai_status tune_lane_lpr(const std::vector<PackSrc>& all, const std::vector<int32_t>& members,
                           const afsai_params* p, cudaStream_t st, int* lpr_out) {
    const int64_t mcap = 1 + static_cast<int64_t>(p->kiter) * p->s;
    static const int pinned = [] {
        const char* e = std::getenv("AFSAI_BATCH_LPR");
        return e ? std::atoi(e) : 0;
    }();
    if (pinned > 0) {
        *lpr_out = pinned;
        return AFSAI_OK;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    const TuneKey key{dev, mcap, p->chol_prec};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *lpr_out = it->second;
            return AFSAI_OK;
        }
    }
    std::vector<int32_t> sample;
    int64_t rows = 0;
    for (int32_t m : members) {
        sample.push_back(m);
        rows += all[m].n;
        if (rows >= 120000) break;
    }
    const int cands[2] = {mcap > 12 ? 4 : 2, mcap > 12 ? 8 : 4};
    float best = 0.f;
    int choice = cands[0];
    cudaEvent_t e0, e1;
    AFSAI_CUDA_TRY(cudaEventCreate(&e0));
    AFSAI_CUDA_TRY(cudaEventCreate(&e1));
    afsai_status result = AFSAI_OK;
    for (int c = 0; c < 2 && result == AFSAI_OK; ++c) {
        SetupTuning t;
        t.lane_lpr = cands[c];
        for (int rep = 0; rep < 2 && result == AFSAI_OK; ++rep) {
            afsai_precond* M = nullptr;
            std::vector<int64_t> off;
            cudaEventRecord(e0, st);
            result = setup_packed(all, sample, p, &t, st, &M, &off);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (M) afsai_destroy(M);
            if (result == AFSAI_OK && (best == 0.f || ms < best)) {
                best = ms;
                choice = cands[c];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    AFSAI_TRY(result);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = choice;
    *lpr_out = choice;
    return AFSAI_OK;
}

}  // namespace

void free_buckets(std::vector<SetupBucket>* buckets) {
    for (auto& b : *buckets) {
        if (b.M) afsai_destroy(b.M);
        b.M = nullptr;
    }
    buckets->clear();
}

afsai_status batch_setup(int32_t nsys, const afsai_csr* A, const afsai_params* p, cudaStream_t st,
                         std::vector<SetupBucket>* buckets) {
    buckets->clear();
    std::vector<PackSrc> all(nsys);
    for (int32_t s = 0; s < nsys; ++s) {
        if (!A[s].rowptr || !A[s].col || !A[s].val || A[s].n <= 0 || A[s].nnz < A[s].n)
            return fail(AFSAI_EINVAL, "system " + std::to_string(s) + ": invalid CSR descriptor");
        all[s] = PackSrc{A[s].n, A[s].nnz, 0, A[s].rowptr, A[s].col, A[s].val};
    }
    // longest row of every system
    std::vector<int32_t> maxrow(nsys, 0);
    {
        DevBuf<PackSrc> dsrc;
        DevBuf<int32_t> dmax;
        AFSAI_TRY(dsrc.alloc(nsys, st));
        AFSAI_TRY(dmax.alloc(nsys, st));
        AFSAI_CUDA_TRY(cudaMemcpyAsync(dsrc.p, all.data(), sizeof(PackSrc) * nsys, cudaMemcpyHostToDevice, st));
        kb_max_row<<<std::max(1, std::min(nsys, num_sms() * 8)), 256, 0, st>>>(nsys, dsrc.p, dmax.p);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        AFSAI_CUDA_TRY(cudaMemcpyAsync(maxrow.data(), dmax.p, sizeof(int32_t) * nsys, cudaMemcpyDeviceToHost, st));
        AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    }
    // buckets by the length of the rows of A: at most kBucketShortRow
    // entries (the lane-per-row set-up path), and longer
    constexpr int32_t kBucketShortRow = 8;
    std::vector<SetupBucket> out(2);
    for (int32_t s = 0; s < nsys; ++s) {
        SetupBucket& b = out[maxrow[s] <= kBucketShortRow ? 0 : 1];
        b.members.push_back(s);
        b.max_row = std::max(b.max_row, maxrow[s]);
    }
    const int64_t mcap = 1 + static_cast<int64_t>(p->kiter) * p->s;
    for (auto& b : out) {
        if (b.members.empty()) continue;
        SetupTuning t;
        if (b.max_row <= kBucketShortRow && mcap <= 20 && p->s <= 4 && p->kiter > 0) {
            const afsai_status ts = tune_lane_lpr(all, b.members, p, st, &b.lane_lpr);
            if (ts != AFSAI_OK) {
                free_buckets(&out);
                return ts;
            }
            t.lane_lpr = b.lane_lpr;
        }
        const afsai_status ss = setup_packed(all, b.members, p, &t, st, &b.M, &b.row_off);
        if (ss != AFSAI_OK) {
            free_buckets(&out);
            return ss;
        }
        buckets->push_back(std::move(b));
    }
    return AFSAI_OK;
}

}  // namespace afsai

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace afsai;

namespace {

afsai_status batch_solve_impl(int32_t nsys, const afsai_csr* A, const afsai_params* params, const double* const* b,
                              double* const* x, double rtol, int32_t maxit, cudaStream_t st, pcg_info* info,
                              afsai_batch_info* binfo) {
    cudaEvent_t e0, e1, e2;
    AFSAI_CUDA_TRY(cudaEventCreate(&e0));
    AFSAI_CUDA_TRY(cudaEventCreate(&e1));
    AFSAI_CUDA_TRY(cudaEventCreate(&e2));
    AFSAI_CUDA_TRY(cudaEventRecord(e0, st));
    std::vector<SetupBucket> buckets;
    AFSAI_TRY(batch_setup(nsys, A, params, st, &buckets));
    AFSAI_CUDA_TRY(cudaEventRecord(e1, st));
    // vectors: systems back to back in batch order
    std::vector<int64_t> row_off(nsys + 1, 0);
    for (int32_t k = 0; k < nsys; ++k) row_off[k + 1] = row_off[k] + A[k].n;
    const int64_t ntot = row_off[nsys];
    int64_t nnz_G = 0;
    for (const auto& bk : buckets) nnz_G += bk.M->info.nnz_G;
    DevBuf<double> vec;
    afsai_status s = vec.alloc(static_cast<size_t>(ntot) * 5, st);
    BatchEngine E;
    if (s == AFSAI_OK) {
        std::vector<BSys> sys(nsys);
        std::vector<BScal> sc(nsys);
        for (const auto& bk : buckets) {
            for (size_t m = 0; m < bk.members.size(); ++m) {
                const int32_t k = bk.members[m];
                const int64_t go = bk.row_off[m];
                BSys& y = sys[k];
                y.Grp = bk.M->G.rowptr + go;
                y.Gcol = bk.M->G.col;
                y.Gval = bk.M->G.val;
                y.Trp = bk.M->Gt.rowptr + go;
                y.Tcol = bk.M->Gt.col;
                y.Tval = bk.M->Gt.val;
            }
        }
        for (int32_t k = 0; k < nsys; ++k) {
            BSys& y = sys[k];
            const int64_t o = row_off[k];
            y.n = A[k].n;
            y.Arp = A[k].rowptr;
            y.Acol = A[k].col;
            y.Aval = A[k].val;
            y.b = b[k];
            y.x = x[k];
            y.r = vec.p + o;
            y.p = vec.p + ntot + o;
            y.q = vec.p + 2 * ntot + o;
            y.z = vec.p + 3 * ntot + o;
            y.t = vec.p + 4 * ntot + o;
            BScal& c = sc[k];
            c = BScal{};
            c.rtol = rtol;
            c.maxit = maxit;
        }
        E.vtype = buckets.front().M->G.vtype;
        s = E.upload(sys, sc, st);
        if (s == AFSAI_OK) s = E.start(st);
        // the whole iteration loop is one graph launch: a device-side while
        // loop over bodies of K iterations, bounded by maxit
        const int K = 4;
        const int64_t max_bodies = maxit > 0 ? (static_cast<int64_t>(maxit) + K - 1) / K + 1 : 0;
        if (s == AFSAI_OK) s = E.capture_loop(K, static_cast<int32_t>(std::min<int64_t>(max_bodies, INT32_MAX)), st);
        int32_t active = nsys;
        int64_t launches = 0;
        if (s == AFSAI_OK) s = E.read_active(st, &active);
        if (s == AFSAI_OK && active > 0 && max_bodies > 0) {
            s = E.arm_loop(st);
            if (s == AFSAI_OK) s = E.launch_graph(st);
            ++launches;
            if (s == AFSAI_OK) s = E.read_active(st, &active);
            // launch_graph counted one body; the loop ran loop_bodies - left
            if (s == AFSAI_OK) count_launches((E.loop_bodies - E.h_counts[2] - 1) * E.per_graph);
        }
        if (s == AFSAI_OK) s = E.finish(st);
        if (s == AFSAI_OK && cudaEventRecord(e2, st) != cudaSuccess) s = fail(AFSAI_ECUDA, "cudaEventRecord");
        std::vector<BScal> out(nsys);
        if (s == AFSAI_OK) {
            if (cudaMemcpyAsync(out.data(), E.d_sc, sizeof(BScal) * nsys, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                s = fail(AFSAI_ECUDA, "reading batch results");
        }
        if (s == AFSAI_OK) {
            float ms_setup = 0.f, ms_solve = 0.f;
            cudaEventElapsedTime(&ms_setup, e0, e1);
            cudaEventElapsedTime(&ms_solve, e1, e2);
            int32_t maxi = 0, nconv = 0;
            for (int32_t k = 0; k < nsys; ++k) {
                const double bn = std::sqrt(out[k].bb);
                if (info) {
                    info[k] = pcg_info{};
                    info[k].iters = out[k].iters;
                    info[k].converged = out[k].done == 1 ? 1 : 0;
                    info[k].relres_rec = bn > 0 ? std::sqrt(out[k].rr) / bn : 0.0;
                    info[k].relres_true = bn > 0 ? std::sqrt(out[k].true_rr) / bn : 0.0;
                    info[k].solve_ms = ms_solve;
                }
                maxi = std::max(maxi, out[k].iters);
                nconv += out[k].done == 1 ? 1 : 0;
            }
            if (binfo) {
                binfo->nsys = nsys;
                binfo->total_rows = ntot;
                binfo->nnz_G = nnz_G;
                binfo->setup_ms = ms_setup;
                binfo->solve_ms = ms_solve;
                binfo->graph_launches = static_cast<int32_t>(launches);
                binfo->max_iters = maxi;
                binfo->converged = nconv;
            }
            if (nconv < nsys) s = fail(AFSAI_ENOCONV, std::to_string(nsys - nconv) + " system(s) reached maxit");
        }
    }
    E.release(st);
    vec.release();
    cudaStreamSynchronize(st);
    free_buckets(&buckets);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    return s;
}

}  // namespace

extern "C" afsai_status afsai_batch_solve(int32_t nsys, const afsai_csr* A, const afsai_params* params,
                                          const double* const* b, double* const* x, double rtol, int32_t maxit,
                                          void* stream, pcg_info* info, afsai_batch_info* binfo) {
    if (nsys <= 0 || !A || !params || !b || !x) return fail(AFSAI_EINVAL, "invalid batch arguments");
    AFSAI_TRY(check_params(params));
    if (params->block_rows != 0) return fail(AFSAI_ENOTSUP, "the locality bound applies to single-system set-ups");
    if (maxit < 0 || !(rtol >= 0.0)) return fail(AFSAI_EINVAL, "invalid rtol or maxit");
    for (int32_t k = 0; k < nsys; ++k)
        if (!b[k] || !x[k]) return fail(AFSAI_EINVAL, "NULL vector of system " + std::to_string(k));
    // the packed set-up uses a private non-blocking stream (graph capture
    // needs one), ordered after and joined back to the caller's stream
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaStream_t st;
    AFSAI_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaEvent_t join;
    AFSAI_CUDA_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    cudaEventRecord(join, user);
    cudaStreamWaitEvent(st, join, 0);
    const afsai_status s = batch_solve_impl(nsys, A, params, b, x, rtol, maxit, st, info, binfo);
    cudaEventRecord(join, st);
    cudaStreamWaitEvent(user, join, 0);
    cudaStreamSynchronize(st);
    cudaEventDestroy(join);
    cudaStreamDestroy(st);
    return s;
}
