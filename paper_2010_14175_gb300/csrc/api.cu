// C ABI of libafsai.so (declarations and contracts in include/afsai.h).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <mutex>
#include <cstdlib>
#include <string>

#include "afsai_internal.cuh"

namespace afsai {

namespace {
thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};

// CSR validation: one thread per row.  Flags: 1 rowptr, 2 column range,
// 4 column order/duplicates, 8 missing diagonal, 16 non-positive diagonal.
__global__ void validate_kernel(int32_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ col, const double* __restrict__ val,
                                int32_t* __restrict__ flags, int32_t* __restrict__ maxrow) {
    int localmax = 0;
    int f = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t b = rowptr[i], e = rowptr[i + 1];
        if (i == 0 && b != 0) f |= 1;
        if (i == n - 1 && static_cast<int64_t>(e) != nnz) f |= 1;
        if (e < b || b < 0 || static_cast<int64_t>(e) > nnz) {
            f |= 1;
            continue;
        }
        localmax = max(localmax, e - b);
        int32_t prev = -1;
        bool diag = false;
        for (int32_t k = b; k < e; ++k) {
            const int32_t c = col[k];
            if (c < 0 || c >= n) {
                f |= 2;
                break;
            }
            if (c <= prev) f |= 4;
            prev = c;
            if (c == i) {
                diag = true;
                if (!(val[k] > 0.0)) f |= 16;
            }
        }
        if (!diag) f |= 8;
    }
    if (f) atomicOr(flags, f);
    if (localmax) atomicMax(maxrow, localmax);
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}


afsai_status check_csr_shape(const afsai_csr* A) {
    if (!A) return fail(AFSAI_EINVAL, "matrix is NULL");
    if (A->n <= 0) return fail(AFSAI_EINVAL, "n must be > 0");
    if (A->nnz < A->n || A->nnz > INT32_MAX) return fail(AFSAI_EINVAL, "nnz out of range (need n <= nnz < 2^31)");
    if (!A->rowptr || !A->col || !A->val) return fail(AFSAI_EINVAL, "NULL CSR array");
    return AFSAI_OK;
}

void destroy_precond(afsai_precond* M, cudaStream_t st) {
    if (!M) return;
    free_csr(&M->G, st);
    free_csr(&M->Gt, st);
    if (M->psi) cudaFreeAsync(M->psi, st);
    if (M->steps) cudaFreeAsync(M->steps, st);
    cudaStreamSynchronize(st);
    delete M;
}

afsai_status export_csr(const CsrDev& C, int32_t* rowptr, int32_t* col, double* val) {
    if (rowptr) AFSAI_CUDA_TRY(cudaMemcpy(rowptr, C.rowptr, sizeof(int32_t) * (C.n + 1), cudaMemcpyDeviceToHost));
    if (col && C.nnz > 0) AFSAI_CUDA_TRY(cudaMemcpy(col, C.col, sizeof(int32_t) * C.nnz, cudaMemcpyDeviceToHost));
    if (val && C.nnz > 0) {
        if (C.vtype == VAL_F64) {
            AFSAI_CUDA_TRY(cudaMemcpy(val, C.val, sizeof(double) * C.nnz, cudaMemcpyDeviceToHost));
        } else {
            const size_t bytes = val_bytes(C.vtype) * C.nnz;
            unsigned char* tmp = new (std::nothrow) unsigned char[bytes];
            if (!tmp) return fail(AFSAI_ENOMEM, "host buffer");
            const cudaError_t e = cudaMemcpy(tmp, C.val, bytes, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                delete[] tmp;
                return fail(AFSAI_ECUDA, cudaGetErrorString(e));
            }
            for (int64_t k = 0; k < C.nnz; ++k) {
                if (C.vtype == VAL_F32) {
                    float f;
                    std::memcpy(&f, tmp + 4 * k, 4);
                    val[k] = f;
                } else {
                    uint16_t h;
                    std::memcpy(&h, tmp + 2 * k, 2);
                    const uint32_t u = static_cast<uint32_t>(h) << 16;
                    float f;
                    std::memcpy(&f, &u, 4);
                    val[k] = f;
                }
            }
            delete[] tmp;
        }
    }
    return AFSAI_OK;
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

namespace {
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kPoolDevices] = {};
bool g_pool_failed[kPoolDevices] = {};
}  // namespace

cudaMemPool_t lib_pool() {
    static const bool enabled = [] {
        const char* e = std::getenv("AFSAI_POOL");
        return !e || std::atoi(e) != 0;
    }();
    if (!enabled) return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kPoolDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (g_pools[dev] || g_pool_failed[dev]) return g_pools[dev];
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        g_pool_failed[dev] = true;  // the default pool serves
        return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
    return pool;
}

void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
void set_launches(int64_t v) { g_launches.store(v, std::memory_order_relaxed); }

afsai_status fail(afsai_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

afsai_status validate_csr(const afsai_csr* A, cudaStream_t st, int32_t* max_row_nnz) {
    AFSAI_TRY(check_csr_shape(A));
    DevBuf<int32_t> flags;
    AFSAI_TRY(flags.alloc(2, st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int32_t), st));
    const int threads = 256;
    const int blocks = std::max(1, std::min(ceil_div(A->n, threads), num_sms() * 8));
    validate_kernel<<<blocks, threads, 0, st>>>(A->n, A->nnz, A->rowptr, A->col, A->val, flags.p, flags.p + 1);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    int32_t h[2] = {0, 0};
    AFSAI_CUDA_TRY(cudaMemcpyAsync(h, flags.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    if (h[0] & 1) return fail(AFSAI_EINVAL, "CSR row pointers are not monotone from 0 to nnz");
    if (h[0] & 2) return fail(AFSAI_EINVAL, "CSR column index out of range");
    if (h[0] & 4) return fail(AFSAI_EINVAL, "CSR columns not strictly increasing within a row");
    if (h[0] & 8) return fail(AFSAI_EINVAL, "CSR row without a diagonal entry");
    if (h[0] & 16) return fail(AFSAI_EINVAL, "non-positive diagonal entry (A is not SPD)");
    if (max_row_nnz) *max_row_nnz = h[1];
    return AFSAI_OK;
}

afsai_status check_params(const afsai_params* p) {
    if (!p) return fail(AFSAI_EINVAL, "params is NULL");
    if (p->kiter < 0) return fail(AFSAI_EINVAL, "kiter must be >= 0");
    if (p->s < 1) return fail(AFSAI_EINVAL, "s must be >= 1");
    if (!(p->eps >= 0.0)) return fail(AFSAI_EINVAL, "eps must be >= 0");
    if (p->exit_mode != 0 && p->exit_mode != 1) return fail(AFSAI_EINVAL, "exit_mode must be 0 or 1");
    if (p->g_prec < 0 || p->g_prec > 2) return fail(AFSAI_EINVAL, "g_prec must be 0, 1 or 2");
    if (p->chol_prec != 0 && p->chol_prec != 1) return fail(AFSAI_EINVAL, "chol_prec must be 0 or 1");
    if (1 + static_cast<int64_t>(p->kiter) * p->s > 128) return fail(AFSAI_ENOTSUP, "1 + kiter*s must be <= 128");
    if (p->block_rows < 0) return fail(AFSAI_EINVAL, "block_rows must be >= 0");
    if (p->block_power < 0 || p->block_power > 64) return fail(AFSAI_EINVAL, "block_power must be in [0, 64]");
    return AFSAI_OK;
}

afsai_status setup_precond(const afsai_csr* A, const afsai_params* params, cudaStream_t st, bool sliced,
                           afsai_precond** out, const SetupTuning* tune) {
    if (!out) return fail(AFSAI_EINVAL, "out is NULL");
    *out = nullptr;
    AFSAI_TRY(check_params(params));
    int32_t maxrow = 0;
    AFSAI_TRY(validate_csr(A, st, &maxrow));
    afsai_precond* M = new (std::nothrow) afsai_precond();
    if (!M) return fail(AFSAI_ENOMEM, "host allocation");
    cudaGetDevice(&M->device);
    M->params = *params;
    const afsai_status s = setup_impl(A, params, maxrow, st, M, sliced, tune);
    if (s != AFSAI_OK) {
        const std::string msg = g_last_error;
        destroy_precond(M, st);
        g_last_error = msg;
        return s;
    }
    if (sliced) static_apply_preload(st);
    *out = M;
    return AFSAI_OK;
}

}  // namespace afsai

using namespace afsai;

extern "C" {

const char* afsai_last_error(void) { return g_last_error.c_str(); }

const char* afsai_version(void) { return "afsai-gb300 0.1 (sm_103a)"; }

int64_t afsai_kernel_launches(void) { return launches_so_far(); }

afsai_status afsai_trim_pool(void) {
    cudaMemPool_t pool = lib_pool();
    if (!pool) return AFSAI_OK;
    AFSAI_CUDA_TRY(cudaMemPoolTrimTo(pool, 0));
    return AFSAI_OK;
}

afsai_status afsai_pool_stats(int64_t* used_bytes, int64_t* reserved_bytes) {
    if (!used_bytes && !reserved_bytes) return fail(AFSAI_EINVAL, "NULL arguments");
    uint64_t used = 0, reserved = 0;
    cudaMemPool_t pool = lib_pool();
    if (pool) {
        AFSAI_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
        AFSAI_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
    }
    if (used_bytes) *used_bytes = static_cast<int64_t>(used);
    if (reserved_bytes) *reserved_bytes = static_cast<int64_t>(reserved);
    return AFSAI_OK;
}

int32_t afsai_spmv_engine(int32_t role, int32_t n, int64_t nnz, int32_t vtype) {
    if (role < 0 || role > 2) return 0;
    return spmv_engine_of(role, n, nnz, vtype);
}


afsai_status afsai_setup(const afsai_csr* A, const afsai_params* params, void* stream, afsai_precond** out) {
    return setup_precond(A, params, static_cast<cudaStream_t>(stream), true, out);
}

afsai_status afsai_apply(const afsai_precond* M, const double* r, double* z, void* stream) {
    if (!M || !r || !z) return fail(AFSAI_EINVAL, "NULL argument");
    if (r == z) return fail(AFSAI_EINVAL, "r and z must not overlap");
    auto st = static_cast<cudaStream_t>(stream);
    DevBuf<double> t;
    AFSAI_TRY(t.alloc(M->G.n, st));
    return apply_precond(M, r, t.p, z, st);
}

afsai_status afsai_spmv(const afsai_csr* A, const double* x, double* y, void* stream) {
    AFSAI_TRY(check_csr_shape(A));
    if (!x || !y) return fail(AFSAI_EINVAL, "NULL vector");
    return spmv_csr(view_of(A), x, y, static_cast<cudaStream_t>(stream));
}

afsai_status pcg_solve(const afsai_csr* A, const afsai_precond* M, const double* b, double* x, double rtol,
                       int32_t maxit, void* stream, pcg_info* info) {
    AFSAI_TRY(check_csr_shape(A));
    if (!b || !x) return fail(AFSAI_EINVAL, "NULL vector");
    if (maxit < 0) return fail(AFSAI_EINVAL, "maxit must be >= 0");
    if (!(rtol >= 0.0)) return fail(AFSAI_EINVAL, "rtol must be >= 0");
    if (M && M->G.n != A->n) return fail(AFSAI_EINVAL, "preconditioner size differs from A");
    return pcg_impl(A, M, b, x, rtol, maxit, static_cast<cudaStream_t>(stream), info);
}

afsai_status afsai_solve_host(const afsai_csr* Ah, const afsai_params* params, const double* b_host, double* x_host,
                              double rtol, int32_t maxit, void* stream, afsai_info* setup_info, pcg_info* info) {
    AFSAI_TRY(check_csr_shape(Ah));
    AFSAI_TRY(check_params(params));
    if (!b_host || !x_host) return fail(AFSAI_EINVAL, "NULL vector");
    if (is_device_pointer(Ah->rowptr) || is_device_pointer(b_host))
        return fail(AFSAI_EINVAL, "afsai_solve_host expects host pointers");
    auto st = static_cast<cudaStream_t>(stream);
    const int32_t n = Ah->n;
    const int64_t nnz = Ah->nnz;
    DevBuf<int32_t> rp, ci;
    DevBuf<double> va, b, x;
    AFSAI_TRY(rp.alloc(static_cast<size_t>(n) + 1, st));
    AFSAI_TRY(ci.alloc(nnz, st));
    AFSAI_TRY(va.alloc(nnz, st));
    AFSAI_TRY(b.alloc(n, st));
    AFSAI_TRY(x.alloc(n, st));
    AFSAI_CUDA_TRY(cudaMemcpyAsync(rp.p, Ah->rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
    AFSAI_CUDA_TRY(cudaMemcpyAsync(ci.p, Ah->col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
    AFSAI_CUDA_TRY(cudaMemcpyAsync(va.p, Ah->val, sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
    AFSAI_CUDA_TRY(cudaMemcpyAsync(b.p, b_host, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(x.p, 0, sizeof(double) * n, st));
    afsai_csr Ad{n, nnz, rp.p, ci.p, va.p};
    afsai_precond* M = nullptr;
    AFSAI_TRY(afsai_setup(&Ad, params, stream, &M));
    if (setup_info) *setup_info = M->info;
    const afsai_status s = pcg_impl(&Ad, M, b.p, x.p, rtol, maxit, st, info);
    const std::string msg = g_last_error;
    destroy_precond(M, st);
    g_last_error = msg;
    if (s != AFSAI_OK && s != AFSAI_ENOCONV) return s;
    AFSAI_CUDA_TRY(cudaMemcpyAsync(x_host, x.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    return s;
}

afsai_status afsai_get_info(const afsai_precond* M, afsai_info* info) {
    if (!M || !info) return fail(AFSAI_EINVAL, "NULL argument");
    *info = M->info;
    return AFSAI_OK;
}

afsai_status afsai_export_G(const afsai_precond* M, int32_t* rowptr, int32_t* col, double* val) {
    if (!M) return fail(AFSAI_EINVAL, "NULL preconditioner");
    return export_csr(M->G, rowptr, col, val);
}

afsai_status afsai_export_Gt(const afsai_precond* M, int32_t* rowptr, int32_t* col, double* val) {
    if (!M) return fail(AFSAI_EINVAL, "NULL preconditioner");
    return export_csr(M->Gt, rowptr, col, val);
}

afsai_status afsai_export_rows(const afsai_precond* M, double* psi, int32_t* steps) {
    if (!M) return fail(AFSAI_EINVAL, "NULL preconditioner");
    if (psi) AFSAI_CUDA_TRY(cudaMemcpy(psi, M->psi, sizeof(double) * M->G.n, cudaMemcpyDeviceToHost));
    if (steps) AFSAI_CUDA_TRY(cudaMemcpy(steps, M->steps, sizeof(int32_t) * M->G.n, cudaMemcpyDeviceToHost));
    return AFSAI_OK;
}

void afsai_destroy(afsai_precond* M) {
    if (!M) return;
    cudaStreamSynchronize(nullptr);
    destroy_precond(M, nullptr);
}

}  // extern "C"
