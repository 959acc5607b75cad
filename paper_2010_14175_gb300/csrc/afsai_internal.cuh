// Internal declarations shared by the translation units of libafsai.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "afsai.h"

namespace afsai {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
afsai_status fail(afsai_status st, const std::string& msg);

#define AFSAI_CUDA_TRY(expr)                                                                   \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            return ::afsai::fail(e_ == cudaErrorMemoryAllocation ? AFSAI_ENOMEM : AFSAI_ECUDA, \
                                 std::string(#expr) + ": " + cudaGetErrorString(e_));          \
        }                                                                                      \
    } while (0)

#define AFSAI_TRY(expr)                         \
    do {                                        \
        afsai_status s_ = (expr);               \
        if (s_ != AFSAI_OK) return s_;          \
    } while (0)

// ---------------------------------------------------------------------------
// device memory: the library's own stream-ordered pool per device
// ---------------------------------------------------------------------------
// Stream-ordered allocation from a pool that the library owns on each
// device (created at first use on the current device).  Freed blocks stay
// in the pool for the next call instead of being unmapped and mapped again
// (a set-up of the 256^3 problem allocates and frees several GB of
// temporaries); afsai_trim_pool returns them to the device.  With
// AFSAI_POOL=0 the device's default pool is used instead.
cudaMemPool_t lib_pool();
inline cudaError_t lib_malloc_async(void** p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = lib_pool();
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
}

// ---------------------------------------------------------------------------
// device buffers (stream-ordered allocation)
// ---------------------------------------------------------------------------
template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    afsai_status alloc(size_t count, cudaStream_t s) {
        release();
        st = s;
        n = count;
        if (count == 0) return AFSAI_OK;
        cudaError_t e = lib_malloc_async(reinterpret_cast<void**>(&p), count * sizeof(T), s);
        if (e != cudaSuccess) {
            p = nullptr;
            n = 0;
            return fail(AFSAI_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        }
        return AFSAI_OK;
    }
    void release() {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        n = 0;
    }
    T* detach() {
        T* q = p;
        p = nullptr;
        n = 0;
        return q;
    }
};

// G / G^T storage: values in one of three types.
enum ValType : int32_t { VAL_F64 = 0, VAL_F32 = 1, VAL_BF16 = 2 };

inline size_t val_bytes(int32_t vt) { return vt == VAL_F64 ? 8 : (vt == VAL_F32 ? 4 : 2); }

// Sliced ELLPACK copy of a CSR matrix (SELL-32-sigma): rows are sorted by
// decreasing length inside windows of 4096 rows (stable, so rows of equal
// length keep their order) and cut into slices of 32; slice s stores its
// entries k-major in slots [32 kptr[s], 32 kptr[s + 1]): entry k of lane l
// at slot 32 (kptr[s] + k) + l, with kptr[s + 1] - kptr[s] the longest row
// of the slice.  Slots past a row's length hold column 0 and value 0 and
// are never read.  rowlen[32 s + l] = (row, length), row -1 past n.  Each
// row keeps the CSR order of its entries.
constexpr int kSellWindowSlices = 128;  // slices per sorting window (4096 rows)

struct SellDev {
    int32_t nslices = 0;
    int64_t nslots = 0;
    int32_t* kptr = nullptr;  // nslices + 1
    int2* rowlen = nullptr;   // 32 nslices
    int32_t* col = nullptr;   // nslots
    void* val = nullptr;      // nslots, the value type of the CSR
    // built with the sliced copy: for each tile of kTileOrderRows rows of
    // the CSR, its rows by length (longest first; ties by row), as indices
    // within the tile (n bytes)
    uint8_t* order = nullptr;
};
constexpr int kTileOrderRows = 256;

struct CsrDev {
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t* rowptr = nullptr;
    int32_t* col = nullptr;
    void* val = nullptr;  // double / float / __nv_bfloat16 by vtype
    int32_t vtype = VAL_F64;
    int32_t max_row = 0;
    SellDev sell;         // empty unless a sliced copy was built
};

}  // namespace afsai

struct afsai_precond {
    afsai::CsrDev G;
    afsai::CsrDev Gt;
    double* psi = nullptr;     // n
    int32_t* steps = nullptr;  // n
    afsai_params params{};
    afsai_info info{};
    int device = 0;
};

namespace afsai {

// ---------------------------------------------------------------------------
// entry points of the translation units
// ---------------------------------------------------------------------------

// Checks set-up parameters on the host (EINVAL / ENOTSUP with a message).
afsai_status check_params(const afsai_params* p);

// Validates a device CSR (see afsai.h); synchronises the stream.
afsai_status validate_csr(const afsai_csr* A, cudaStream_t st, int32_t* max_row_nnz);

// SpMV engine chosen so far for a role (0 A, 1 G, 2 G^T) and matrix shape
// on the current device (0 if none).
int spmv_engine_of(int role, int32_t n, int64_t nnz, int vtype);

// Set-up (setup.cu).  Fills M->G, M->Gt, M->psi, M->steps.
// sliced = true also builds the sliced copies of G and G^T (the PCG and
// apply engines of a single system); the batched and serving forms, which
// run their own kernels on the CSR, pass false.
// Lanes per row of the solve kernel of the small-stencil set-up path (0:
// the default for the pattern size).  The batched form's autotuner sets it
// per bucket of systems.
struct SetupTuning {
    int lane_lpr = 0;
};

afsai_status setup_impl(const afsai_csr* A, const afsai_params* p, int32_t max_row_nnz, cudaStream_t st,
                        afsai_precond* M, bool sliced, const SetupTuning* tune = nullptr);

// afsai_setup with the choice of sliced copies (api.cu).
afsai_status setup_precond(const afsai_csr* A, const afsai_params* p, cudaStream_t st, bool sliced,
                           afsai_precond** out, const SetupTuning* tune = nullptr);

// Sparse building blocks (sparse.cu).
afsai_status exclusive_scan_i32(const int32_t* in, int32_t* out, int32_t n, cudaStream_t st, int64_t* total_host);
afsai_status build_transpose(const CsrDev& G, CsrDev* Gt, cudaStream_t st);
// Sliced copy of C (sell.cu), with_order: and the tile row order; *S stays
// empty on failure.
afsai_status build_sell(const CsrDev& C, SellDev* S, cudaStream_t st, bool with_order = true);
void free_sell(SellDev* S, cudaStream_t st);
afsai_status spmv_csr(const CsrDev& A, const double* x, double* y, cudaStream_t st);
afsai_status apply_precond(const afsai_precond* M, const double* r, double* t, double* z, cudaStream_t st);
void free_csr(CsrDev* A, cudaStream_t st);
int32_t* error_flag();  // device flag set by a bounded device-side wait that ran out

// Loads the device array of afsai_apply_static on the current device
// (apply_static.cu); best effort, called by afsai_setup.
void static_apply_preload(cudaStream_t st);

// PCG (pcg.cu).
afsai_status pcg_impl(const afsai_csr* A, const afsai_precond* M, const double* b, double* x, double rtol,
                      int32_t maxit, cudaStream_t st, pcg_info* info);

inline CsrDev view_of(const afsai_csr* A) {
    CsrDev v;
    v.n = A->n;
    v.nnz = A->nnz;
    v.rowptr = const_cast<int32_t*>(A->rowptr);
    v.col = const_cast<int32_t*>(A->col);
    v.val = const_cast<double*>(A->val);
    v.vtype = VAL_F64;
    return v;
}

inline int ceil_div(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

int num_sms();

// Blocks of `kern` (threads, dynamic shared memory) resident on the GPU at
// once, capped at `blocks`.  The SpMV engines loop grid-stride, so a grid
// trimmed to this count does the same work; the engine plans count shared
// memory and threads, not the registers of the kernel that finally runs.
// A fused kernel a few registers above the plain product would run its
// last blocks as a second wave (rows of 7 entries: 7 blocks of 256
// threads per SM at 32 registers, 6 at 34, so every seventh block waits
// for the others and the product takes twice as long).
template <typename K>
int resident_grid(K kern, int blocks, int threads, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        return blocks;
    }
    return per_sm * num_sms() < blocks ? per_sm * num_sms() : blocks;
}

// Kernel launch accounting (reported by afsai_kernel_launches()).
void count_launches(int64_t k);
int64_t launches_so_far();
void set_launches(int64_t v);

}  // namespace afsai
