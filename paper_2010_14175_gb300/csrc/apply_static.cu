// afsai_apply_static: the preconditioner application z = G^T (G r) for
// callers that cannot allocate device memory.  See include/afsai.h.
//
// The intermediate vector t = G r lives in a file-scope device array of
// fixed size instead of a per-call allocation.  Host code cannot pass the
// array's name to a kernel (in host code it names a host-side stand-in),
// so its device address is looked up with cudaGetSymbolAddress while the
// device is current and cached per device.  The runtime loads this file's
// module, and with it the array, lazily, at that first lookup; afsai_setup
// therefore does the lookup (static_apply_preload), so that the array is
// in place before a caller that cannot allocate holds a preconditioner.
#include <mutex>
#include <string>

#include "afsai_internal.cuh"
#include "spmv_tiled.cuh"

namespace afsai {
namespace {

// Largest n served: 2^20 rows, i.e. 8 MiB of device memory held by every
// GPU that loads the library, for the whole life of the process.
constexpr int32_t kStaticApplyMaxRows = 1 << 20;

__device__ __align__(256) double g_apply_scratch[kStaticApplyMaxRows];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_apply_scratch on the current device, looked up (and
// the module loaded) on the first request per device.  `may_load` = false
// refuses to do that first lookup during a stream capture, where loading a
// module is not allowed, with a message that says what to do instead.
afsai_status scratch_address(double** out, cudaStream_t st, bool may_load) {
    int dev = 0;
    AFSAI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(AFSAI_ENOTSUP, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        if (!may_load) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
                return fail(AFSAI_EINVAL,
                            "afsai_apply_static: its device array is not loaded on this device yet and the "
                            "stream is capturing; call afsai_setup (or afsai_apply_static once) on this device "
                            "before the capture");
        }
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? AFSAI_ENOMEM : AFSAI_ECUDA,
                        std::string("loading the 8 MiB device array of afsai_apply_static: ") +
                            cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return AFSAI_OK;
}

}  // namespace

// Called at the end of a successful afsai_setup on the current device.
// Best effort: a failure here (no device memory left for the array) is not
// an error of the set-up; afsai_apply_static reports it at its first call.
void static_apply_preload(cudaStream_t st) {
    const std::string keep = afsai_last_error();
    double* p = nullptr;
    if (scratch_address(&p, st, true) != AFSAI_OK) set_error(keep);
}

}  // namespace afsai

using namespace afsai;

extern "C" afsai_status afsai_apply_static(const afsai_precond* M, const double* r, double* z, void* stream) {
    if (!M || !r || !z) return fail(AFSAI_EINVAL, "NULL argument");
    if (r == z) return fail(AFSAI_EINVAL, "r and z must not overlap");
    if (M->G.n > kStaticApplyMaxRows)
        return fail(AFSAI_EINVAL, "afsai_apply_static serves n <= " + std::to_string(kStaticApplyMaxRows) +
                                      " rows (got n = " + std::to_string(M->G.n) + "); use afsai_apply");
    auto st = static_cast<cudaStream_t>(stream);
    int dev = -1;
    AFSAI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != M->device)
        return fail(AFSAI_EINVAL, "afsai_apply_static: the preconditioner belongs to device " +
                                      std::to_string(M->device) + ", the current device is " + std::to_string(dev));
    double* t = nullptr;
    AFSAI_TRY(scratch_address(&t, st, false));
    // engines: the cached choice if the matrix was tuned before, else the
    // default for its row length (no timing, no allocation)
    SpmvMode mg, mt;
    AFSAI_TRY(spmv_mode_for(ROLE_G, M->G, st, &mg, false));
    AFSAI_TRY(spmv_mode_for(ROLE_GT, M->Gt, st, &mt, false));
    // t is written in full by the first product, so nothing needs clearing
    AFSAI_TRY(spmv_launch_role(ROLE_G, mg, M->G, r, t, st));
    return spmv_launch_role(ROLE_GT, mt, M->Gt, t, z, st);
}
