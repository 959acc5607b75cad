// Sliced ELLPACK (SELL-32-sigma) copies of CSR matrices for the row engine
// of spmv_tiled.cuh that gives one row to each lane of a warp.
//
// With one lane per row every FP64 fma of a warp instruction is a useful
// product as long as the 32 rows of a slice have the same length, and no
// lane-combining shuffles are needed; loads of a slice are k-major, so the
// 32 lanes read 32 consecutive columns and values.  Sorting rows by length
// inside windows of 4096 rows keeps the slices even on matrices whose rows
// vary (the rows of G^T are the column counts of G: 1 to ~80 on 3D
// problems) while the window bounds how far the rows of a slice lie apart.
//
// A copy whose padding would exceed the matrix's own entries is not built
// (the CSR engines serve such matrices).
//
// Build: (1) one block per window sorts its rows by (decreasing length,
// increasing index) with a bitonic network on 32-bit keys in shared memory;
// (2) one warp per slice takes the longest row of the slice; (3) an
// exclusive scan of those lengths gives the slice offsets; (4) one warp per
// slice copies its rows, lane l writing slot 32 (kptr[s] + k) + l.
#include <algorithm>

#include "afsai_internal.cuh"

namespace afsai {
namespace {

constexpr int kWin = 32 * kSellWindowSlices;    // rows per sorting window
constexpr int kWinLog2 = 12;
static_assert(kWin == 1 << kWinLog2, "window of 4096 rows");
constexpr uint32_t kLenClamp = (1u << 20) - 2;  // keys stay below 0xffffffff
constexpr uint32_t kNoRow = 0xffffffffu;

__global__ void __launch_bounds__(1024) sell_sort_windows(int32_t n, const int32_t* __restrict__ rowptr,
                                                          int64_t nlanes, int2* __restrict__ rowlen) {
    __shared__ uint32_t key[kWin];
    const int64_t w0 = static_cast<int64_t>(blockIdx.x) * kWin;
    for (int j = threadIdx.x; j < kWin; j += blockDim.x) {
        const int64_t i = w0 + j;
        uint32_t k = kNoRow;
        if (i < n) {
            const uint32_t len = static_cast<uint32_t>(rowptr[i + 1] - rowptr[i]);
            k = ((kLenClamp - (len < kLenClamp ? len : kLenClamp)) << kWinLog2) | static_cast<uint32_t>(j);
        }
        key[j] = k;
    }
    __syncthreads();
    // ascending bitonic sort of unique keys
    for (int size = 2; size <= kWin; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int j = threadIdx.x; j < kWin; j += blockDim.x) {
                const int partner = j ^ stride;
                if (partner > j) {
                    const uint32_t a = key[j], b = key[partner];
                    const bool up = (j & size) == 0;
                    if ((a > b) == up) {
                        key[j] = b;
                        key[partner] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int j = threadIdx.x; j < kWin; j += blockDim.x) {
        const int64_t pos = w0 + j;
        if (pos >= nlanes) continue;
        const uint32_t k = key[j];
        int2 v = make_int2(-1, 0);
        if (k != kNoRow) {
            const int32_t i = static_cast<int32_t>(w0 + (k & (kWin - 1)));
            v = make_int2(i, rowptr[i + 1] - rowptr[i]);
        }
        rowlen[pos] = v;
    }
}

// kcount[s] = longest row of slice s (one warp per slice)
__global__ void sell_slice_len(int32_t nslices, const int2* __restrict__ rowlen, int32_t* __restrict__ kcount) {
    const int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    int32_t m = rowlen[s * 32 + lane].y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) kcount[s] = m;
}

template <typename VT>
__global__ void sell_fill(int32_t nslices, const int32_t* __restrict__ kptr, const int2* __restrict__ rowlen,
                          const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const VT* __restrict__ val, int32_t* __restrict__ scol, VT* __restrict__ sval) {
    const int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    const int2 rl = rowlen[s * 32 + lane];
    const int32_t K = kptr[s + 1] - kptr[s];
    const int64_t b = rl.x >= 0 ? static_cast<int64_t>(rowptr[rl.x]) : 0;
    const int64_t base = static_cast<int64_t>(kptr[s]) * 32 + lane;
    for (int32_t k = 0; k < K; ++k) {
        const int64_t dst = base + static_cast<int64_t>(k) * 32;
        if (k < rl.y) {
            scol[dst] = col[b + k];
            sval[dst] = val[b + k];
        } else {
            scol[dst] = 0;
            sval[dst] = VT(0.0f);
        }
    }
}

}  // namespace

// Row order of each tile of kTileOrderRows rows, longest row first (ties
// by row index): thread t of the tile counts the rows that precede its row
// in that order (a deterministic rank; a few hundred comparisons per row,
// once per matrix).
__global__ void tile_order_kernel(int32_t n, const int32_t* __restrict__ rowptr, uint8_t* __restrict__ order) {
    __shared__ int32_t len[kTileOrderRows];
    const int t = threadIdx.x;
    for (int64_t r0 = static_cast<int64_t>(blockIdx.x) * kTileOrderRows; r0 < n;
         r0 += static_cast<int64_t>(gridDim.x) * kTileOrderRows) {
        const int nr = static_cast<int>(n - r0 < kTileOrderRows ? n - r0 : kTileOrderRows);
        const int32_t mine = t < nr ? rowptr[r0 + t + 1] - rowptr[r0 + t] : -1;
        len[t] = mine;
        __syncthreads();
        if (t < nr) {
            int rank = 0;
            for (int j = 0; j < nr; ++j) {
                const int32_t lj = len[j];
                rank += (lj > mine || (lj == mine && j < t)) ? 1 : 0;
            }
            order[r0 + rank] = static_cast<uint8_t>(t);
        }
        __syncthreads();
    }
}

void free_sell(SellDev* S, cudaStream_t st) {
    if (S->order) cudaFreeAsync(S->order, st);
    if (S->kptr) cudaFreeAsync(S->kptr, st);
    if (S->rowlen) cudaFreeAsync(S->rowlen, st);
    if (S->col) cudaFreeAsync(S->col, st);
    if (S->val) cudaFreeAsync(S->val, st);
    *S = SellDev{};
}

afsai_status build_sell(const CsrDev& C, SellDev* S, cudaStream_t st, bool with_order) {
    *S = SellDev{};
    if (C.n <= 0) return AFSAI_OK;
    const int32_t nslices = static_cast<int32_t>((static_cast<int64_t>(C.n) + 31) / 32);
    const int64_t nlanes = static_cast<int64_t>(nslices) * 32;
    const int nwin = static_cast<int>((static_cast<int64_t>(C.n) + kWin - 1) / kWin);
    DevBuf<int32_t> kptr, kcount;
    DevBuf<int2> rowlen;
    AFSAI_TRY(rowlen.alloc(static_cast<size_t>(nlanes), st));
    AFSAI_TRY(kcount.alloc(static_cast<size_t>(nslices), st));
    AFSAI_TRY(kptr.alloc(static_cast<size_t>(nslices) + 1, st));
    sell_sort_windows<<<nwin, 1024, 0, st>>>(C.n, C.rowptr, nlanes, rowlen.p);
    const int sblocks = ceil_div(nlanes, 256);
    sell_slice_len<<<sblocks, 256, 0, st>>>(nslices, rowlen.p, kcount.p);
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    int64_t kslots = 0;
    AFSAI_TRY(exclusive_scan_i32(kcount.p, kptr.p, nslices, st, &kslots));
    const int64_t nslots = kslots * 32;
    // a few very long rows (an arrowhead matrix) pad their slices to their
    // length: past twice the entries the copy is not built
    if (nslots > 2 * C.nnz + 32 * static_cast<int64_t>(kSellWindowSlices))
        return fail(AFSAI_ENOTSUP, "sliced copy not built: padding would exceed the matrix entries");
    const size_t vb = val_bytes(C.vtype);
    DevBuf<int32_t> scol;
    DevBuf<unsigned char> sval;
    AFSAI_TRY(scol.alloc(static_cast<size_t>(std::max<int64_t>(nslots, 1)), st));
    AFSAI_TRY(sval.alloc(static_cast<size_t>(std::max<int64_t>(nslots, 1)) * vb, st));
    if (C.vtype == VAL_F64)
        sell_fill<double><<<sblocks, 256, 0, st>>>(nslices, kptr.p, rowlen.p, C.rowptr, C.col,
                                                   static_cast<const double*>(C.val), scol.p,
                                                   reinterpret_cast<double*>(sval.p));
    else if (C.vtype == VAL_F32)
        sell_fill<float><<<sblocks, 256, 0, st>>>(nslices, kptr.p, rowlen.p, C.rowptr, C.col,
                                                  static_cast<const float*>(C.val), scol.p,
                                                  reinterpret_cast<float*>(sval.p));
    else
        sell_fill<__nv_bfloat16><<<sblocks, 256, 0, st>>>(nslices, kptr.p, rowlen.p, C.rowptr, C.col,
                                                          static_cast<const __nv_bfloat16*>(C.val), scol.p,
                                                          reinterpret_cast<__nv_bfloat16*>(sval.p));
    AFSAI_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    if (with_order) {
        DevBuf<uint8_t> order;
        AFSAI_TRY(order.alloc(static_cast<size_t>(C.n), st));
        const int oblocks = std::max(1, std::min(ceil_div(C.n, kTileOrderRows), num_sms() * 8));
        tile_order_kernel<<<oblocks, kTileOrderRows, 0, st>>>(C.n, C.rowptr, order.p);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        S->order = order.detach();
    }
    S->nslices = nslices;
    S->nslots = nslots;
    S->kptr = kptr.detach();
    S->rowlen = rowlen.detach();
    S->col = scol.detach();
    S->val = sval.detach();
    return AFSAI_OK;
}

}  // namespace afsai
