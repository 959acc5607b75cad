// Batched PCG engine shared by afsai_batch_solve and the solve server.
#pragma once

#include <vector>

#include "afsai_internal.cuh"

namespace afsai {

constexpr int kChunk = 256;  // rows per chunk = threads per block

// One PCG problem of a batch: its matrix, preconditioner and vectors (all
// device pointers, system-local indices).
struct BSys {
    int32_t n;
    int32_t chunk0;   // first chunk of this system
    int32_t nchunks;  // chunks of this system
    int32_t pad;
    const int32_t* Arp;
    const int32_t* Acol;
    const double* Aval;
    const int32_t* Grp;  // rows of G (entries index the packed col/val arrays)
    const int32_t* Gcol;
    const void* Gval;
    const int32_t* Trp;  // rows of G^T
    const int32_t* Tcol;
    const void* Tval;
    const double* b;
    double* x;
    double* r;
    double* p;
    double* q;
    double* z;
    void* t;
};

// Per-system scalars (device).
struct BScal {
    double rz, alpha, beta, rr, bb, tolr, rtol, true_rr;  // tolr = rtol ||b||
    int32_t done;   // 0 running, 1 converged, 2 maxit reached, 3 true residual to check (within an iteration)
    int32_t iters;
    int32_t maxit;
    int32_t fresh;  // 1: not initialised yet (the start kernels act on fresh systems only)
    int32_t* active;  // device counter of running systems
    unsigned ticket[6];
};

struct BChunk {
    int32_t sys, row0, row1;
};

// The chunks a kernel visits: act[0 .. *count) (indices into the chunk
// table), or the whole table (act null, *count the table's size).
struct ChunkList {
    const int32_t* act;
    const int32_t* count;
};

struct PackSrc {
    int32_t n;
    int64_t nnz;
    int64_t nnz_off;
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
};

// Device tables + a captured graph of `graph_iters` PCG iterations.
struct BatchEngine {
    BSys* d_sys = nullptr;
    BScal* d_sc = nullptr;
    BChunk* d_chunks = nullptr;
    double* d_partials = nullptr;
    double* d_partials2 = nullptr;
    // [0] active systems, [1] chunks, [2] loop budget, [3] finished in a
    // launch, [4] chunks of running systems (d_act), [5] [3] when d_act was
    // built, [6] d_act to be rebuilt
    int32_t* d_counts = nullptr;
    int32_t* h_counts = nullptr;  // pinned
    int32_t* d_act = nullptr;     // chunks of the running systems
    ChunkList all() const { return ChunkList{nullptr, d_counts + 1}; }
    ChunkList active() const { return use_act ? ChunkList{d_act, d_counts + 4} : all(); }
    // The solve server rebuilds the chunk table of running systems before
    // every launch and ends a launch on any retirement, so it keeps the
    // whole table (use_act = false; set before capture_loop).
    bool use_act = true;
    // The running systems' chunks listed again (forced, or when a system
    // finished since the last listing): the iteration kernels then skip no
    // chunk of a finished system, which at the tail of an uneven batch (a
    // few systems running, tens of thousands of chunks) is most of their
    // work.
    afsai_status refresh_active(cudaStream_t st, bool force);
    int32_t cap_sys = 0;
    int64_t cap_chunks = 0;
    int32_t vtype = VAL_F64;
    std::vector<BChunk> chunks_h;
    cudaGraphExec_t exec = nullptr;
    int graph_iters = 0;
    int64_t per_graph = 0;

    afsai_status reserve(int32_t max_sys, int64_t max_chunks, cudaStream_t st);
    void release(cudaStream_t st);
    afsai_status upload(const std::vector<BSys>& sys, const std::vector<BScal>& sc, cudaStream_t st);
    // Slot-indexed tables: rewrites every descriptor (n = 0 marks a free
    // slot), rebuilds the chunk table over slots with running systems, and
    // sets the device count of running systems.  Scalars are not touched.
    afsai_status set_tables(const std::vector<BSys>& sys, const std::vector<char>& running, int32_t nrunning,
                            cudaStream_t st);
    afsai_status set_scalars(int32_t slot, const BScal& sc, cudaStream_t st);
    afsai_status start(cudaStream_t st);  // r = b - A x, z = M r, p = z
    afsai_status iteration(cudaStream_t st);
    afsai_status precond(int init, cudaStream_t st);
    afsai_status capture(int iters_per_graph, cudaStream_t st);
    // The whole PCG loop as one graph: a device-side while loop (a
    // conditional graph node) whose body runs iters_per_body iterations and
    // then a kernel that continues the loop while systems are running and
    // at most max_bodies bodies have run (the bound is kept on the device,
    // so the loop always ends).
    // With stop_on_retire the loop also ends after a body in which a system
    // finished (counts[3] > 0), and with host_flag (device view of mapped
    // pinned memory) once the host sets it (a request arrived).
    afsai_status capture_loop(int iters_per_body, int32_t max_bodies, cudaStream_t st, bool stop_on_retire = false,
                              const volatile int32_t* host_flag = nullptr);
    int32_t loop_bodies = 0;
    // Before a launch of the loop graph: the body budget, and the count of
    // systems finished during the launch cleared.
    afsai_status arm_loop(cudaStream_t st);
    afsai_status launch_graph(cudaStream_t st);
    afsai_status read_active(cudaStream_t st, int32_t* active);
    afsai_status finish(cudaStream_t st, int only_done = 0);  // true residuals (of finished systems only)
};

// Systems set up together: packed block-diagonally into one CSR whose
// set-up runs once over all its rows.
struct SetupBucket {
    std::vector<int32_t> members;   // system indices of the batch
    std::vector<int64_t> row_off;   // first packed row of each member (members + 1 entries)
    afsai_precond* M = nullptr;     // G and G^T of the bucket, system-local column indices
    int32_t max_row = 0;            // longest row of A in the bucket
    int lane_lpr = 0;               // solve-kernel lanes per row chosen by the autotuner (0: default)
};

// Groups the systems into buckets by the length of their rows of A (rows of
// at most 8 entries take the lane-per-row set-up path, longer rows the
// warp-per-row path), chooses each bucket's solve-kernel tile (rows per
// warp) with the set-up autotuner, packs each bucket and runs its set-up.
// Each system's G lives in exactly one bucket and equals the G of that
// system alone.
afsai_status batch_setup(int32_t nsys, const afsai_csr* A, const afsai_params* p, cudaStream_t st,
                         std::vector<SetupBucket>* buckets);
void free_buckets(std::vector<SetupBucket>* buckets);

}  // namespace afsai
