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
    double rz, alpha, beta, rr, bb, tol2, rtol, true_rr;
    int32_t done;   // 0 running, 1 converged, 2 maxit reached
    int32_t iters;
    int32_t maxit;
    int32_t fresh;  // 1: not initialised yet (the start kernels act on fresh systems only)
    int32_t* active;  // device counter of running systems
    unsigned ticket[6];
};

struct BChunk {
    int32_t sys, row0, row1;
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
    int32_t* d_counts = nullptr;  // [0] active systems, [1] chunks
    int32_t* h_counts = nullptr;  // pinned
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
    afsai_status launch_graph(cudaStream_t st);
    afsai_status read_active(cudaStream_t st, int32_t* active);
    afsai_status finish(cudaStream_t st, int only_done = 0);  // true residuals (of finished systems only)
};

// Packs the systems into one block-diagonal CSR and runs the set-up on it.
// On return G and G^T of *out are packed with system-local column indices;
// row_off holds the first packed row of every system (nsys + 1 entries).
afsai_status batch_setup(int32_t nsys, const afsai_csr* A, const afsai_params* p, cudaStream_t st,
                         afsai_precond** out, std::vector<int64_t>* row_off);

}  // namespace afsai
