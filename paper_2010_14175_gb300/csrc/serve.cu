// Solve server: continuous batching of aFSAI-PCG solves on one GPU.
//
// Matrices are registered once (copied to the device); the aFSAI set-up of
// a matrix runs at its first request and its G, G^T stay resident and are
// reused by later requests of the same matrix.  A request brings 1..k
// right-hand sides; each becomes one system of the batched engine
// (batch.cu) in a slot with its own vectors.  A server thread runs the step
// loop:
//   admit   queued requests in arrival order while they fit (free slots for
//           their right-hand sides, device-memory budget for their vectors):
//           allocate vectors, copy b, initialise only the new systems.  A
//           request whose matrix has no preconditioner yet hands its
//           set-up to the set-up thread (its own stream, so the set-up
//           overlaps the running systems on the GPU) and waits for it;
//           the requests behind it may be admitted meanwhile;
//   step    one graph launch: a device-side loop of bodies of K PCG
//           iterations of every running system, which ends after the body
//           in which a system finished, when a new request arrives (the
//           submitting thread raises a flag in mapped host memory that the
//           loop reads) or after a bounded number of bodies;
//   retire  systems that converged (or hit maxit) get their true residual,
//           x goes back to the request's host buffer, the slot and its
//           memory are freed and the next requests can enter.
// Requests arriving while others are on the GPU join at the next admission,
// so their work overlaps on the device with the running ones.  A system's
// arithmetic never depends on its neighbours in the batch (see batch.cu),
// so a result is identical whether it ran alone or in a mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "afsai_batch.cuh"

namespace afsai {
namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct ServeMatrix {
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t *rowptr = nullptr, *col = nullptr;
    double* val = nullptr;
    afsai_precond* M = nullptr;  // built at the first request
    int64_t g_bytes = 0;
    int32_t running = 0;         // right-hand sides of this matrix on the GPU
    bool building = false;       // set-up queued or running on the set-up thread
    double setup_ms = 0.0;       // duration of its last set-up
    std::string setup_error;     // message of a failed set-up
    Clock::time_point last_use;
};

enum ReqState { Q_WAIT = 0, Q_RUN = 1, Q_DONE = 2, Q_FAIL = 3 };

struct ServeRequest {
    int32_t matrix = 0;
    int32_t nrhs = 0;
    double rtol = 1e-8;
    std::vector<double> b, x;  // host, n * nrhs (right-hand side k at offset k n)
    ReqState state = Q_WAIT;
    int32_t remaining = 0;
    std::vector<pcg_info> info;
    Clock::time_point t_submit, t_admit, t_done;
    double setup_ms = 0.0;
    bool triggered_setup = false;  // its arrival started its matrix's set-up
    std::string error;
};

struct Slot {
    bool used = false;
    int64_t ticket = -1;
    int32_t rhs = 0;
    double* vec = nullptr;  // 7 n doubles: b x r p q z t
    int64_t bytes = 0;
};

}  // namespace

struct ServerImpl {
    int device = 0;
    afsai_params params{};
    int32_t maxit = 10000;
    int64_t budget = 0;
    int32_t max_slots = 0;
    int iters_per_step = 4;
    int32_t max_bodies = 16;      // bodies of K iterations per step at most
    cudaStream_t st = nullptr;
    cudaStream_t setup_st = nullptr;
    BatchEngine E;
    std::mutex mu;
    std::condition_variable cv;
    std::condition_variable setup_cv;
    bool stop = false;
    std::thread th;
    std::thread setup_th;
    std::deque<int32_t> setup_queue;
    int32_t* arrival_flag = nullptr;  // mapped pinned host memory, raised by serve_submit
    int32_t* arrival_flag_dev = nullptr;
    std::vector<std::unique_ptr<ServeMatrix>> mats;
    std::map<int64_t, ServeRequest> reqs;
    std::deque<int64_t> queue;
    std::vector<Slot> slots;
    std::vector<BSys> sys;
    int64_t next_ticket = 1;
    int64_t mem_used = 0;
    afsai_status fatal = AFSAI_OK;
    std::string fatal_msg;
    serve_stats stats{};

    int64_t vec_bytes(int32_t n) const { return static_cast<int64_t>(n) * 7 * 8; }
    int64_t g_estimate(const ServeMatrix& m) const {
        const int64_t per_row = 1 + static_cast<int64_t>(params.kiter) * params.s;
        const int64_t w = params.g_prec == 0 ? 8 : (params.g_prec == 1 ? 4 : 2);
        return 2 * (static_cast<int64_t>(m.n) * per_row * (4 + w) + 4 * (m.n + 1L)) + 24L * m.n;
    }

    afsai_status init_engine() {
        AFSAI_TRY(E.reserve(max_slots, static_cast<int64_t>(4) << 20, st));
        E.vtype = params.g_prec;
        sys.assign(max_slots, BSys{});
        std::vector<char> running(max_slots, 0);
        AFSAI_TRY(E.set_tables(sys, running, 0, st));
        AFSAI_CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&arrival_flag), sizeof(int32_t), cudaHostAllocMapped));
        *arrival_flag = 0;
        AFSAI_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&arrival_flag_dev), arrival_flag, 0));
        E.use_act = false;
        AFSAI_TRY(E.capture_loop(iters_per_step, max_bodies, st, true, arrival_flag_dev));
        return AFSAI_OK;
    }

    // The set-up thread: builds the preconditioners of matrices at their
    // first request on its own stream.
    void setup_loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lock(mu);
        while (!stop) {
            if (setup_queue.empty()) {
                setup_cv.wait_for(lock, std::chrono::milliseconds(5));
                continue;
            }
            const int32_t id = setup_queue.front();
            setup_queue.pop_front();
            ServeMatrix& m = *mats[id];
            afsai_csr A{m.n, m.nnz, m.rowptr, m.col, m.val};
            const afsai_params prm = params;
            lock.unlock();
            afsai_precond* M = nullptr;
            const auto t0 = Clock::now();
            const afsai_status s = setup_precond(&A, &prm, setup_st, false, &M);
            const double ms = ms_between(t0, Clock::now());
            const std::string msg = s == AFSAI_OK ? std::string() : std::string(afsai_last_error());
            lock.lock();
            m.building = false;
            if (s == AFSAI_OK) {
                m.M = M;
                m.setup_ms = ms;
            } else {
                // the requests waiting for this matrix fail; its reserved memory is returned
                mem_used -= m.g_bytes;
                m.g_bytes = 0;
                m.setup_error = msg;
                for (auto it = queue.begin(); it != queue.end();) {
                    ServeRequest& R = reqs[*it];
                    if (R.matrix == id) {
                        R.state = Q_FAIL;
                        R.error = "set-up failed: " + msg;
                        R.t_done = Clock::now();
                        it = queue.erase(it);
                    } else {
                        ++it;
                    }
                }
            }
            cv.notify_all();
        }
    }

    // Frees preconditioners of idle matrices, oldest use first, until
    // `need` bytes fit the budget; `keep` (the matrix being admitted) is
    // never a victim.  Caller holds the lock.
    void evict_for(int64_t need, const ServeMatrix* keep) {
        while (mem_used + need > budget) {
            ServeMatrix* victim = nullptr;
            for (auto& m : mats)
                if (m.get() != keep && m->M && m->running == 0 && (!victim || m->last_use < victim->last_use))
                    victim = m.get();
            if (!victim) return;
            cudaStreamSynchronize(st);  // no step in flight reads it any more
            afsai_destroy(victim->M);
            victim->M = nullptr;
            mem_used -= victim->g_bytes;
            victim->g_bytes = 0;
        }
    }

    // Admission (caller holds the lock).  Returns true if tables changed.
    bool admit(afsai_status* err) {
        bool changed = false;
        for (auto it = queue.begin(); it != queue.end();) {
            const int64_t t = *it;
            ServeRequest& R = reqs[t];
            ServeMatrix& m = *mats[R.matrix];
            if (!m.M) {
                // the preconditioner is built on the set-up thread; the
                // request keeps its place and the ones behind it may go first
                if (!m.building) {
                    R.triggered_setup = true;
                    const int64_t need_g = g_estimate(m);
                    if (mem_used + need_g > budget) evict_for(need_g, &m);
                    if (mem_used + need_g > budget) break;
                    m.building = true;
                    m.g_bytes = need_g;
                    mem_used += need_g;
                    setup_queue.push_back(R.matrix);
                    setup_cv.notify_all();
                }
                ++it;
                continue;
            }
            int32_t free_slots = 0;
            for (const Slot& s : slots) free_slots += s.used ? 0 : 1;
            if (free_slots < R.nrhs) break;
            const int64_t need = vec_bytes(m.n) * R.nrhs;
            if (mem_used + need > budget) evict_for(need, &m);
            if (mem_used + need > budget) break;
            it = queue.erase(it);
            R.t_admit = Clock::now();
            if (R.triggered_setup) R.setup_ms = m.setup_ms;
            m.last_use = Clock::now();
            R.state = Q_RUN;
            R.remaining = R.nrhs;
            R.info.assign(R.nrhs, pcg_info{});
            for (int32_t k = 0; k < R.nrhs; ++k) {
                int32_t slot = 0;
                while (slots[slot].used) ++slot;
                Slot& S = slots[slot];
                const int64_t bytes = vec_bytes(m.n);
                if (lib_malloc_async(reinterpret_cast<void**>(&S.vec), bytes, st) != cudaSuccess) {
                    *err = fail(AFSAI_ENOMEM, "vectors of a served system");
                    return changed;
                }
                mem_used += bytes;
                S.used = true;
                S.ticket = t;
                S.rhs = k;
                S.bytes = bytes;
                const size_t n = m.n;
                cudaMemcpyAsync(S.vec, R.b.data() + k * n, sizeof(double) * n, cudaMemcpyHostToDevice, st);
                cudaMemsetAsync(S.vec + n, 0, sizeof(double) * n, st);  // x0 = 0
                BSys& y = sys[slot];
                y = BSys{};
                y.n = m.n;
                y.Arp = m.rowptr;
                y.Acol = m.col;
                y.Aval = m.val;
                y.Grp = m.M->G.rowptr;
                y.Gcol = m.M->G.col;
                y.Gval = m.M->G.val;
                y.Trp = m.M->Gt.rowptr;
                y.Tcol = m.M->Gt.col;
                y.Tval = m.M->Gt.val;
                y.b = S.vec;
                y.x = S.vec + n;
                y.r = S.vec + 2 * n;
                y.p = S.vec + 3 * n;
                y.q = S.vec + 4 * n;
                y.z = S.vec + 5 * n;
                y.t = S.vec + 6 * n;
                BScal sc{};
                sc.rtol = R.rtol;
                sc.maxit = maxit;
                sc.fresh = 1;
                if (E.set_scalars(slot, sc, st) != AFSAI_OK) {
                    *err = AFSAI_ECUDA;
                    return changed;
                }
                ++m.running;
            }
            changed = true;
        }
        return changed;
    }

    afsai_status push_tables() {
        std::vector<char> running(max_slots, 0);
        int32_t nrun = 0;
        for (int32_t s = 0; s < max_slots; ++s)
            if (slots[s].used) {
                running[s] = 1;
                ++nrun;
            }
        return E.set_tables(sys, running, nrun, st);
    }

    // Reads the scalars; retires finished systems.  Caller holds the lock.
    afsai_status retire(bool* changed) {
        std::vector<BScal> sc(max_slots);
        AFSAI_CUDA_TRY(cudaMemcpyAsync(sc.data(), E.d_sc, sizeof(BScal) * max_slots, cudaMemcpyDeviceToHost, st));
        AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
        bool any = false;
        for (int32_t s = 0; s < max_slots; ++s)
            if (slots[s].used && sc[s].done != 0 && !sc[s].fresh) any = true;
        if (!any) return AFSAI_OK;
        AFSAI_TRY(E.finish(st, 1));
        AFSAI_CUDA_TRY(cudaMemcpyAsync(sc.data(), E.d_sc, sizeof(BScal) * max_slots, cudaMemcpyDeviceToHost, st));
        AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
        for (int32_t s = 0; s < max_slots; ++s) {
            Slot& S = slots[s];
            if (!S.used || sc[s].done == 0 || sc[s].fresh) continue;
            ServeRequest& R = reqs[S.ticket];
            ServeMatrix& m = *mats[R.matrix];
            const size_t n = m.n;
            cudaMemcpyAsync(R.x.data() + S.rhs * n, S.vec + n, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
            const double bn = std::sqrt(sc[s].bb);
            pcg_info& inf = R.info[S.rhs];
            inf.iters = sc[s].iters;
            inf.converged = sc[s].done == 1 ? 1 : 0;
            inf.relres_rec = bn > 0 ? std::sqrt(sc[s].rr) / bn : 0.0;
            inf.relres_true = bn > 0 ? std::sqrt(sc[s].true_rr) / bn : 0.0;
            cudaFreeAsync(S.vec, st);
            mem_used -= S.bytes;
            S = Slot{};
            sys[s] = BSys{};
            --m.running;
            m.last_use = Clock::now();
            stats.solves += 1;
            if (--R.remaining == 0) {
                R.state = Q_DONE;
                R.t_done = Clock::now();
                stats.requests_done += 1;
            }
            *changed = true;
        }
        AFSAI_CUDA_TRY(cudaStreamSynchronize(st));  // x copies landed before anyone polls
        cv.notify_all();
        return AFSAI_OK;
    }

    void loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lock(mu);
        while (!stop) {
            afsai_status err = AFSAI_OK;
            bool changed = admit(&err);
            if (err == AFSAI_OK && changed) {
                err = push_tables();
                if (err == AFSAI_OK) err = E.start(st);
            }
            int32_t nrun = 0;
            for (const Slot& s : slots) nrun += s.used ? 1 : 0;
            if (err == AFSAI_OK && nrun == 0) {
                cv.wait_for(lock, std::chrono::milliseconds(2));
                continue;
            }
            if (err == AFSAI_OK) {
                // requests queued from here on raise the flag again and end this step
                *reinterpret_cast<volatile int32_t*>(arrival_flag) = 0;
                err = E.arm_loop(st);
                if (err == AFSAI_OK) err = E.launch_graph(st);
                stats.steps += 1;
            }
            // the lock is released while the GPU works, so callers can submit
            if (err == AFSAI_OK) {
                lock.unlock();
                const cudaError_t e = cudaStreamSynchronize(st);
                lock.lock();
                if (e != cudaSuccess) err = fail(AFSAI_ECUDA, cudaGetErrorString(e));
            }
            bool ch = false;
            if (err == AFSAI_OK) err = retire(&ch);
            if (err == AFSAI_OK && ch) err = push_tables();
            if (err != AFSAI_OK) {
                fatal = err;
                fatal_msg = afsai_last_error();
                for (auto& kv : reqs)
                    if (kv.second.state == Q_WAIT || kv.second.state == Q_RUN) {
                        kv.second.state = Q_FAIL;
                        kv.second.error = fatal_msg;
                    }
                cv.notify_all();
                break;
            }
            stats.peak_mem_bytes = std::max<int64_t>(stats.peak_mem_bytes, mem_used);
        }
    }
};

}  // namespace afsai

using namespace afsai;

struct afsai_server {
    ServerImpl impl;
};

extern "C" {

afsai_status serve_create(size_t mem_budget_bytes, int32_t max_slots, const afsai_params* params, int32_t maxit,
                          int32_t iters_per_step, afsai_server** out) {
    if (!out || !params || max_slots <= 0 || mem_budget_bytes == 0 || maxit <= 0)
        return fail(AFSAI_EINVAL, "invalid server arguments");
    *out = nullptr;
    AFSAI_TRY(check_params(params));
    if (params->block_rows != 0) return fail(AFSAI_ENOTSUP, "the locality bound applies to single-system set-ups");
    auto* S = new (std::nothrow) afsai_server();
    if (!S) return fail(AFSAI_ENOMEM, "host allocation");
    ServerImpl& I = S->impl;
    cudaGetDevice(&I.device);
    I.params = *params;
    I.maxit = maxit;
    I.budget = static_cast<int64_t>(mem_budget_bytes);
    I.max_slots = max_slots;
    I.iters_per_step = iters_per_step > 0 ? iters_per_step : 4;
    I.slots.assign(max_slots, Slot{});
    if (cudaStreamCreateWithFlags(&I.st, cudaStreamNonBlocking) != cudaSuccess) {
        delete S;
        return fail(AFSAI_ECUDA, "cudaStreamCreate");
    }
    if (cudaStreamCreateWithFlags(&I.setup_st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaStreamDestroy(I.st);
        delete S;
        return fail(AFSAI_ECUDA, "cudaStreamCreate");
    }
    const afsai_status s = I.init_engine();
    if (s != AFSAI_OK) {
        I.E.release(I.st);
        if (I.arrival_flag) cudaFreeHost(I.arrival_flag);
        cudaStreamDestroy(I.st);
        cudaStreamDestroy(I.setup_st);
        delete S;
        return s;
    }
    I.th = std::thread([&I] { I.loop(); });
    I.setup_th = std::thread([&I] { I.setup_loop(); });
    *out = S;
    return AFSAI_OK;
}

afsai_status serve_register(afsai_server* S, const afsai_csr* A, int32_t* matrix_id) {
    if (!S || !A || !matrix_id || !A->rowptr || !A->col || !A->val || A->n <= 0) return fail(AFSAI_EINVAL, "invalid matrix");
    ServerImpl& I = S->impl;
    auto m = std::make_unique<ServeMatrix>();
    m->n = A->n;
    m->nnz = A->nnz;
    const int64_t bytes = 4 * (A->n + 1L) + 12 * A->nnz;
    std::lock_guard<std::mutex> lock(I.mu);
    if (I.mem_used + bytes > I.budget) return fail(AFSAI_EBUSY, "matrix does not fit the memory budget");
    // the server stream is busy with the step loop; copies use their own stream
    cudaStream_t cs;
    AFSAI_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    afsai_status st = AFSAI_OK;
    if (lib_malloc_async(reinterpret_cast<void**>(&m->rowptr), 4 * (A->n + 1L), cs) != cudaSuccess ||
        lib_malloc_async(reinterpret_cast<void**>(&m->col), 4 * A->nnz, cs) != cudaSuccess ||
        lib_malloc_async(reinterpret_cast<void**>(&m->val), 8 * A->nnz, cs) != cudaSuccess)
        st = fail(AFSAI_ENOMEM, "matrix copy");
    if (st == AFSAI_OK &&
        (cudaMemcpyAsync(m->rowptr, A->rowptr, 4 * (A->n + 1L), cudaMemcpyDefault, cs) != cudaSuccess ||
         cudaMemcpyAsync(m->col, A->col, 4 * A->nnz, cudaMemcpyDefault, cs) != cudaSuccess ||
         cudaMemcpyAsync(m->val, A->val, 8 * A->nnz, cudaMemcpyDefault, cs) != cudaSuccess ||
         cudaStreamSynchronize(cs) != cudaSuccess))
        st = fail(AFSAI_ECUDA, "matrix copy");
    cudaStreamDestroy(cs);
    if (st != AFSAI_OK) return st;
    I.mem_used += bytes;
    m->last_use = Clock::now();
    *matrix_id = static_cast<int32_t>(I.mats.size());
    I.mats.push_back(std::move(m));
    return AFSAI_OK;
}

afsai_status serve_submit(afsai_server* S, int32_t matrix_id, const double* b, int32_t nrhs, double rtol,
                          int64_t* ticket) {
    if (!S || !b || !ticket || nrhs <= 0 || !(rtol > 0.0)) return fail(AFSAI_EINVAL, "invalid request");
    ServerImpl& I = S->impl;
    std::lock_guard<std::mutex> lock(I.mu);
    if (I.fatal != AFSAI_OK) return fail(I.fatal, "server stopped: " + I.fatal_msg);
    if (matrix_id < 0 || matrix_id >= static_cast<int32_t>(I.mats.size())) return fail(AFSAI_EINVAL, "unknown matrix");
    if (nrhs > I.max_slots) return fail(AFSAI_EINVAL, "more right-hand sides than server slots");
    const ServeMatrix& m = *I.mats[matrix_id];
    const int64_t t = I.next_ticket++;
    ServeRequest& R = I.reqs[t];
    R.matrix = matrix_id;
    R.nrhs = nrhs;
    R.rtol = rtol;
    R.b.assign(b, b + static_cast<size_t>(m.n) * nrhs);
    R.x.assign(static_cast<size_t>(m.n) * nrhs, 0.0);
    R.t_submit = Clock::now();
    I.queue.push_back(t);
    I.stats.requests_submitted += 1;
    if (I.arrival_flag) *reinterpret_cast<volatile int32_t*>(I.arrival_flag) = 1;  // ends the running step
    I.cv.notify_all();
    *ticket = t;
    return AFSAI_OK;
}

afsai_status serve_poll(afsai_server* S, int64_t ticket, double* x, pcg_info* info, serve_result* res) {
    if (!S) return fail(AFSAI_EINVAL, "NULL server");
    ServerImpl& I = S->impl;
    std::lock_guard<std::mutex> lock(I.mu);
    auto it = I.reqs.find(ticket);
    if (it == I.reqs.end()) return fail(AFSAI_EINVAL, "unknown ticket");
    ServeRequest& R = it->second;
    if (R.state == Q_WAIT || R.state == Q_RUN) return AFSAI_EAGAIN;
    if (R.state == Q_FAIL) {
        const std::string e = R.error;
        I.reqs.erase(it);
        return fail(AFSAI_ECUDA, "request failed: " + e);
    }
    if (x) std::memcpy(x, R.x.data(), sizeof(double) * R.x.size());
    if (info) std::memcpy(info, R.info.data(), sizeof(pcg_info) * R.info.size());
    if (res) {
        res->nrhs = R.nrhs;
        res->max_iters = 0;
        res->converged = 1;
        res->max_relres_true = 0.0;
        for (const pcg_info& f : R.info) {
            res->max_iters = std::max(res->max_iters, f.iters);
            res->converged &= f.converged;
            res->max_relres_true = std::max(res->max_relres_true, f.relres_true);
        }
        res->queue_ms = ms_between(R.t_submit, R.t_admit);
        res->setup_ms = R.setup_ms;
        res->latency_ms = ms_between(R.t_submit, R.t_done);
    }
    const bool conv = !res || res->converged;
    I.reqs.erase(it);
    return conv ? AFSAI_OK : fail(AFSAI_ENOCONV, "a right-hand side reached maxit");
}

afsai_status serve_get_stats(afsai_server* S, serve_stats* out) {
    if (!S || !out) return fail(AFSAI_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(S->impl.mu);
    *out = S->impl.stats;
    out->mem_used_bytes = S->impl.mem_used;
    out->queued = static_cast<int64_t>(S->impl.queue.size());
    int64_t run = 0;
    for (const auto& s : S->impl.slots) run += s.used ? 1 : 0;
    out->running = run;
    return AFSAI_OK;
}

void serve_destroy(afsai_server* S) {
    if (!S) return;
    ServerImpl& I = S->impl;
    {
        std::lock_guard<std::mutex> lock(I.mu);
        I.stop = true;
    }
    I.cv.notify_all();
    I.setup_cv.notify_all();
    if (I.th.joinable()) I.th.join();
    if (I.setup_th.joinable()) I.setup_th.join();
    cudaSetDevice(I.device);
    cudaStreamSynchronize(I.setup_st);
    cudaStreamSynchronize(I.st);
    for (auto& s : I.slots)
        if (s.vec) cudaFreeAsync(s.vec, I.st);
    for (auto& m : I.mats) {
        if (m->M) afsai_destroy(m->M);
        if (m->rowptr) cudaFreeAsync(m->rowptr, I.st);
        if (m->col) cudaFreeAsync(m->col, I.st);
        if (m->val) cudaFreeAsync(m->val, I.st);
    }
    I.E.release(I.st);
    cudaStreamSynchronize(I.st);
    if (I.arrival_flag) cudaFreeHost(I.arrival_flag);
    cudaStreamDestroy(I.st);
    cudaStreamDestroy(I.setup_st);
    delete S;
}

}  // extern "C"
