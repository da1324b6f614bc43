// Serving GP posterior means with continuous batching.
//
// A request is one solve Ktilde v = y (Alg. 2 with the pivoted-Cholesky
// preconditioner of Eq. woodbury) followed by the predictive mean
// mu* = K(X*, X) v (Sec. 2.1).  The server keeps every admitted request's
// inputs, preconditioner and CG state resident in one pre-allocated device
// arena and runs the requests as independent per-slot streams:
//
//   engine thread:  admit (FIFO, free slot + first-fit arena block)
//                   -> for every slot whose last phase has completed
//                      (cudaEventQuery), enqueue its next phase
//
// A phase is a short run of kernels ending with a 4-byte copy of the solver's
// active-column count and an event record, so the engine never blocks on the
// device and the phases of all admitted requests overlap on the GPU: a small
// request's kernels run beside a large one's, and a request that arrives while
// others are in flight starts as soon as a slot and its footprint are free.
//
// Each request's arithmetic is fixed by its own shapes (launch plans depend on
// N, d and the SM count only), so its result does not depend on the mix.
#include "gpk_internal.cuh"

#include <math.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

namespace gpk {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, cap) in 256-byte units of alignment.
class Arena {
  public:
    explicit Arena(size_t cap) : cap_(cap) { free_[0] = cap; }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, start = it->first + bytes;
            free_.erase(it);
            if (rest) free_[start] = rest;
            used_ += bytes;
            if (used_ > peak_) peak_ = used_;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    size_t cap_, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

struct Request {
    uint64_t id = 0;
    gp_hyp_t hyp{};
    std::vector<float> ls;
    const float *X = nullptr, *y = nullptr, *Xs = nullptr;
    float* mean_out = nullptr;
    bool out_pinned = false;   // page-locked: the mean is copied asynchronously
    int64_t N = 0, n_test = 0;
    size_t bytes = 0;
    // result
    bool done = false;
    gp_request_stats_t st{};
};

enum Phase { IDLE, SOLVING, FINAL };

struct Slot {
    Ctx ctx;                 // per-slot error word, pinned scratch, launch counter
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    Phase phase = IDLE;
    std::shared_ptr<Request> req;
    size_t off = 0;
    CgSolver cg;
    KOp mop;
    // device views into the request's arena block
    float *X = nullptr, *y = nullptr, *v = nullptr, *Xs = nullptr, *mean = nullptr, *L = nullptr;
    int32_t* piv = nullptr;
    double* core = nullptr;
    uint8_t* scratch = nullptr;
    size_t scratch_bytes = 0;
    int* host_flag = nullptr;       // inside ctx.host_pinned
    int* host_err = nullptr;
    ColState* host_state = nullptr;
};

// Persistent part of a request's block, in carve order; the phase scratch
// (preconditioner, then CG, then the predictive-mean operator, which never
// overlap in time on the slot's stream) follows it.
template <class A>
void persistent_layout(A& a, int64_t N, int d, int64_t n_test, int rank) {
    a.template take<float>((size_t)N * d);       // X
    a.template take<float>((size_t)N);           // y
    a.template take<float>((size_t)N);           // v
    a.template take<float>((size_t)n_test * d);  // X*
    a.template take<float>((size_t)n_test);      // mu*
    if (rank > 0) {
        a.template take<float>((size_t)N * rank);            // L
        a.template take<int32_t>((size_t)rank);              // pivots
        a.template take<double>((size_t)rank * rank);        // Woodbury core factor
    }
}

gp_cg_opts_t cg_opts_of(const gp_server_opts_t& o) {
    gp_cg_opts_t c{};
    c.tol = o.tol;
    c.max_iter = o.max_iter;
    c.min_iter = 0;
    c.precision = o.precision;
    c.algorithm = GP_CG_STABLE;
    c.reorth = o.reorth;
    c.reorth_passes = 1;
    c.x0_given = 0;
    c.restarts = o.restarts;
    c.check_precision = GP_PREC_FP32;
    c.escalate = 1;
    c.refine_precision = o.refine_precision;
    c.refine_resid = o.refine_resid;
    return c;
}

int check_opts(const gp_server_opts_t* o) {
    if (!o || o->arena_bytes == 0 || o->max_slots < 1 || o->max_slots > 64) return GP_ERR_INVALID;
    if (o->rank < 0 || o->rank > 512 || !(o->tol >= 0.0) || o->max_iter < 1 || o->max_iter > 1000) return GP_ERR_INVALID;
    if (o->restarts < 0 || o->restarts > 16) return GP_ERR_INVALID;
    if (o->large_reserve < 0 || o->large_n < 0) return GP_ERR_INVALID;
    if (o->reorth < GP_REORTH_NONE || o->reorth > GP_REORTH_EUCLID) return GP_ERR_INVALID;
    GPK_TRY(check_mvm_flags(o->precision, false));
    GPK_TRY(check_mvm_flags(o->mean_precision, false));
    if (o->refine_precision != 0) {
        GPK_TRY(check_mvm_flags(o->refine_precision, false));
        if (!(o->refine_resid >= 0.0) || (o->refine_resid == 0.0 && o->restarts < 1)) return GP_ERR_INVALID;
    }
    return GP_OK;
}

// SMs a request's kernels are planned for (its own N decides, not the mix).
int request_sms(const gp_server_opts_t& o, int64_t N, int num_sms) {
    if (o.large_reserve > 0 && N >= o.large_n && o.large_reserve < num_sms) return num_sms - o.large_reserve;
    return num_sms;
}

// Footprint: persistent part + the largest phase scratch; 0 if not servable.
size_t request_bytes(const Ctx* ctx, const gp_server_opts_t& o, const gp_hyp_t* hyp, int64_t N, int64_t n_test,
                     size_t* scratch_out) {
    if (check_hyp(hyp) != GP_OK || N < 1 || n_test < 1 || !(hyp->noise > 0.0)) return 0;
    const int rank = o.rank < N ? o.rank : (int)N;
    WsCounter c;
    persistent_layout(c, N, hyp->d, n_test, rank);
    const gp_cg_opts_t co = cg_opts_of(o);
    const size_t cg = cg_workspace(ctx, hyp, N, 1, rank, &co);
    const size_t pcw = rank > 0 ? pivchol_workspace(ctx, N, hyp->d, rank) : 0;
    const size_t mw = kop_workspace(ctx, hyp, n_test, N, 1, o.mean_precision, false);
    if (cg == 0 || mw == 0) return 0;
    size_t sc = cg > pcw ? cg : pcw;
    sc = sc > mw ? sc : mw;
    sc = (sc + 255) & ~size_t(255);
    if (scratch_out) *scratch_out = sc;
    return c.off + sc;
}

}  // namespace

struct Server {
    int device = 0;
    int num_sms = 0;
    gp_server_opts_t o{};
    uint8_t* arena_base = nullptr;
    std::unique_ptr<Arena> arena;
    int* dev_err = nullptr;            // one 256-byte error word per slot
    std::vector<std::unique_ptr<Slot>> slots;
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread engine;
    // statistics (under mu)
    uint64_t submitted = 0, completed = 0;
    size_t peak = 0, in_use = 0;
    int inflight = 0, max_inflight = 0;
    std::atomic<int64_t> launches{0};

    double ms_now() const {
        return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    }

    int admit(Slot& sl, std::shared_ptr<Request> r, size_t off);
    int advance(Slot& sl);
    void complete(Slot& sl, int status);
    void run();
};

int Server::admit(Slot& sl, std::shared_ptr<Request> r, size_t off) {
    sl.req = r;
    sl.off = off;
    sl.phase = SOLVING;
    sl.ctx.num_sms = request_sms(o, r->N, num_sms);
    const int64_t N = r->N;
    const int d = r->hyp.d;
    const int rank = o.rank < N ? o.rank : (int)N;
    WsCarver wc(arena_base + off, r->bytes);
    sl.X = wc.take<float>((size_t)N * d);
    sl.y = wc.take<float>((size_t)N);
    sl.v = wc.take<float>((size_t)N);
    sl.Xs = wc.take<float>((size_t)r->n_test * d);
    sl.mean = wc.take<float>((size_t)r->n_test);
    sl.L = nullptr;
    sl.piv = nullptr;
    sl.core = nullptr;
    if (rank > 0) {
        sl.L = wc.take<float>((size_t)N * rank);
        sl.piv = wc.take<int32_t>((size_t)rank);
        sl.core = wc.take<double>((size_t)rank * rank);
    }
    if (!wc.ok) return GP_ERR_WORKSPACE;
    sl.scratch = wc.base + wc.off;
    sl.scratch_bytes = wc.cap - wc.off;
    cudaStream_t s = sl.s;
    GPK_CUDA_TRY(cudaMemsetAsync(sl.ctx.dev_err, 0, sizeof(int), s));
    GPK_CUDA_TRY(cudaMemcpyAsync(sl.X, r->X, sizeof(float) * (size_t)N * d, cudaMemcpyHostToDevice, s));
    GPK_CUDA_TRY(cudaMemcpyAsync(sl.y, r->y, sizeof(float) * (size_t)N, cudaMemcpyHostToDevice, s));
    GPK_CUDA_TRY(cudaMemcpyAsync(sl.Xs, r->Xs, sizeof(float) * (size_t)r->n_test * d, cudaMemcpyHostToDevice, s));
    gp_precond_t pc{sl.L, sl.core, rank};
    if (rank > 0) {
        WsCarver w1(sl.scratch, sl.scratch_bytes);
        GPK_TRY(pivchol_run(&sl.ctx, w1, &r->hyp, sl.X, N, rank, sl.L, sl.piv, sl.core, nullptr, s));
    }
    const gp_cg_opts_t co = cg_opts_of(o);
    WsCarver w2(sl.scratch, sl.scratch_bytes);
    sl.cg = CgSolver();
    return sl.cg.setup(&sl.ctx, w2, &r->hyp, sl.X, N, sl.y, 1, sl.v, rank > 0 ? &pc : nullptr, &co, s, sl.host_flag,
                       sl.ev);
}

int Server::advance(Slot& sl) {
    if (sl.phase == SOLVING) {
        bool done = false;
        GPK_TRY(sl.cg.step(&done));
        if (!done) return GP_OK;
        // solve finished: copy its state back, then the predictive mean (its
        // operator reuses the solver's scratch; the stream orders the two)
        Request& r = *sl.req;
        GPK_TRY(sl.cg.enqueue_state(sl.host_state));
        GPK_CUDA_TRY(cudaMemcpyAsync(sl.host_err, sl.ctx.dev_err, sizeof(int), cudaMemcpyDeviceToHost, sl.s));
        WsCarver w3(sl.scratch, sl.scratch_bytes);
        sl.mop = KOp();
        GPK_TRY(kop_prepare(&sl.ctx, w3, sl.mop, &r.hyp, sl.Xs, r.n_test, sl.X, r.N, 1, o.mean_precision, sl.s));
        GPK_TRY(kop_apply(&sl.ctx, sl.mop, sl.v, 1, sl.mean, r.n_test, false, sl.s));
        if (r.out_pinned)
            GPK_CUDA_TRY(cudaMemcpyAsync(r.mean_out, sl.mean, sizeof(float) * (size_t)r.n_test,
                                         cudaMemcpyDeviceToHost, sl.s));
        GPK_CUDA_TRY(cudaEventRecord(sl.ev, sl.s));
        sl.phase = FINAL;
        return GP_OK;
    }
    // FINAL: everything of this request has completed.  A pageable output
    // buffer is filled now (a short copy of finished data) rather than by an
    // asynchronous copy, which would stall this thread until the stream drains.
    if (!sl.req->out_pinned &&
        cudaMemcpy(sl.req->mean_out, sl.mean, sizeof(float) * (size_t)sl.req->n_test, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return GP_ERR_CUDA;
    gp_cg_stats_t cs{};
    int status = sl.cg.summarize(sl.host_state, &cs);
    const int e = *sl.host_err;
    if (e == DEV_TIMEOUT) status = GP_ERR_TIMEOUT;
    else if (e == DEV_NONFINITE) status = GP_ERR_NONFINITE;
    else if (e != DEV_OK) status = GP_ERR_CUDA;
    Request& r = *sl.req;
    r.st.iters = cs.iters;
    r.st.restarts = cs.restarts;
    r.st.rel_resid = sl.host_state[0].relres;
    complete(sl, status);
    return GP_OK;
}

void Server::complete(Slot& sl, int status) {
    if (status != GP_OK && status != GP_ERR_NOT_CONVERGED && status != GP_ERR_BREAKDOWN) {
        // a failed phase may have left work on the stream: drain it before the
        // block can be handed to another request
        cudaStreamSynchronize(sl.s);
        cudaGetLastError();
    }
    launches += sl.ctx.launches;
    sl.ctx.launches = 0;
    std::shared_ptr<Request> r = sl.req;
    sl.req.reset();
    sl.phase = IDLE;
    std::lock_guard<std::mutex> lk(mu);
    arena->release(sl.off, r->bytes);
    in_use = arena->used();
    --inflight;
    r->st.status = status;
    r->st.t_done_ms = ms_now();
    r->done = true;
    ++completed;
    cv_done.notify_all();
}

void Server::run() {
    cudaSetDevice(device);
    for (;;) {
        bool progressed = false;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (inflight == 0 && pending.empty()) {
                if (stop) break;
                cv_work.wait(lk, [&] { return stop || !pending.empty(); });
                if (stop && pending.empty()) break;
            }
        }
        // admission: strict arrival order; the head waits for a slot and memory
        for (;;) {
            Slot* free_slot = nullptr;
            for (auto& p : slots)
                if (p->phase == IDLE) { free_slot = p.get(); break; }
            if (!free_slot) break;
            std::shared_ptr<Request> r;
            size_t off = 0;
            {
                std::lock_guard<std::mutex> lk(mu);
                if (pending.empty()) break;
                if (!arena->alloc(pending.front()->bytes, &off)) break;
                r = pending.front();
                pending.pop_front();
                in_use = arena->used();
                peak = arena->peak();
                ++inflight;
                if (inflight > max_inflight) max_inflight = inflight;
                r->st.t_admit_ms = ms_now();
            }
            const int st = admit(*free_slot, r, off);
            if (st != GP_OK) complete(*free_slot, st);
            progressed = true;
        }
        for (auto& p : slots) {
            Slot& sl = *p;
            if (sl.phase == IDLE) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            progressed = true;
            const int st = q == cudaSuccess ? advance(sl) : GP_ERR_CUDA;
            if (st != GP_OK) complete(sl, st);
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
}

}  // namespace gpk

struct gp_server : public gpk::Server {};

extern "C" {

size_t gp_server_request_bytes(const gp_server_opts_t* opts, const gp_hyp_t* hyp, int64_t N, int64_t n_test) {
    if (gpk::check_opts(opts) != GP_OK) return 0;
    gpk::Ctx probe;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&probe.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) probe.num_sms = 148;
    probe.num_sms = gpk::request_sms(*opts, N, probe.num_sms);
    return gpk::request_bytes(&probe, *opts, hyp, N, n_test, nullptr);
}

void gp_server_destroy(gp_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->engine.joinable()) srv->engine.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->device);
    for (auto& p : srv->slots) {
        if (p->s) cudaStreamSynchronize(p->s);
        if (p->ev) cudaEventDestroy(p->ev);
        if (p->s) cudaStreamDestroy(p->s);
        if (p->ctx.host_pinned) cudaFreeHost(p->ctx.host_pinned);
    }
    if (srv->dev_err) cudaFree(srv->dev_err);
    if (srv->arena_base) cudaFree(srv->arena_base);
    cudaSetDevice(prev);
    delete srv;
}

int gp_server_create(int device, const gp_server_opts_t* opts, gp_server** out) {
    if (!out) return GP_ERR_INVALID;
    *out = nullptr;
    GPK_TRY(gpk::check_opts(opts));
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return GP_ERR_INVALID;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return GP_ERR_CUDA;
    gp_server* srv = new (std::nothrow) gp_server();
    if (!srv) return GP_ERR_OOM;
    srv->device = device;
    srv->o = *opts;
    srv->t0 = gpk::Clock::now();
    int st = GP_OK;
    if (cudaDeviceGetAttribute(&srv->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) st = GP_ERR_CUDA;
    if (st == GP_OK && cudaMalloc((void**)&srv->arena_base, opts->arena_bytes) != cudaSuccess) {
        srv->arena_base = nullptr;
        st = GP_ERR_OOM;
    }
    if (st == GP_OK && (cudaMalloc((void**)&srv->dev_err, 256 * (size_t)opts->max_slots) != cudaSuccess ||
                        cudaMemset(srv->dev_err, 0, 256 * (size_t)opts->max_slots) != cudaSuccess))
        st = GP_ERR_OOM;
    if (st == GP_OK) srv->arena.reset(new gpk::Arena(opts->arena_bytes));
    for (int i = 0; st == GP_OK && i < opts->max_slots; ++i) {
        std::unique_ptr<gpk::Slot> sl(new (std::nothrow) gpk::Slot());
        if (!sl) { st = GP_ERR_OOM; break; }
        sl->ctx.device = device;
        sl->ctx.num_sms = srv->num_sms;
        sl->ctx.dev_err = srv->dev_err + 64 * i;
        if (cudaMallocHost((void**)&sl->ctx.host_pinned, 4096) != cudaSuccess) {
            sl->ctx.host_pinned = nullptr;
            st = GP_ERR_OOM;
        }
        if (st == GP_OK && (cudaStreamCreateWithFlags(&sl->s, cudaStreamNonBlocking) != cudaSuccess ||
                            cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming) != cudaSuccess))
            st = GP_ERR_CUDA;
        if (sl->ctx.host_pinned) {
            // pinned scratch: [0] active-column flag, [1] device error word, [16..) column state
            sl->host_flag = sl->ctx.host_pinned;
            sl->host_err = sl->ctx.host_pinned + 8;   // [0, 4): the solver's flag words
            sl->host_state = (gpk::ColState*)(sl->ctx.host_pinned + 16);
        }
        srv->slots.push_back(std::move(sl));
    }
    if (st == GP_OK) {
        try {
            srv->engine = std::thread([srv] { srv->run(); });
        } catch (...) {
            st = GP_ERR_OOM;
        }
    }
    cudaSetDevice(prev);
    if (st != GP_OK) {
        gp_server_destroy(srv);
        return st;
    }
    *out = srv;
    return GP_OK;
}

int gp_server_submit(gp_server* srv, const gp_hyp_t* hyp, const float* X, int64_t N, const float* y,
                     const float* X_test, int64_t n_test, float* mean_out, uint64_t* id_out) {
    if (!srv || !hyp || !X || !y || !X_test || !mean_out || !id_out) return GP_ERR_INVALID;
    GPK_TRY(gpk::check_hyp(hyp));
    auto r = std::make_shared<gpk::Request>();
    r->ls.assign(hyp->lengthscale, hyp->lengthscale + hyp->d);
    r->hyp = *hyp;
    r->hyp.lengthscale = r->ls.data();
    r->X = X;
    r->y = y;
    r->Xs = X_test;
    r->mean_out = mean_out;
    r->N = N;
    r->n_test = n_test;
    cudaPointerAttributes pa{};
    r->out_pinned = cudaPointerGetAttributes(&pa, mean_out) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    cudaGetLastError();
    gpk::Ctx probe;
    probe.num_sms = gpk::request_sms(srv->o, N, srv->num_sms);
    r->bytes = gpk::request_bytes(&probe, srv->o, &r->hyp, N, n_test, nullptr);
    if (r->bytes == 0) return GP_ERR_INVALID;
    if (((r->bytes + 255) & ~size_t(255)) > srv->o.arena_bytes) return GP_ERR_WORKSPACE;
    r->st.bytes = r->bytes;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return GP_ERR_INVALID;
        r->id = srv->next_id++;
        r->st.t_submit_ms = srv->ms_now();
        srv->reqs[r->id] = r;
        srv->pending.push_back(r);
        ++srv->submitted;
        *id_out = r->id;
    }
    srv->cv_work.notify_all();
    return GP_OK;
}

int gp_server_wait(gp_server* srv, uint64_t id, double timeout_s, gp_request_stats_t* stats) {
    if (!srv) return GP_ERR_INVALID;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return GP_ERR_INVALID;
    std::shared_ptr<gpk::Request> r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_s < 0) {
        srv->cv_done.wait(lk, pred);
    } else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        return GP_ERR_TIMEOUT;
    }
    srv->reqs.erase(id);
    if (stats) *stats = r->st;
    return r->st.status;
}

int gp_server_stats(gp_server* srv, gp_server_stats_t* out) {
    if (!srv || !out) return GP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    out->submitted = srv->submitted;
    out->completed = srv->completed;
    out->arena_bytes = srv->o.arena_bytes;
    out->peak_bytes = srv->peak;
    out->in_use_bytes = srv->in_use;
    out->max_inflight = srv->max_inflight;
    out->launches = srv->launches.load();
    return GP_OK;
}

}  // extern "C"
