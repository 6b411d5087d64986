// Serving loop with continuous batching over independent s-step GMRES solves.
//
// Requests (a CSR matrix, b, x0 and options; sizes and options may differ)
// are queued on submit.  A worker thread repeats:
//   1. admission: in arrival order, while the next request's device footprint
//      (gmres_footprint: basis (m+1) n, CSR, workspace) fits the free memory
//      budget and a slot is free, create its context in that slot and enqueue
//      its first convergence check;
//   2. a pass over the active requests that polls each one's stream: a request
//      whose check has completed is decided at once and, if it goes on, gets
//      its next restart cycle and the check after it enqueued back to back, so
//      no request waits for another's cycle (the GPU overlaps their kernels);
//   3. finished requests copy x out, return their memory and slot, and record
//      their latency (submit to completion).
// A request admitted while others are running joins them at once.  Every
// request keeps its Krylov basis, Hessenberg and Givens state resident on the
// device until it finishes.  Nothing on the worker's path allocates or frees
// with a device-wide synchronization: the slots (stream, capture stream,
// page-locked state mirror) are created with the server, and each context's
// device buffers come from the server's stream-ordered memory pool, reserved
// at start.  Each solve runs the same kernels with the same reduction order as
// a lone gmres_solve, so its result does not depend on what else is served.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <vector>
#include "solver_run.cuh"

namespace gm {
namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

struct Request {
    int64_t id = 0;
    int64_t n = 0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> colind;
    std::vector<double> vals, b, x;
    gmres_opts opts{};
    size_t bytes = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    cudaStream_t stream = nullptr;
    int slot = -1;
    gmres_ctx* ctx = nullptr;
    SolveRun run;
    gmres_result res{};
    int status = 0;
    bool done = false;
};

}  // namespace
}  // namespace gm

using namespace gm;

struct gmres_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::vector<Request*> active;
    std::map<int64_t, Request*> finished;
    std::set<int64_t> live;          // ids submitted and not yet collected by wait / poll
    std::vector<double> latencies;   // seconds, completed requests
    size_t budget = 0, used = 0;
    int max_active = 0;
    int device = 0;
    bool stopping = false;
    int64_t next_id = 1;
    int64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, failed = 0;
    double t_first_submit = -1, t_last_done = -1;
    std::thread worker;
    cudaMemPool_t pool = nullptr;
    std::vector<CtxSlot> slots;
    std::vector<cudaStream_t> streams;
    std::vector<int> free_slots;
};

namespace {

void retire(gmres_server* S, Request* q) {
    q->t_done = now_s();
    gmres_destroy(q->ctx);    // waits for this request's stream only; buffers go back to the pool
    q->ctx = nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    if (q->slot >= 0) S->free_slots.push_back(q->slot);
    q->slot = -1;
    q->stream = nullptr;
    S->used -= q->bytes;
    q->done = true;
    S->finished[q->id] = q;
    S->latencies.push_back(q->t_done - q->t_submit);
    ++S->completed;
    if (q->status < 0) ++S->failed;
    S->t_last_done = q->t_done;
    S->cv_done.notify_all();
}

void finish(gmres_server* S, Request* q) {
    int rc = run_finish(&q->run, q->x.data());
    q->res = q->run.r;
    q->status = rc ? rc : q->run.status;
    q->res.status = q->status;
    retire(S, q);
}

// Create the request's context in its slot and enqueue its first check;
// returns false when the request finished already (an error or b = 0).
bool admit_one(gmres_server* S, Request* q) {
    q->t_admit = now_s();
    q->stream = S->streams[q->slot];
    int rc = create_ctx(&q->ctx, q->n, q->rowptr[q->n], q->rowptr.data(), q->colind.data(), q->vals.data(), 0,
                        &q->opts, q->stream, &S->slots[q->slot]);
    if (!rc) rc = run_begin(q->ctx, &q->run, q->b.data(), q->x.data(), 0);
    if (rc) {
        q->status = rc;
        q->res.status = rc;
        retire(S, q);
        return false;
    }
    if (q->run.finished) {
        finish(S, q);
        return false;
    }
    if (run_enqueue_check(&q->run)) {
        q->run.status = GMRES_ERR_CUDA;
        finish(S, q);
        return false;
    }
    return true;
}

void worker_main(gmres_server* S) {
    cudaSetDevice(S->device);
    std::vector<Request*> act;
    for (;;) {
        std::vector<Request*> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (act.empty())
                S->cv_work.wait_for(lk, std::chrono::milliseconds(20),
                                    [&] { return S->stopping || !S->pending.empty(); });
            while (!S->pending.empty() && !S->free_slots.empty() &&
                   S->used + S->pending.front()->bytes <= S->budget) {
                Request* q = S->pending.front();
                S->pending.pop_front();
                S->used += q->bytes;
                ++S->admitted;
                q->slot = S->free_slots.back();
                S->free_slots.pop_back();
                admit.push_back(q);
            }
            if (S->stopping && S->pending.empty() && act.empty() && admit.empty()) return;
        }
        for (Request* q : admit)
            if (admit_one(S, q)) act.push_back(q);
        // one polling pass: every request whose check has landed moves on
        bool progressed = false;
        std::vector<Request*> still;
        for (Request* q : act) {
            const cudaError_t qe = cudaStreamQuery(q->stream);
            if (qe == cudaErrorNotReady) {
                still.push_back(q);
                continue;
            }
            progressed = true;
            bool stop = false;
            if (qe != cudaSuccess) {
                q->run.status = GMRES_ERR_CUDA;
                stop = true;
            } else if (run_decide(&q->run)) {
                stop = true;
            } else if (run_enqueue_cycle(&q->run) || run_enqueue_check(&q->run)) {
                q->run.status = GMRES_ERR_CUDA;
                stop = true;
            }
            if (stop) finish(S, q);
            else still.push_back(q);
        }
        act.swap(still);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->active = act;
        }
        if (!progressed && admit.empty() && !act.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

double pct(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double r = p * (v.size() - 1);
    const size_t i = (size_t)r;
    const double f = r - i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int gmres_server_start(gmres_server** out, size_t mem_budget, int32_t max_active) {
    clear_error();
    GM_ARG(out != nullptr, "out is NULL");
    GM_ARG(max_active >= 1, "max_active must be >= 1");
    *out = nullptr;
    gmres_server* S = new gmres_server();
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        set_error("cudaGetDevice failed");
        return GMRES_ERR_CUDA;
    }
    if (mem_budget == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        mem_budget = fr / 10 * 9;
    }
    S->budget = mem_budget;
    S->max_active = max_active;
    // the slots and the memory pool, before any request: the worker never
    // creates a stream, allocates page-locked memory or frees device memory
    // with a device-wide synchronization
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    cudaError_t e = cudaMemPoolCreate(&S->pool, &props);
    if (e == cudaSuccess) {
        unsigned long long thr = (unsigned long long)mem_budget;
        e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    S->slots.resize(max_active);
    S->streams.resize(max_active, nullptr);
    for (int i = 0; i < max_active && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&S->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->slots[i].capture, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocHost(&S->slots[i].host_state, sizeof(DevState));
        S->slots[i].pool = S->pool;
        S->free_slots.push_back(max_active - 1 - i);
    }
    if (e == cudaSuccess && !S->streams.empty()) {
        // reserve up to 16 GB of the budget in the pool now; beyond that it grows on demand
        void* p = nullptr;
        const size_t reserve = std::min<size_t>(mem_budget, (size_t)16 << 30);
        e = cudaMallocFromPoolAsync(&p, reserve, S->pool, S->streams[0]);
        if (e == cudaSuccess) e = cudaFreeAsync(p, S->streams[0]);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->streams[0]);
    }
    if (e != cudaSuccess) {
        set_error("gmres_server_start: %s", cudaGetErrorString(e));
        gmres_server_stop(S);
        return e == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA;
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return GMRES_OK;
}

int gmres_server_submit(gmres_server* S, int64_t n, const int64_t* rowptr, const int32_t* colind,
                        const double* vals, const double* b, const double* x0, const gmres_opts* opts,
                        int64_t* id) {
    clear_error();
    GM_ARG(S != nullptr && id != nullptr && rowptr != nullptr && b != nullptr, "NULL argument");
    GM_ARG(n >= 1, "n must be >= 1");
    const int64_t nnz = rowptr[n];
    GM_ARG(nnz >= 0 && (nnz == 0 || (colind && vals)), "bad CSR");
    gmres_opts o;
    if (opts) o = *opts; else gmres_default_opts(&o);
    const size_t bytes = gmres_footprint(n, nnz, &o);
    GM_ARG(bytes > 0, "invalid options for this request");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        GM_ARG(!S->stopping, "server is stopping");
    }
    Request* q = new Request();
    q->n = n;
    q->rowptr.assign(rowptr, rowptr + n + 1);
    q->colind.assign(colind, colind + nnz);
    q->vals.assign(vals, vals + nnz);
    q->b.assign(b, b + n);
    q->x.assign(n, 0.0);
    if (x0) std::memcpy(q->x.data(), x0, n * sizeof(double));
    q->opts = o;
    q->opts.timing = 0;
    q->bytes = bytes;
    q->t_submit = now_s();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) {
        delete q;
        set_error("server is stopping");
        return GMRES_ERR_ARG;
    }
    q->id = S->next_id++;
    *id = q->id;
    S->live.insert(q->id);
    ++S->submitted;
    if (S->t_first_submit < 0) S->t_first_submit = q->t_submit;
    if (bytes > S->budget) {
        // can never fit: finish at once with an out-of-memory status
        q->status = GMRES_ERR_OOM;
        q->res.status = GMRES_ERR_OOM;
        q->done = true;
        q->t_done = q->t_submit;
        S->finished[q->id] = q;
        ++S->rejected;
        S->cv_done.notify_all();
        return GMRES_OK;
    }
    S->pending.push_back(q);
    S->cv_work.notify_one();
    return GMRES_OK;
}

int gmres_server_wait(gmres_server* S, int64_t id, double* x, gmres_result* res, double timeout_s) {
    clear_error();
    GM_ARG(S != nullptr, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    GM_ARG(S->live.count(id) > 0, "request %lld was never submitted or is already collected", (long long)id);
    auto ready = [&] { return S->finished.count(id) > 0; };
    if (timeout_s < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return 0;
    Request* q = S->finished[id];
    S->finished.erase(id);
    S->live.erase(id);
    lk.unlock();
    if (x) std::memcpy(x, q->x.data(), q->n * sizeof(double));
    if (res) *res = q->res;
    delete q;
    return 1;
}

int gmres_server_poll(gmres_server* S, int64_t id, double* x, gmres_result* res) {
    return gmres_server_wait(S, id, x, res, 0.0);
}

int gmres_server_get_stats(gmres_server* S, gmres_server_stats* st) {
    clear_error();
    GM_ARG(S != nullptr && st != nullptr, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = S->submitted;
    st->admitted = S->admitted;
    st->completed = S->completed;
    st->rejected = S->rejected;
    st->failed = S->failed;
    st->active = (int64_t)S->active.size();
    st->pending = (int64_t)S->pending.size();
    st->mem_budget = S->budget;
    st->mem_in_use = S->used;
    st->p50_ms = 1e3 * pct(S->latencies, 0.50);
    st->p99_ms = 1e3 * pct(S->latencies, 0.99);
    double sum = 0;
    for (double v : S->latencies) sum += v;
    st->mean_ms = S->latencies.empty() ? 0.0 : 1e3 * sum / S->latencies.size();
    st->busy_s = (S->t_first_submit >= 0 && S->t_last_done >= S->t_first_submit) ? S->t_last_done - S->t_first_submit : 0;
    st->solves_per_s = st->busy_s > 0 ? S->completed / st->busy_s : 0.0;
    return GMRES_OK;
}

int gmres_server_stop(gmres_server* S) {
    if (!S) return GMRES_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->finished) delete kv.second;
    for (size_t i = 0; i < S->slots.size(); ++i) {
        if (S->streams[i]) {
            cudaStreamSynchronize(S->streams[i]);
            cudaStreamDestroy(S->streams[i]);
        }
        if (S->slots[i].capture) cudaStreamDestroy(S->slots[i].capture);
        if (S->slots[i].host_state) cudaFreeHost(S->slots[i].host_state);
    }
    if (S->pool) cudaMemPoolDestroy(S->pool);
    delete S;
    return GMRES_OK;
}

}  // extern "C"
