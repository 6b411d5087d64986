// Serving loop with continuous batching over independent s-step GMRES solves.
//
// Requests (a CSR matrix, b, x0 and options; sizes and options may differ)
// are queued on submit.  A worker thread repeats:
//   1. admission: in arrival order, while the next request's device footprint
//      (gmres_footprint: basis (m+1) n, CSR, workspace) fits the free memory
//      budget and a slot is free, create its context on a stream of its own;
//   2. one restart cycle for every active request, all enqueued before any
//      waits, so the GPU overlaps their kernels;
//   3. a convergence check per request (the FP64 restart residual); finished
//      requests copy x out, release their memory and slot, and record their
//      latency (submit to completion).
// A request admitted while others are running joins them at the next cycle
// boundary.  Every request keeps its Krylov basis, Hessenberg and Givens
// state resident on the device until it finishes.  Each solve runs the same
// kernels with the same reduction order as a lone gmres_solve, so its result
// does not depend on what else is being served.
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
};

namespace {

void retire(gmres_server* S, Request* q) {
    q->t_done = now_s();
    gmres_destroy(q->ctx);
    q->ctx = nullptr;
    if (q->stream) cudaStreamDestroy(q->stream);
    q->stream = nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= q->bytes;
    q->done = true;
    S->finished[q->id] = q;
    S->latencies.push_back(q->t_done - q->t_submit);
    ++S->completed;
    if (q->status < 0) ++S->failed;
    S->t_last_done = q->t_done;
    S->cv_done.notify_all();
}

// Create the request's context and start its solve; errors finish the request.
void admit_one(gmres_server* S, Request* q) {
    q->t_admit = now_s();
    int rc = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking) == cudaSuccess ? GMRES_OK : GMRES_ERR_CUDA;
    if (!rc)
        rc = gmres_create(&q->ctx, q->n, q->rowptr[q->n], q->rowptr.data(), q->colind.data(), q->vals.data(), 0,
                          &q->opts, q->stream);
    if (!rc) rc = run_begin(q->ctx, &q->run, q->b.data(), q->x.data(), 0);
    if (rc) {
        q->status = rc;
        q->res.status = rc;
        retire(S, q);
        return;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->active.push_back(q);
}

void worker_main(gmres_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Request*> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait_for(lk, std::chrono::milliseconds(20), [&] {
                return S->stopping || !S->pending.empty() || !S->active.empty();
            });
            while (!S->pending.empty() && (int)(S->active.size() + admit.size()) < S->max_active &&
                   S->used + S->pending.front()->bytes <= S->budget) {
                Request* q = S->pending.front();
                S->pending.pop_front();
                S->used += q->bytes;
                ++S->admitted;
                admit.push_back(q);
            }
            if (S->stopping && S->pending.empty() && S->active.empty() && admit.empty()) return;
        }
        for (Request* q : admit) admit_one(S, q);
        std::vector<Request*> act;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            act = S->active;
        }
        if (act.empty()) continue;
        // one convergence check + (if needed) one restart cycle per active request,
        // enqueued for all of them before any wait
        for (Request* q : act) {
            if (!q->run.finished) {
                int rc = run_enqueue_check(&q->run);
                if (rc) { q->run.finished = true; q->run.status = rc; }
            }
        }
        std::vector<Request*> still;
        for (Request* q : act) {
            bool stop = q->run.finished;
            if (!stop) {
                if (cudaStreamSynchronize(q->stream) != cudaSuccess) {
                    q->run.status = GMRES_ERR_CUDA;
                    stop = true;
                } else if (run_decide(&q->run)) {
                    stop = true;
                } else if (run_enqueue_cycle(&q->run)) {
                    q->run.status = GMRES_ERR_CUDA;
                    stop = true;
                }
            }
            if (stop) {
                int rc = run_finish(&q->run, q->x.data());
                q->res = q->run.r;
                q->status = rc ? rc : q->run.status;
                q->res.status = q->status;
                retire(S, q);
            } else {
                still.push_back(q);
            }
        }
        std::lock_guard<std::mutex> lk(S->mu);
        std::vector<Request*> keep;
        for (Request* q : S->active)
            if (std::find(still.begin(), still.end(), q) != still.end()) keep.push_back(q);
        S->active.swap(keep);
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
    delete S;
    return GMRES_OK;
}

}  // extern "C"
