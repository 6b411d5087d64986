// Step-wise solve on a gmres_ctx (used by gmres_solve and by the serving loop).
#pragma once
#include <vector>
#include <utility>
#include "solver_state.cuh"

namespace gm {

// What a serving slot lends a context: a memory pool for its device buffers
// (stream-ordered allocation, no device-wide synchronization), the stream to
// capture its cycle graphs on, and a page-locked mirror of its DevState.
struct CtxSlot {
    cudaMemPool_t pool = nullptr;
    cudaStream_t capture = nullptr;
    DevState* host_state = nullptr;
};

// gmres_create with an optional slot (nullptr: the context allocates and owns
// everything, as gmres_create does).
int create_ctx(gmres_ctx** out, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colind,
               const double* vals, int32_t ptr_on_device, const gmres_opts* opts, void* stream, const CtxSlot* slot);

struct SolveRun {
    gmres_ctx* c = nullptr;
    gmres_result r{};
    double bnorm = 0.0;
    int cyc = 0;
    int status = GMRES_WARN_MAXIT;
    int on_device = 0;
    bool finished = false;
    CycleBasis cb;               // basis of the next restart cycle
    CycleBasis ran;              // basis of the last cycle enqueued
    bool auto_pending = false;   // GMRES_BASIS_NEWTON_AUTO before its shifts are chosen
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    std::vector<std::pair<int, int>> marks;
};

// Copy b and x0, compute ||b|| (synchronizes the context's stream).  Sets
// R->finished for b = 0 (x = 0) or a non-finite b.
int run_begin(gmres_ctx* c, SolveRun* R, const double* b, const double* x, int on_device);
// Enqueue r = b - A x and the read-back of the cycle state (asynchronous).
int run_enqueue_check(SolveRun* R);
// Once the stream has passed the read-back: 1 = stop (R->status final), 0 = run another cycle.
int run_decide(SolveRun* R);
// Enqueue one restart cycle (asynchronous).
int run_enqueue_cycle(SolveRun* R);
// Copy x out and synchronize; R->r.status holds the final status.
int run_finish(SolveRun* R, double* x);
cudaStream_t run_stream(const SolveRun* R);

}  // namespace gm
