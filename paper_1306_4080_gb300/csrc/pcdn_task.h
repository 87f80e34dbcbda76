// Non-blocking solve: the outer loop of Algorithm 3 (the same stages and stop rule as pcdn_solve)
// as a state machine that issues one stage at a time on the problem's own stream and never waits
// on the host.  The batch solver and the request server (pcdn_sched.cu) drive many of these at
// once, one stream each, so independent solves overlap on the device.
//
// Stages: [refresh + KKT at the start point] -> ([partition, items, walk, refresh, KKT] per outer
// iteration) -> [objective, counters].  Each stage ends by copying its scalars (KKT norm,
// objective, error flags, counters) into a pinned host mailbox and recording an event;
// task_poll() consumes a finished stage and issues the next.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pcdn.h"

namespace pcdn {

struct SolveTask;

// A task with its pinned mailbox and completion event (created once, reused across solves).
int task_create(SolveTask** out);
void task_destroy(SolveTask* t);

// Start a solve of `prob` (P, eps, seed, opts as pcdn_solve).  grid = blocks of the bundle
// walker: 1 runs it as one thread block (an ordinary launch, no waits between blocks), 0 takes
// pcdn_solve's choice.  Enqueues the first stage and returns.
int task_start(SolveTask* t, pcdn_problem* prob, int32_t P, double eps, uint64_t seed, const pcdn_opts* opts,
               int grid);

// If the stage in flight has finished, consume it and enqueue the next one.  *done becomes 1
// when the solve has ended; the return value is then its status (PCDN_OK, PCDN_ENOTCONVERGED or
// an error); before that it is PCDN_OK unless issuing a stage failed.
int task_poll(SolveTask* t, int* done);

// Block until the stage in flight has finished (then task_poll advances without waiting).
int task_wait(SolveTask* t);

// After the solve has ended: its statistics and (w_out may be NULL) the final w, copied to the
// host synchronously on the problem's stream.
int task_result(SolveTask* t, double* w_out, pcdn_stats* stats);

// Number of features of a problem.
int64_t problem_n_features(pcdn_problem* p);

// Device bytes a problem of this shape holds once created (and at most transiently while it is
// created), for admission under a memory budget.
int64_t problem_bytes_estimate(int64_t n, int64_t m, int64_t nnz, int32_t P);

}  // namespace pcdn
