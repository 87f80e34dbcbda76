// Non-blocking solve: the outer loop of Algorithm 3 (the same stages and stop rule as pcdn_solve)
// as a state machine that issues one stage at a time on the problem's own stream and never waits
// on the host.  The batch solver and the request server (pcdn_sched.cpp) drive many of these at
// once, one stream each, so independent solves overlap on the device.
//
// Stages: [refresh + KKT at the start point] -> ([partition, items, walk, refresh, KKT] per outer
// iteration, replayed from a CUDA graph captured at the first one) -> [objective, counters].  Each
// stage ends by copying its scalars (KKT norm, objective, error flags, counters) into a pinned host
// mailbox and recording an event; task_poll() consumes a finished stage and issues the next.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "pcdn.h"

namespace pcdn {

struct SolveTask;

// Thread blocks that the multi-block (cooperative) walkers of concurrent solves may hold together.
// A solve takes its blocks when it starts and returns them when it ends.  Keeping the cooperative walkers' total within what the GPU holds resident next to the
// one-block walkers guarantees that each of them can become fully resident: what it may wait for
// (one-block walkers, the other kernels) finishes on its own, and no two cooperative walkers can
// each hold part of the GPU while waiting for the rest.
struct BlockBudget {
  std::atomic<int> free{0};
};

// Walker blocks a solve of this problem wants at bundle size P: about kBlockNnz nonzeros of a
// bundle per block, at most kMaxBlocks; 1 for bundles that one block handles quickly.
constexpr int64_t kBlockNnz = 2048;
constexpr int kMaxBlocks = 64;
int walker_blocks_wanted(pcdn_problem* p, int32_t P);

// Let the task's solves take up to `want` walker blocks from `budget` (a multi-block walker when at
// least 2 are free, else one block), held from the solve's start to its end.  budget NULL: the
// grid passed to task_start.
void task_set_blocks(SolveTask* t, BlockBudget* budget, int want);

// Replay each solve's outer iterations from a CUDA graph captured at its first one (default on;
// a solve whose capture fails issues its kernels directly).
void task_set_graphs(SolveTask* t, bool on);
// Whether the task's last solve replayed its outer iterations from a graph.
bool task_used_graph(SolveTask* t);

// Walker blocks the current device holds resident at once (the whole-GPU walker's grid).
int device_walker_capacity(int* out);

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

// Number of features and of nonzeros of a problem.
int64_t problem_n_features(pcdn_problem* p);
int64_t problem_nnz(pcdn_problem* p);
// the row-sorted layout fits the problem (its exact sums take fewer than 2^24 terms)
bool problem_rows_layout_ok(pcdn_problem* p);

// Device bytes a problem of this shape holds once created (and at most transiently while it is
// created), for admission under a memory budget.
int64_t problem_bytes_estimate(int64_t n, int64_t m, int64_t nnz, int32_t P);

}  // namespace pcdn
