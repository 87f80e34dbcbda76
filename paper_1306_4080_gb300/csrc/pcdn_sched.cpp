// Many solves at once on one GPU: the batch solver (independent problems, each along a
// warm-started regularisation path), the bundle-size autotuner, and the request server
// (continuous batching under a device-memory budget).
//
// Every solve is a non-blocking SolveTask (pcdn_task.h) on its problem's own stream with the bundle
// walker as a single thread block (an ordinary launch: no waits between blocks, so any number of
// walkers can share the GPU without co-residency requirements).  Host threads poll the tasks and
// issue each problem's next stage as soon as its previous one ends, so problems advance
// independently and at their own pace: a small problem is never held back by a large one.
//
// The method's arithmetic is unchanged: each solve runs the same stages, kernels and stop rule as
// pcdn_solve (Algorithm 3 with Algorithm 4; relative minimum-norm subgradient after every outer
// iteration).

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pcdn.h"
#include "pcdn_task.h"

namespace pcdn {
void set_last_error(const char* msg);
}

using namespace pcdn;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kCreators = 4;  // request server: threads copying admitted requests to the device

int sfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

// Keep the first error of a group of jobs (code and message) for the caller's thread.
struct FirstError {
  std::mutex mu;
  int code = PCDN_OK;
  std::string msg;
  void note(int rc) {
    if (rc >= 0) return;
    std::lock_guard<std::mutex> lock(mu);
    if (code == PCDN_OK) {
      code = rc;
      msg = pcdn_last_error();
    }
  }
};

// Solves in flight by default: one per hardware work queue.  Streams beyond the queues share them,
// and a stream waiting for its own previous kernel then holds up the others in its queue.  The
// queue count is CUDA_DEVICE_MAX_CONNECTIONS (CUDA's default 8, at most 32), read when the CUDA
// context is created: set it before the process touches the GPU.
int default_slots() {
  int conn = 8;
  if (const char* v = std::getenv("CUDA_DEVICE_MAX_CONNECTIONS")) {
    const int c = std::atoi(v);
    if (c > 0) conn = std::min(c, 32);
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 64;
  }
  return std::min(conn, 2 * sms);
}

// Bundle sizes the autotuner tries: powers of four from 16, those not above n_features (at
// least one candidate: n_features itself when it is below 16).
std::vector<int32_t> default_candidates(int64_t m) {
  std::vector<int32_t> c;
  for (int64_t P = 16; P <= 4096 && P <= m; P *= 4) c.push_back((int32_t)P);
  if (c.empty()) c.push_back((int32_t)m);
  return c;
}

// Autotuner score of a probe solve: device seconds of its bundle walks (CUDA events on its stream,
// which unlike host time do not include the host's polling of many concurrent solves) per decade
// of relative-KKT reduction; a probe that stops at its epoch cap before the probe tolerance is
// scored by the progress it made.
double probe_score(const pcdn_stats& st) {
  const double decades = st.kkt_rel > 0 ? -std::log10(st.kkt_rel) : 16.0;
  return st.walk_s / std::max(decades, 1e-3);
}

// A probe that got fewer walker blocks than it asked for (other solves held the shared budget) ran
// slower than its path's solves will once they hold their blocks, which biases the choice toward
// small bundles.  Its time is scaled to the blocks it wanted by the walker's per-bundle time law
// in its block count, time ~ blocks^-0.56 (31, 42 and 67 us per bundle at 304, 152 and 76 blocks on
// the 2M x 3M workload).  A probe that got its blocks keeps its measured time.
double probe_score_for_blocks(const pcdn_stats& st, int wanted) {
  double s = probe_score(st);
  if (wanted > 1 && st.walk_grid > 0 && st.walk_grid < wanted) s *= std::pow((double)st.walk_grid / wanted, 0.56);
  return s;
}

// The C a job's probes run at: the geometric middle of its path (the larger C values of a path
// cost the most outer iterations, the smallest the fewest).
double probe_C(const pcdn_batch_job& j) { return std::sqrt(j.C_path[0] * j.C_path[j.n_C - 1]); }

// ------------------------------------------------------------------------------------------ batch
struct JobRun {
  pcdn_batch_job* job = nullptr;
  int64_t m = 0;
  // autotuner
  std::vector<int32_t> cand;
  std::vector<int32_t> cand_layout;  // the walker layout of each candidate (PCDN_LAYOUT_*)
  size_t probe = 0;
  double best_s = 0.0;
  int32_t best_P = 0, best_layout = PCDN_LAYOUT_AUTO;
  int32_t layout = PCDN_LAYOUT_AUTO;  // of the path's solves
  bool probing = false;
  // path
  int32_t P = 0;
  int32_t ci = 0;
  bool warm = false;  // the next solve continues from the problem's current w
  // repeated solves of one C: the product of the earlier attempts' relative KKT values and the
  // first attempt's starting KKT value, so that the target stays eps times the latter
  double kkt_scale = 1.0, kkt0 = 0.0;
  int status = PCDN_OK;
};

struct BatchShared {
  pcdn_batch_job* jobs;
  int32_t n_jobs;
  std::vector<int32_t> order;  // jobs in the order they are started: most work first
  pcdn_opts opts;
  double probe_eps;
  int32_t probe_epochs;
  bool use_graphs = true;
  bool tune_layout = true;
  std::vector<int32_t> cand;
  std::atomic<int32_t> next{0};
  std::atomic<int64_t> solves{0}, probes{0}, epochs{0}, coord{0}, graphs{0}, retries{0};
  std::mutex acc_mu;
  double bytes_model = 0.0;
  FirstError err;
  BlockBudget budget;  // walker blocks for multi-block walkers
};

// Start the job's next solve on task t; returns a status (< 0: the job failed).
int start_next(BatchShared& B, JobRun& r, SolveTask* t) {
  pcdn_batch_job& j = *r.job;
  pcdn_opts o = B.opts;
  if (r.probing) {
    o.warm_start = 0;
    if (B.probe_epochs > 0 && o.max_epochs > B.probe_epochs) o.max_epochs = B.probe_epochs;
    int rc = pcdn_set_C(j.prob, probe_C(j));
    if (rc) return rc;
    o.layout = r.cand_layout[r.probe];
    task_set_blocks(t, &B.budget, walker_blocks_wanted(j.prob, r.cand[r.probe]));
    return task_start(t, j.prob, r.cand[r.probe], B.probe_eps, j.seed, &o, 1);
  }
  if (j.P == 0) o.layout = r.layout;
  if (r.ci > 0 || r.warm) o.warm_start = 1;
  int rc = pcdn_set_C(j.prob, j.C_path[r.ci]);
  if (rc) return rc;
  task_set_blocks(t, &B.budget, walker_blocks_wanted(j.prob, r.P));
  return task_start(t, j.prob, r.P, j.eps / r.kkt_scale, j.seed, &o, 1);
}

// A solve of the job ended on task t (status rc): record it and start the next one.
// Returns true when the job is complete.
bool on_done(BatchShared& B, JobRun& r, SolveTask* t, int rc) {
  pcdn_batch_job& j = *r.job;
  pcdn_stats st;
  if (r.probing) {
    int rr = task_result(t, nullptr, &st);
    B.probes.fetch_add(1);
    if (rr < 0) {
      r.status = rr;
      return true;
    }
    const double score = probe_score_for_blocks(st, walker_blocks_wanted(j.prob, r.cand[r.probe]));
    if (r.best_P == 0 || score < r.best_s) {
      r.best_s = score;
      r.best_P = r.cand[r.probe];
      r.best_layout = r.cand_layout[r.probe];
    }
    if (++r.probe >= r.cand.size()) {
      r.probing = false;
      r.P = r.best_P;
      r.layout = r.best_layout;
      j.P_used = r.P;
      j.layout_used = r.layout;
    }
  } else {
    double* w = j.w_out ? j.w_out + (int64_t)r.ci * r.m : nullptr;
    int rr = task_result(t, w, &st);
    if (rr < 0 || rc < 0) {
      r.status = rr < 0 ? rr : rc;
      return true;
    }
    B.epochs.fetch_add(st.epochs);
    B.coord.fetch_add(st.coord_updates);
    {
      std::lock_guard<std::mutex> lock(B.acc_mu);
      B.bytes_model += st.bytes_model;
    }
    if (task_used_graph(t)) B.graphs.fetch_add(1);
    int32_t smaller = 0;
    if (rr == PCDN_ENOTCONVERGED && j.P == 0)
      for (int32_t c : r.cand)
        if (c < r.P && c > smaller) smaller = c;
    if (smaller > 0) {
      // stalled at this C with the autotuned size: solve it again from here with the next smaller
      // one, its relative tolerance measured from this C's first start
      B.retries.fetch_add(1);
      if (r.kkt_scale == 1.0) r.kkt0 = st.kkt0;
      r.kkt_scale *= st.kkt_rel;
      r.P = smaller;
      j.P_used = smaller;
      r.layout = PCDN_LAYOUT_AUTO;  // the library's choice for the new size
      j.layout_used = PCDN_LAYOUT_AUTO;
      r.warm = true;
    } else {
      if (r.kkt_scale != 1.0) {
        st.kkt_rel *= r.kkt_scale;
        st.kkt0 = r.kkt0;
        r.kkt_scale = 1.0;
      }
      if (j.stats) j.stats[r.ci] = st;
      if (rr == PCDN_ENOTCONVERGED) r.status = PCDN_ENOTCONVERGED;
      B.solves.fetch_add(1);
      if (++r.ci >= j.n_C) return true;
    }
  }
  int s = start_next(B, r, t);
  if (s < 0) {
    r.status = s;
    return true;
  }
  return false;
}

void batch_worker(BatchShared& B, int cap, int device) {
  cudaSetDevice(device);
  std::vector<SolveTask*> tasks(cap, nullptr);
  std::vector<JobRun> runs(cap);
  std::vector<bool> busy(cap, false);
  for (int k = 0; k < cap; ++k) {
    int rc = task_create(&tasks[k]);
    if (!rc) task_set_graphs(tasks[k], B.use_graphs);
    if (rc) {
      B.err.note(rc);
      for (int i = 0; i < k; ++i) task_destroy(tasks[i]);
      // the jobs this worker would have taken are left to the others; mark the ones it claims
      for (;;) {
        int32_t idx = B.next.fetch_add(1);
        if (idx >= B.n_jobs) return;
        B.jobs[B.order[idx]].status = rc;
      }
    }
  }
  auto finish = [&](int k) {
    JobRun& r = runs[k];
    r.job->status = r.status;
    B.err.note(r.status);
    busy[k] = false;
  };
  int active = 0;
  bool more = true;
  while (true) {
    // fill free slots with new jobs
    for (int k = 0; k < cap && more; ++k) {
      if (busy[k]) continue;
      int32_t idx = B.next.fetch_add(1);
      if (idx >= B.n_jobs) {
        more = false;
        break;
      }
      JobRun& r = runs[k];
      r = JobRun();
      r.job = &B.jobs[B.order[idx]];
      r.job->status = PCDN_OK;
      r.m = problem_n_features(r.job->prob);
      r.P = r.job->P;
      r.job->P_used = r.P;
      r.job->layout_used = B.opts.layout;
      if (r.P == 0) {
        r.probing = true;
        std::vector<int32_t> sizes = B.cand.empty() ? default_candidates(r.m) : B.cand, ok;
        for (int32_t P : sizes)
          if (P >= 1 && P <= r.m) ok.push_back(P);
        if (ok.empty()) ok.push_back((int32_t)r.m);
        // every size with the library's layout; a size whose walker takes several blocks also with
        // the other layout (the two differ only when the walker has more than one block)
        r.cand.clear();
        r.cand_layout.clear();
        for (int32_t P : ok) {
          r.cand.push_back(P);
          r.cand_layout.push_back(B.opts.layout);
          if (B.tune_layout && B.opts.layout == PCDN_LAYOUT_AUTO && walker_blocks_wanted(r.job->prob, P) > 1 &&
              problem_rows_layout_ok(r.job->prob)) {
            r.cand.push_back(P);
            r.cand_layout.push_back(B.opts.prec == PCDN_PREC_FP64 ? PCDN_LAYOUT_SCATTER : PCDN_LAYOUT_ROWS);
          }
        }
      }
      busy[k] = true;
      ++active;
      int s = start_next(B, r, tasks[k]);
      if (s < 0) {
        r.status = s;
        finish(k);
        --active;
      }
    }
    if (active == 0 && !more) break;
    bool progressed = false;
    for (int k = 0; k < cap; ++k) {
      if (!busy[k]) continue;
      int done = 0;
      int rc = task_poll(tasks[k], &done);
      if (!done) {
        if (rc < 0) {  // issuing a stage failed
          runs[k].status = rc;
          task_wait(tasks[k]);
          finish(k);
          --active;
          progressed = true;
        }
        continue;
      }
      progressed = true;
      if (on_done(B, runs[k], tasks[k], rc)) {
        finish(k);
        --active;
      }
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  for (int k = 0; k < cap; ++k) task_destroy(tasks[k]);
}

// ------------------------------------------------------------------------------------------ server
struct Request {
  int64_t ticket = 0;
  // X and y on the host: the server's own copies, or (borrowed) the caller's arrays
  std::vector<int64_t> col_ptr;
  std::vector<int32_t> row_idx;
  std::vector<float> val;
  std::vector<int8_t> y;
  const int64_t* xcp = nullptr;
  const int32_t* xri = nullptr;
  const float* xv = nullptr;
  const int8_t* xy = nullptr;
  int64_t n = 0, m = 0, nnz = 0;
  double C = 1.0;
  int loss = 0;
  int32_t P = 1;
  double eps = 1e-3;
  uint64_t seed = 0;
  int64_t bytes = 0;
  double t_submit = 0.0, t_admit = 0.0, t_start = 0.0, t_done = 0.0;
  pcdn_problem* prob = nullptr;
  bool started = false;   // its solve has been started by the driver
  bool done = false;      // result (or error) available to pcdn_server_wait
  bool retired = false;   // its problem is destroyed (or was never created)
  bool handed = false;    // pcdn_server_wait has returned it; the request is deleted once retired
  int status = PCDN_OK;
  std::string msg;
  std::vector<double> w;
  pcdn_stats stats{};
  int32_t retries = 0;    // solves repeated with a smaller bundle size after reaching max_epochs
  double kkt_scale = 1.0, kkt0 = 0.0;  // as JobRun's, for those repeats
};

}  // namespace

struct pcdn_server {
  int device = 0;
  int32_t slots = 1;
  int64_t budget = 0;
  pcdn_opts opts{};
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_admit;  // admission thread: a request arrived, a slot or memory freed
  std::condition_variable cv_create; // creator threads: a request was admitted
  std::condition_variable cv_done;   // waiters: a request finished
  std::deque<Request*> queue;        // submitted, not yet admitted (FIFO)
  std::deque<Request*> to_create;    // admitted (slot and memory reserved), problem not yet created
  std::deque<Request*> incoming;     // problem created, solve not yet started
  std::deque<Request*> retire;       // finished, problem to destroy
  std::unordered_map<int64_t, Request*> all;
  int64_t next_ticket = 1;
  int32_t in_flight = 0;             // admitted and not yet retired
  int64_t bytes_in_use = 0;
  bool stop = false;
  BlockBudget blocks;                // walker blocks for multi-block walkers
  std::thread admit_thread, drive_thread;
  std::vector<std::thread> creators;
  int64_t submitted = 0, finished = 0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Admission, in arrival order: reserve a slot and the request's device footprint, then hand it to
// a creator thread.  Also destroys the problems of finished requests, which frees both.
void admission_loop(pcdn_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (true) {
    while (!s->retire.empty()) {
      Request* r = s->retire.front();
      s->retire.pop_front();
      pcdn_problem* p = r->prob;
      const int64_t bytes = r->bytes;
      r->prob = nullptr;
      r->retired = true;
      if (r->handed) delete r;
      lock.unlock();
      pcdn_destroy(p);
      lock.lock();
      s->bytes_in_use -= bytes;
      s->in_flight -= 1;
      s->cv_done.notify_all();
    }
    if (s->stop) break;
    Request* head = s->queue.empty() ? nullptr : s->queue.front();
    const bool fits = head && s->in_flight < s->slots &&
                      (s->bytes_in_use + head->bytes <= s->budget || s->in_flight == 0);
    if (!fits) {
      s->cv_admit.wait(lock);
      continue;
    }
    s->queue.pop_front();
    s->in_flight += 1;
    s->bytes_in_use += head->bytes;
    head->t_admit = s->now();
    s->to_create.push_back(head);
    s->cv_create.notify_one();
  }
}

// Creator threads copy admitted requests to the device (pcdn_create: host validation, copy, row
// mirror) in parallel, so one large request does not hold back the admission of the next.
void creator_loop(pcdn_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (true) {
    while (!s->stop && s->to_create.empty()) s->cv_create.wait(lock);
    if (s->stop) break;
    Request* r = s->to_create.front();
    s->to_create.pop_front();
    lock.unlock();
    pcdn_csc X;
    X.n_samples = r->n;
    X.n_features = r->m;
    X.nnz = r->nnz;
    X.col_ptr = r->xcp;
    X.row_idx = r->xri;
    X.val = r->xv;
    pcdn_problem* p = nullptr;
    int rc = pcdn_create(&X, r->xy, r->C, (pcdn_loss)r->loss, &p);
    std::string msg = rc ? pcdn_last_error() : "";
    // the device has its copy: release the host one
    std::vector<int64_t>().swap(r->col_ptr);
    std::vector<int32_t>().swap(r->row_idx);
    std::vector<float>().swap(r->val);
    std::vector<int8_t>().swap(r->y);
    r->xcp = nullptr;
    r->xri = nullptr;
    r->xv = nullptr;
    r->xy = nullptr;
    lock.lock();
    if (rc) {
      r->status = rc;
      r->msg = msg;
      r->done = true;
      r->retired = true;
      r->t_done = s->now();
      s->in_flight -= 1;
      s->bytes_in_use -= r->bytes;
      s->finished += 1;
      s->cv_done.notify_all();
      s->cv_admit.notify_all();
      continue;
    }
    r->prob = p;
    s->incoming.push_back(r);
    s->cv_done.notify_all();  // wakes an idle driver
  }
}

void drive_loop(pcdn_server* s) {
  cudaSetDevice(s->device);
  std::vector<SolveTask*> tasks(s->slots, nullptr);
  std::vector<Request*> run(s->slots, nullptr);
  int ok_tasks = 0;
  for (int k = 0; k < s->slots; ++k) {
    if (task_create(&tasks[k])) break;
    ++ok_tasks;
  }
  while (true) {
    // take admitted requests into free slots
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (s->stop) break;
      for (int k = 0; k < ok_tasks && !s->incoming.empty(); ++k) {
        if (run[k]) continue;
        Request* r = s->incoming.front();
        s->incoming.pop_front();
        run[k] = r;
      }
    }
    bool progressed = false;
    for (int k = 0; k < ok_tasks; ++k) {
      Request* r = run[k];
      if (!r) continue;
      int done = 0, rc = PCDN_OK;
      if (r->started) {
        rc = task_poll(tasks[k], &done);
        if (!done && rc < 0) {
          task_wait(tasks[k]);
          done = 1;
        }
      } else {
        pcdn_opts o = s->opts;
        o.warm_start = 0;
        task_set_blocks(tasks[k], &s->blocks, walker_blocks_wanted(r->prob, r->P));
        rc = task_start(tasks[k], r->prob, r->P, r->eps, r->seed, &o, 1);
        r->started = true;
        r->t_start = s->now();
        progressed = true;
        if (rc < 0) done = 1;
      }
      if (!done) continue;
      progressed = true;
      std::vector<double> w((size_t)r->m);
      pcdn_stats st;
      std::memset(&st, 0, sizeof(st));
      int rr = rc < 0 ? rc : task_result(tasks[k], w.data(), &st);
      int32_t smaller = 0;
      if (rr == PCDN_ENOTCONVERGED)
        for (int32_t c : default_candidates(r->m))
          if (c < r->P && c > smaller) smaller = c;
      if (smaller > 0) {
        // stalled with the requested bundle size: go on from the w reached with the next smaller
        // default size, the relative tolerance still measured from w = 0
        if (r->kkt_scale == 1.0) r->kkt0 = st.kkt0;
        r->kkt_scale *= st.kkt_rel;
        r->P = smaller;
        r->retries += 1;
        pcdn_opts o = s->opts;
        o.warm_start = 1;
        task_set_blocks(tasks[k], &s->blocks, walker_blocks_wanted(r->prob, r->P));
        rr = task_start(tasks[k], r->prob, r->P, r->eps / r->kkt_scale, r->seed, &o, 1);
        if (rr >= 0) continue;
      }
      if (rr >= 0 && r->kkt_scale != 1.0) {
        st.kkt_rel *= r->kkt_scale;
        st.kkt0 = r->kkt0;
      }
      std::string msg = rr < 0 ? pcdn_last_error() : "";
      std::lock_guard<std::mutex> lock(s->mu);
      r->w.swap(w);
      r->stats = st;
      r->status = rr;
      r->msg = msg;
      r->t_done = s->now();
      r->done = true;
      s->finished += 1;
      s->retire.push_back(r);
      run[k] = nullptr;
      s->cv_done.notify_all();
      s->cv_admit.notify_all();
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lock(s->mu);
      bool any = false;
      for (int k = 0; k < ok_tasks; ++k) any = any || run[k];
      if (!any && s->incoming.empty() && !s->stop) {
        // nothing in flight: sleep until the admission thread hands over a request
        s->cv_done.wait_for(lock, std::chrono::microseconds(200));
      } else {
        lock.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      }
    }
  }
  // stopping: let the stages in flight end, then hand their problems to the admission thread
  for (int k = 0; k < ok_tasks; ++k) {
    if (run[k]) {
      task_wait(tasks[k]);
      std::lock_guard<std::mutex> lock(s->mu);
      s->retire.push_back(run[k]);
      s->cv_admit.notify_all();
    }
    task_destroy(tasks[k]);
  }
}

}  // namespace

extern "C" {

void pcdn_default_batch_opts(pcdn_batch_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_inflight = 0;
  o->threads = 0;
  o->probe_eps = 0.1;
  o->probe_epochs = 3;
  o->n_candidates = 0;
  o->candidates = nullptr;
  o->tune_layout = 0;
}

int pcdn_solve_batch(pcdn_batch_job* jobs, int32_t n_jobs, const pcdn_opts* opts, const pcdn_batch_opts* bopts,
                     pcdn_batch_stats* out) {
  set_last_error("");
  if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return sfail(PCDN_EINVAL, "jobs must be given");
  pcdn_batch_opts bo;
  if (bopts) bo = *bopts;
  else pcdn_default_batch_opts(&bo);
  pcdn_opts o;
  if (opts) o = *opts;
  else pcdn_default_opts(&o);
  if (bo.max_inflight < 0 || bo.threads < 0 || bo.n_candidates < 0 || (bo.n_candidates > 0 && !bo.candidates))
    return sfail(PCDN_EINVAL, "bad batch options");
  for (int32_t i = 0; i < n_jobs; ++i) {
    const pcdn_batch_job& j = jobs[i];
    if (!j.prob) return sfail(PCDN_EINVAL, "job %d: problem missing", i);
    if (j.n_C < 1 || !j.C_path) return sfail(PCDN_EINVAL, "job %d: C path missing", i);
    for (int32_t k = 0; k < j.n_C; ++k)
      if (!(j.C_path[k] > 0) || !std::isfinite(j.C_path[k])) return sfail(PCDN_EINVAL, "job %d: C must be positive", i);
    if (j.P < 0 || j.P > problem_n_features(j.prob)) return sfail(PCDN_EINVAL, "job %d: P out of range", i);
    if (j.P == 0 && o.warm_start) return sfail(PCDN_EINVAL, "job %d: the autotuner (P = 0) needs a cold start", i);
    if (!(j.eps > 0)) return sfail(PCDN_EINVAL, "job %d: eps must be positive", i);
    for (int32_t k = 0; k < i; ++k)
      if (jobs[k].prob == j.prob) return sfail(PCDN_EINVAL, "jobs %d and %d share a problem", k, i);
  }
  if (!(bo.probe_eps > 0)) bo.probe_eps = 0.1;
  if (out) std::memset(out, 0, sizeof(*out));
  if (n_jobs == 0) return PCDN_OK;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return sfail(PCDN_ECUDA, "no CUDA device");
  }
  const auto t0 = Clock::now();
  BatchShared B;
  B.jobs = jobs;
  B.n_jobs = n_jobs;
  B.opts = o;
  B.probe_eps = bo.probe_eps;
  B.probe_epochs = bo.probe_epochs;
  B.use_graphs = bo.no_graphs == 0;
  B.tune_layout = bo.tune_layout != 0;
  // longest jobs first (nonzeros times path length), so that the batch's critical paths start at
  // once and take the walker blocks they want before the short jobs fill the GPU
  B.order.resize(n_jobs);
  for (int32_t i = 0; i < n_jobs; ++i) B.order[i] = i;
  std::stable_sort(B.order.begin(), B.order.end(), [&](int32_t a, int32_t b) {
    return (double)problem_nnz(jobs[a].prob) * jobs[a].n_C > (double)problem_nnz(jobs[b].prob) * jobs[b].n_C;
  });
  for (int32_t k = 0; k < bo.n_candidates; ++k) B.cand.push_back(bo.candidates[k]);
  int inflight = bo.max_inflight > 0 ? bo.max_inflight : default_slots();
  inflight = std::min<int>(inflight, n_jobs);
  // multi-block walkers share what the one-block walkers of the in-flight jobs leave of the GPU
  int cap = 0;
  if (device_walker_capacity(&cap) != PCDN_OK) return PCDN_ECUDA;
  B.budget.free = std::max(0, cap - inflight);
  int threads = bo.threads > 0 ? bo.threads : 4;
  threads = std::max(1, std::min(threads, inflight));
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t) {
    const int cap = inflight / threads + (t < inflight % threads ? 1 : 0);
    pool.emplace_back(batch_worker, std::ref(B), cap, device);
  }
  for (auto& th : pool) th.join();
  if (out) {
    out->wall_s = std::chrono::duration<double>(Clock::now() - t0).count();
    out->solves = B.solves.load();
    out->probe_solves = B.probes.load();
    out->retries = B.retries.load();
    out->epochs = B.epochs.load();
    out->coord_updates = B.coord.load();
    out->bytes_model = B.bytes_model;
    out->graph_solves = B.graphs.load();
  }
  if (B.err.code < 0) {
    set_last_error(B.err.msg.c_str());
    return B.err.code;
  }
  for (int32_t i = 0; i < n_jobs; ++i)
    if (jobs[i].status == PCDN_ENOTCONVERGED) return PCDN_ENOTCONVERGED;
  return PCDN_OK;
}

int pcdn_autotune(pcdn_problem* prob, const int32_t* candidates, int32_t n_candidates, double probe_eps,
                  int32_t probe_epochs, uint64_t seed, const pcdn_opts* opts, int32_t* P_best, double* probe_s) {
  set_last_error("");
  if (!prob || !P_best) return sfail(PCDN_EINVAL, "problem and P_best must be given");
  if (n_candidates < 0 || (n_candidates > 0 && !candidates)) return sfail(PCDN_EINVAL, "bad candidates");
  const int64_t m = problem_n_features(prob);
  std::vector<int32_t> cand;
  if (n_candidates > 0) cand.assign(candidates, candidates + n_candidates);
  else cand = default_candidates(m);
  for (int32_t P : cand)
    if (P < 1 || P > m) return sfail(PCDN_EINVAL, "candidate P = %d out of [1, n_features]", P);
  if (!(probe_eps > 0)) probe_eps = 0.1;
  pcdn_opts o;
  if (opts) o = *opts;
  else pcdn_default_opts(&o);
  o.warm_start = 0;
  if (probe_epochs > 0 && o.max_epochs > probe_epochs) o.max_epochs = probe_epochs;
  SolveTask* t = nullptr;
  int rc = task_create(&t);
  if (rc) return rc;
  double best = 0.0;
  int32_t bestP = 0;
  for (size_t k = 0; k < cand.size(); ++k) {
    rc = task_start(t, prob, cand[k], probe_eps, seed, &o, 1);
    int done = 0;
    while (rc >= 0 && !done) {
      if ((rc = task_wait(t)) < 0) break;
      rc = task_poll(t, &done);
    }
    pcdn_stats st;
    int rr = (rc < 0 && !done) ? rc : task_result(t, nullptr, &st);
    if (rr < 0) {
      task_destroy(t);
      return rr;
    }
    const double score = probe_score(st);
    if (probe_s) probe_s[k] = score;
    if (bestP == 0 || score < best) {
      best = score;
      bestP = cand[k];
    }
  }
  task_destroy(t);
  *P_best = bestP;
  return PCDN_OK;
}

void pcdn_default_server_opts(pcdn_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->slots = 0;
  o->hbm_budget = int64_t(8) << 30;
  pcdn_default_opts(&o->solve);
}

int pcdn_server_create(const pcdn_server_opts* opts, pcdn_server** out) {
  set_last_error("");
  if (!out) return sfail(PCDN_EINVAL, "out must be given");
  *out = nullptr;
  pcdn_server_opts so;
  if (opts) so = *opts;
  else pcdn_default_server_opts(&so);
  if (so.slots < 0 || so.hbm_budget < 0) return sfail(PCDN_EINVAL, "bad server options");
  int device = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0 || cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return sfail(PCDN_ECUDA, "no CUDA device");
  }
  pcdn_server* s = new (std::nothrow) pcdn_server();
  if (!s) return sfail(PCDN_ENOMEM, "host allocation");
  s->device = device;
  s->slots = so.slots > 0 ? so.slots : default_slots();
  s->budget = so.hbm_budget > 0 ? so.hbm_budget : (int64_t(8) << 30);
  s->opts = so.solve;
  s->t0 = Clock::now();
  int cap = 0;
  if (device_walker_capacity(&cap) != PCDN_OK) {
    delete s;
    return PCDN_ECUDA;
  }
  s->blocks.free = std::max(0, cap - s->slots);
  s->admit_thread = std::thread(admission_loop, s);
  s->drive_thread = std::thread(drive_loop, s);
  for (int k = 0; k < kCreators; ++k) s->creators.emplace_back(creator_loop, s);
  *out = s;
  return PCDN_OK;
}

namespace {
int submit(pcdn_server* s, const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss, int32_t P, double eps,
           uint64_t seed, int64_t* ticket, bool borrow) {
  if (!s || !X || !y || !ticket) return sfail(PCDN_EINVAL, "server, X, y and ticket must be given");
  if (X->n_samples <= 0 || X->n_features <= 0 || X->nnz < 0 || !X->col_ptr || (X->nnz > 0 && (!X->row_idx || !X->val)))
    return sfail(PCDN_EINVAL, "bad CSC");
  if (X->col_ptr[X->n_features] != X->nnz || X->col_ptr[0] != 0) return sfail(PCDN_EINVAL, "col_ptr must run from 0 to nnz");
  if (!(C > 0) || !std::isfinite(C)) return sfail(PCDN_EINVAL, "C must be positive and finite");
  if (loss != PCDN_LOSS_LOGISTIC && loss != PCDN_LOSS_L2SVM) return sfail(PCDN_EINVAL, "unknown loss");
  if (P < 1 || P > X->n_features) return sfail(PCDN_EINVAL, "P must be in [1, n_features]");
  if (!(eps > 0)) return sfail(PCDN_EINVAL, "eps must be positive");
  Request* r = new (std::nothrow) Request();
  if (!r) return sfail(PCDN_ENOMEM, "host allocation");
  if (borrow) {
    r->xcp = X->col_ptr;
    r->xri = X->row_idx;
    r->xv = X->val;
    r->xy = y;
  } else {
    try {
      r->col_ptr.assign(X->col_ptr, X->col_ptr + X->n_features + 1);
      r->row_idx.assign(X->row_idx, X->row_idx + X->nnz);
      r->val.assign(X->val, X->val + X->nnz);
      r->y.assign(y, y + X->n_samples);
    } catch (...) {
      delete r;
      return sfail(PCDN_ENOMEM, "host allocation");
    }
    r->xcp = r->col_ptr.data();
    r->xri = r->row_idx.data();
    r->xv = r->val.data();
    r->xy = r->y.data();
  }
  r->n = X->n_samples;
  r->m = X->n_features;
  r->nnz = X->nnz;
  r->C = C;
  r->loss = (int)loss;
  r->P = P;
  r->eps = eps;
  r->seed = seed;
  r->bytes = problem_bytes_estimate(r->n, r->m, r->nnz, P);
  std::lock_guard<std::mutex> lock(s->mu);
  r->ticket = s->next_ticket++;
  r->t_submit = s->now();
  s->all[r->ticket] = r;
  s->queue.push_back(r);
  s->submitted += 1;
  *ticket = r->ticket;
  s->cv_admit.notify_all();
  return PCDN_OK;
}
}  // namespace

int pcdn_server_submit(pcdn_server* s, const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss, int32_t P,
                       double eps, uint64_t seed, int64_t* ticket) {
  set_last_error("");
  return submit(s, X, y, C, loss, P, eps, seed, ticket, false);
}

int pcdn_server_submit_borrowed(pcdn_server* s, const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss,
                                int32_t P, double eps, uint64_t seed, int64_t* ticket) {
  set_last_error("");
  return submit(s, X, y, C, loss, P, eps, seed, ticket, true);
}

int pcdn_server_wait(pcdn_server* s, int64_t ticket, double timeout_s, double* w_out, pcdn_request_info* info) {
  set_last_error("");
  if (!s) return sfail(PCDN_EINVAL, "server must be given");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return sfail(PCDN_EINVAL, "unknown ticket %lld", (long long)ticket);
  Request* r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                                           timeout_s > 0 ? timeout_s : 1e9));
  while (!r->done) {
    if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && !r->done)
      return sfail(PCDN_ETIMEOUT, "request %lld not finished within the timeout", (long long)ticket);
  }
  if (w_out && !r->w.empty()) std::memcpy(w_out, r->w.data(), sizeof(double) * r->w.size());
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = r->status;
    info->t_submit = r->t_submit;
    info->t_admit = r->t_admit;
    info->t_start = r->t_start;
    info->t_done = r->t_done;
    info->bytes = r->bytes;
    info->stats = r->stats;
    info->P_used = r->P;
    info->retries = r->retries;
  }
  const int status = r->status;
  if (status < 0) set_last_error(r->msg.c_str());
  // the result has been handed over: forget the request; if its problem is still to be destroyed,
  // the admission thread deletes it afterwards
  s->all.erase(it);
  if (r->retired) delete r;
  else r->handed = true;
  return status;
}

int pcdn_server_stats(pcdn_server* s, int64_t* submitted, int64_t* finished, int32_t* in_flight, int64_t* bytes_in_use) {
  if (!s) return sfail(PCDN_EINVAL, "server must be given");
  std::lock_guard<std::mutex> lock(s->mu);
  if (submitted) *submitted = s->submitted;
  if (finished) *finished = s->finished;
  if (in_flight) *in_flight = s->in_flight;
  if (bytes_in_use) *bytes_in_use = s->bytes_in_use;
  return PCDN_OK;
}

void pcdn_server_destroy(pcdn_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    s->cv_admit.notify_all();
    s->cv_create.notify_all();
    s->cv_done.notify_all();
  }
  // the driver ends the stages in flight and hands their problems over for destruction; creators
  // finish the problem they are creating
  if (s->drive_thread.joinable()) s->drive_thread.join();
  s->cv_create.notify_all();
  for (auto& th : s->creators)
    if (th.joinable()) th.join();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (Request* r : s->incoming) s->retire.push_back(r);
    s->incoming.clear();
    s->cv_admit.notify_all();
  }
  // the admission thread destroys every handed-over problem, then stops
  if (s->admit_thread.joinable()) s->admit_thread.join();
  for (Request* r : s->retire) {
    if (r->prob) pcdn_destroy(r->prob);
    r->prob = nullptr;
    if (r->handed) delete r;
  }
  for (auto& kv : s->all) {
    if (kv.second->prob) pcdn_destroy(kv.second->prob);
    delete kv.second;
  }
  delete s;
}

}  // extern "C"
