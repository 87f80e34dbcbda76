#!/usr/bin/env python
"""Benchmark of the GB300 PCDN solver: time to relative KKT 1e-3 on the 2M x 3M logistic workload.

One step = one full solve from w = 0 (Algorithm 3 with Algorithm 4, every bundle step, the
per-outer-iteration refresh and KKT test) to relative minimum-norm subgradient <= 1e-3.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line.  `value` is seconds per solve (lower is better) with the inputs resident in
HBM, timed by CUDA events on the library's stream; `e2e` is the same through the C ABI from host
buffers (host->device copy of X and y, device set-up, solve, copy of w back).  `roofline` reports
the bundle walker (the dominant kernel): algorithmic bytes of its bundle steps (16 nnz_B +
33 |U_B| + 16 P per bundle) over its CUDA-event time, against the measured HBM copy bandwidth.
`cpu_baseline` times the FP64 CPU oracle on a bounded sample of the same workload and projects it
to a whole solve.  Under torchrun each rank solves its own replica (no collective on the data
path); `value` is then the slowest rank's time divided by the number of solves in flight.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# one hardware work queue per concurrent solve of the batched and served legs (read when the CUDA
# context is created, so before torch touches the GPU)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "time-to-eps (KKT 1e-3) & bundle-step HBM GB/s vs peak; batched/served vs plain"
UNIT = "s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lr_2m_3m")
    ap.add_argument("--scale", type=float, default=1.0, help="scale n and m of the workload (profiling runs)")
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--also-fp64", type=int, default=1, help="also time the FP64 mode (reported under 'fp64')")
    ap.add_argument("--also-shrink", type=int, default=1,
                    help="also time solves that shrink between outer iterations (reported under 'shrinking')")
    ap.add_argument("--max-epochs", type=int, default=1000)
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--cpu-bundles", type=int, default=0, help="oracle sample size in bundles (0 = auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--grid", type=int, default=0)
    ap.add_argument("--layout", default="auto", choices=["auto", "scatter", "rows"],
                    help="how d^T x reaches the samples (pcdn_opts.layout)")
    ap.add_argument("--batched", type=int, default=1, help="also run the batched workload (reported under 'batched')")
    ap.add_argument("--batch-jobs", type=int, default=64)
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--batch-nC", type=int, default=16)
    ap.add_argument("--serving", type=int, default=1, help="also run the request server (reported under 'serving')")
    ap.add_argument("--serve-rates", default="10,30,100,300,1000")
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="arrival window per rate (requests = rate x this, capped)")
    ap.add_argument("--serve-max-requests", type=int, default=200)
    ap.add_argument("--batch-plain-every", type=int, default=1,
                    help="one-at-a-time comparison on every k-th job (batched again on the same jobs); 1 = all")
    ap.add_argument("--serve-seq", type=int, default=40, help="requests timed through the sequential plain loop")
    ap.add_argument("--main", type=int, default=1, help="run the 2M x 3M solve (the headline metric)")
    return ap.parse_args()


def workload(args):
    import datagen
    if args.scale != 1.0:
        return datagen.scaled(args.workload, args.scale)
    return datagen.workload(args.workload)


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def walker_source_hash(layout: str = "scatter"):
    """Hash of a walker's sources (its kernel and the header with its constants)."""
    h = hashlib.sha256()
    for f in ({"scatter": "pcdn_walk.cu", "rows": "pcdn_walk_rows.cu"}[layout], "pcdn_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1306_4080_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


WALKERS = {"scatter": "pcdn::walk_kernel", "rows": "pcdn::rows::walk_rows_kernel"}


def walker_layout(requested: str, prec: str, grid: int) -> str:
    """The walker a solve ran: the requested layout, else the library's default (row-sorted for
    FP64 on more than one block, scatter otherwise)."""
    if requested in WALKERS:
        return requested
    return "rows" if (prec == "fp64" and grid > 1) else "scatter"


def walker_traffic(layout: str):
    """DRAM bytes per walker launch from the committed ncu summary of that walker, if it was taken
    on the current walker sources; else None."""
    path = os.path.join(ROOT, "profiles", "walk_traffic.json")
    try:
        d = json.load(open(path)).get(layout)
        if not d or d.get("walk_source_sha256_16") != walker_source_hash(layout):
            return None
        return d
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        rows = []
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            if self.uuid and self.uuid not in f[1]:
                continue
            rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_uuid(dev):
    import torch
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def cpu_sample(prob, wl, bundles_total, epochs_total, n_bundles, openmp=False):
    """The FP64 oracle as it stands, single-threaded (or its OpenMP variant, the paper's shared-memory
    scheme on all host cores): the set-up of a solve (refresh + KKT at w = 0, which is also the
    per-outer-iteration cost) and the first n_bundles bundle steps, projected to a whole solve of
    bundles_total bundles over epochs_total outer iterations."""
    import oracle
    o = oracle.Oracle.from_problem(prob, wl.C, wl.loss)
    solve = o.solve_omp if openmp else o.solve
    t0 = time.perf_counter()
    solve(wl.P, eps=wl.eps, seed=wl.solver_seed, bundle_limit=0)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    solve(wl.P, eps=wl.eps, seed=wl.solver_seed, bundle_limit=n_bundles)
    t_run = time.perf_counter() - t0
    per_bundle = max(0.0, t_run - t_setup) / n_bundles
    projected = t_setup * (epochs_total + 1) + per_bundle * bundles_total
    if openmp:
        cores = oracle.omp_threads()
        return dict(value=projected, unit=UNIT, cores=cores, kind="oracle-openmp",
                    sample=f"the oracle's algorithm with the paper's shared-memory parallel scheme (OpenMP, {cores} "
                           f"threads, FP64) on {n_bundles} bundles of outer iteration 0 plus one solve set-up, "
                           f"projected to {bundles_total} bundles and {epochs_total} outer iterations: per bundle "
                           f"{per_bundle * 1e3:.3f} ms, per outer-iteration refresh+KKT {t_setup:.3f} s",
                    per_bundle_s=per_bundle, setup_s=t_setup)
    return dict(value=projected, unit=UNIT, cores=1, kind="oracle",
                sample=f"oracle (1 thread, FP64) on {n_bundles} bundles of outer iteration 0 plus one solve set-up "
                       f"(refresh + KKT) of this workload, projected to {bundles_total} bundles and "
                       f"{epochs_total} outer iterations: per bundle {per_bundle * 1e3:.3f} ms, per outer-iteration "
                       f"refresh+KKT {t_setup:.3f} s; sample wall {t_setup + t_run:.1f} s",
                per_bundle_s=per_bundle, setup_s=t_setup)


def oracle_record(name):
    path = os.path.join(ROOT, "tests", "golden", "oracle_records.json")
    try:
        return json.load(open(path))[name]
    except Exception:
        return None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    import datagen
    wl = workload(args)
    prob = datagen.generate(wl.spec, with_csr=False)
    rec = oracle_record(wl.name)
    if rec is not None:
        bundles_total, epochs_total, basis = rec["bundles"], rec["epochs"], "oracle's own full solve (recorded)"
    else:
        nb = (prob.n_features + wl.P - 1) // wl.P
        bundles_total, epochs_total, basis = nb * 10, 10, "assumed 10 outer iterations"
    nbun = args.cpu_bundles or max(8, min(200, (prob.n_features + wl.P - 1) // wl.P))
    vals = []
    last = None
    for i in range(args.warmup + args.steps):
        last = cpu_sample(prob, wl, bundles_total, epochs_total, nbun)
        if i >= args.warmup:
            vals.append(last["value"])
    v = statistics.mean(vals)
    cb = {k: last[k] for k in ("kind", "cores", "sample")}
    cb["value"] = v
    cb["unit"] = UNIT
    cb["projection_basis"] = basis
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, prob, "fp64"), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_of(wl, prob, prec):
    if wl.spec.kind == "zipf":
        shape = f"Zipf {wl.spec.zipf_s} columns, tf-idf rows L2-normalised"
    else:
        shape = f"uniform density {wl.spec.density}, |N(0,1)| values, rows L2-normalised"
    return {"workload": f"{wl.name}: L1 {wl.loss}, n_samples={prob.n_samples}, n_features={prob.n_features}, "
                        f"nnz={prob.nnz}, {shape}, C={wl.C}, P={wl.P}, eps={wl.eps}",
            "n_samples": prob.n_samples, "n_features": prob.n_features, "nnz": prob.nnz, "loss": wl.loss,
            "C": wl.C, "P": wl.P, "eps": wl.eps, "precision": prec,
            "cache": "inputs larger than L2 (X alone is %.2f GB)" % (prob.nnz * 8 / 1e9)}


def batch_pool(args):
    """The batched workload: problems of uneven sizes, each along a 16-value C path."""
    import datagen
    jobs = datagen.batch_jobs(args.batch_jobs, seed=0, scale=args.batch_scale, n_C=args.batch_nC)
    return [(j, datagen.generate(j.spec, with_csr=False)) for j in jobs]


def run_batched(args, pk, pool):
    """Every job's whole C path (warm-started, FP32 bulk / FP64 line search, relative KKT 1e-3)
    through pcdn_solve_batch, bundle size autotuned per job (probes included in the time).  The
    one-at-a-time comparison runs on every k-th job: the same paths solve by solve through
    pcdn_solve with the bundle sizes the autotuner chose, and the batch again on just those jobs.
    Host wall time around each arm; inputs resident on the device."""
    import torch
    probs = [pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, j.C_path[0], j.loss) for j, p in pool]

    def batch(idx, P):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, res, bs = pk.pcdn_solve_batch([probs[k].handle for k in idx], [probs[k].n_features for k in idx],
                                          [pool[k][0].C_path for k in idx], P, eps=1e-3, seed=0,
                                          opts=pk.pcdn_default_opts(prec="mixed", max_epochs=args.max_epochs),
                                          want_w=False)
        return time.perf_counter() - t0, rc, res, bs

    try:
        every = max(1, args.batch_plain_every)
        all_idx = list(range(len(pool)))
        t_batch, rc, res, bs = batch(all_idx, 0)
        Ps = [r["P_used"] for r in res]
        launches = sum(st["kernel_launches"] for r in res for st in r["stats"])
        sub = all_idx[::every]
        if every == 1:
            t_sub, res_sub = t_batch, res
        else:
            t_sub, _, res_sub, _ = batch(sub, [Ps[k] for k in sub])
        F_batch = [[st["F_final"] for st in r["stats"]] for r in res_sub]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F_plain, epochs_plain, conv = [], 0, True
        for k in sub:
            q, job = probs[k], pool[k][0]
            row = []
            for ci, C in enumerate(job.C_path):
                pk.pcdn_set_C(q.handle, C)
                o = pk.pcdn_default_opts(prec="mixed", max_epochs=args.max_epochs, warm_start=1 if ci else 0,
                                         layout=res[k]["layout_used"])
                _, _, st, _ = pk.pcdn_solve(q.handle, Ps[k], 1e-3, 0, o, q.n_features, want_w=False)
                row.append(st["F_final"])
                epochs_plain += st["epochs"]
                conv = conv and bool(st["converged"])
            F_plain.append(row)
        t_plain = time.perf_counter() - t0
        diff = max(abs(a - b) / abs(b) for ra, rb in zip(F_batch, F_plain) for a, b in zip(ra, rb))
        # per job: its path's host time inside the batch (sum of its solves), size, bundle size
        jobs_diag = []
        for r, (job, p) in zip(res, pool):
            sts = r["stats"]
            bund = sum(st["bundles"] for st in sts)
            walk = sum(st["walk_s"] for st in sts)
            jobs_diag.append({"path_s": sum(st["wall_s"] for st in sts), "n": p.n_samples, "m": p.n_features,
                              "nnz": p.nnz, "loss": job.loss, "P": r["P_used"], "epochs": sum(st["epochs"] for st in sts),
                              "bundles": bund, "walk_blocks_max": max(st["walk_grid"] for st in sts),
                              "walk_us_per_bundle": walk / bund * 1e6 if bund else 0.0})
        crit = sorted(jobs_diag, key=lambda d: -d["path_s"])
        n_solves = sum(len(j.C_path) for j, _ in pool)
        # throughput counts the solves that reached the tolerance, nothing else
        n_conv = sum(1 for r in res for st in r["stats"] if st["converged"])
        n_sub = sum(len(pool[k][0].C_path) for k in sub)
        nnz = [p.nnz for _, p in pool]
        return ({"metric": "solves/s (whole C paths, relative KKT 1e-3)", "unit": "solves/s",
                 "value": n_conv / t_batch, "batch_s": t_batch, "solves": n_solves, "solves_converged": n_conv,
                 "status": rc, "job_statuses": {str(s_): sum(1 for r in res if r["status"] == s_)
                                                for s_ in sorted({r["status"] for r in res})},
                 "retries": bs["retries"],
                 "probe_solves": bs["probe_solves"], "epochs_batched": bs["epochs"], "gpu_launches": int(launches),
                 "graph_solves": bs["graph_solves"],
                 "vs_plain": {"jobs": len(sub), "solves": n_sub, "batched_s": t_sub, "plain_s": t_plain,
                              "batched_solves_per_s": n_sub / t_sub, "plain_solves_per_s": n_sub / t_plain,
                              "speedup": t_plain / t_sub, "plain_converged": conv, "epochs_plain": epochs_plain,
                              "max_rel_F_diff": diff,
                              "how": f"every {every}-th job; plain = pcdn_solve one solve at a time, same bundle sizes, "
                                     "its own choice of walker blocks"},
                 "P_chosen": {str(P): Ps.count(P) for P in sorted(set(Ps))},
                 "layout_chosen": {k: sum(1 for r in res if r["layout_used"] == k)
                                   for k in sorted({r["layout_used"] for r in res})},
                 "critical_jobs": crit[:2], "sum_path_s": sum(d["path_s"] for d in jobs_diag),
                 "config": {"workload": f"{len(pool)} problems, n_samples log-uniform [1k, 50k] x {args.batch_scale:g}, "
                                        f"n_features log-uniform [5k, 200k] x {args.batch_scale:g}, density U[0.1%, 1%], "
                                        "Zipf 1.1 columns, tf-idf rows L2-normalised, losses alternating logistic / "
                                        f"L2-SVM, each along {args.batch_nC} C values log-spaced over [1e-2, 1e1] "
                                        "(warm-started)", "nnz_total": int(sum(nnz)), "nnz_max": int(max(nnz)),
                            "precision": "mixed", "bundle_size": "autotuned per problem (probes timed)"}}, Ps)
    finally:
        for q in probs:
            q.close()


def run_serving(args, pk, pool, P_of):
    """Poisson arrivals of single solves drawn from the batched workload's problems (loss of the
    problem, C log-uniform over [1e-2, 1e1]) into a request server with an 8 GiB device budget;
    latency = submit to result on the host.  Baseline: the same requests one at a time
    (pcdn_create + pcdn_solve + pcdn_destroy)."""
    import numpy as np
    rates = [float(r) for r in args.serve_rates.split(",") if r]
    out = {"metric": "solves/s and p50/p99 latency to relative KKT 1e-3", "budget_bytes": 8 << 30, "rates": []}
    opts = pk.pcdn_default_opts(prec="mixed", max_epochs=args.max_epochs)
    rng = np.random.default_rng(12345)
    draws = []
    for rate in rates:
        R = int(min(args.serve_max_requests, max(20, rate * args.serve_seconds)))
        gaps = rng.exponential(1.0 / rate, size=R)
        picks = rng.integers(0, len(pool), size=R)
        Cs = 10.0 ** rng.uniform(-2.0, 1.0, size=R)
        draws.append((rate, R, gaps, picks, Cs))
    for rate, R, gaps, picks, Cs in draws:
        srv = pk.Server(slots=0, hbm_budget=8 << 30, opts=opts)
        try:
            tickets = []
            t0 = time.perf_counter()
            t_next = t0
            for k in range(R):
                t_next += gaps[k]
                d = t_next - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                job, p = pool[picks[k]]
                tickets.append(srv.submit(p.col_ptr, p.row_idx, p.val, p.y, float(Cs[k]), job.loss, P_of[picks[k]],
                                          1e-3, 0, borrow=True))
            submit_lag = time.perf_counter() - t0 - float(np.sum(gaps))
            res = [srv.wait(t, 600) for t in tickets]
            lat = np.array([r[2]["t_done"] - r[2]["t_submit"] for r in res])
            queue = np.array([r[2]["t_admit"] - r[2]["t_submit"] for r in res])
            create = np.array([r[2]["t_start"] - r[2]["t_admit"] for r in res])
            solve = np.array([r[2]["t_done"] - r[2]["t_start"] for r in res])
            first = min(r[2]["t_submit"] for r in res)
            last = max(r[2]["t_done"] for r in res)
            ok = sum(1 for r in res if r[0] == pk.PCDN_OK)  # converged to the tolerance, nothing else
            statuses = {}
            for r in res:
                statuses[str(r[0])] = statuses.get(str(r[0]), 0) + 1
            errors = sorted({r[2].get("message", "") for r in res if r[0] < 0})[:5]
            failed = [{"request": k, "problem": int(picks[k]), "C": float(Cs[k]), "loss": pool[picks[k]][0].loss,
                       "status": int(res[k][0])} for k in range(R) if res[k][0] != pk.PCDN_OK][:8]
            retried = sum(1 for r in res if r[2].get("retries", 0) > 0)
            out["rates"].append({"rate_per_s": rate, "requests": R, "ok": ok, "statuses": statuses, "errors": errors,
                                 "failed": failed, "retried_smaller_P": retried,
                                 "not_converged": sum(1 for r in res if r[0] == pk.PCDN_ENOTCONVERGED),
                                 "solves_per_s": ok / (last - first),
                                 "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                                 "max_s": float(lat.max()),
                                 "mean_s": float(lat.mean()), "mean_queue_s": float(queue.mean()),
                                 "mean_create_s": float(create.mean()), "mean_solve_s": float(solve.mean()),
                                 "submit_lag_s": float(submit_lag)})
        finally:
            srv.close()
    # sequential plain loop on the first requests of the highest rate's draw
    rate, R, gaps, picks, Cs = draws[-1]
    S = min(args.serve_seq, R)
    t0 = time.perf_counter()
    lat = []
    for k in range(S):
        job, p = pool[picks[k]]
        ts = time.perf_counter()
        h = pk.pcdn_create(p.col_ptr, p.row_idx, p.val, p.y, float(Cs[k]), job.loss)
        pk.pcdn_solve(h, P_of[picks[k]], 1e-3, 0, opts, p.n_features, want_w=True)
        pk.pcdn_destroy(h)
        lat.append(time.perf_counter() - ts)
    t_seq = time.perf_counter() - t0
    out["sequential_plain"] = {"requests": S, "solves_per_s": S / t_seq, "mean_s": float(np.mean(lat)),
                               "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99))}
    best = max(r["solves_per_s"] for r in out["rates"])
    out["speedup_vs_sequential"] = best / out["sequential_plain"]["solves_per_s"]
    out["config"] = {"workload": f"Poisson arrivals at {args.serve_rates}/s of single solves drawn from the "
                                 f"{len(pool)} batched problems (their loss, C log-uniform [1e-2, 1e1], their autotuned "
                                 "bundle size), mixed precision, 8 GiB device budget, slots 2 per SM (at most 128)"}
    return out


def init_replicas():
    """One process per GPU under torchrun: each rank solves its own replica of the workload (no
    collective on the data path).  Returns the process group module, or None for one process.
    NCCL with a GPU, gloo without (the host-side logic is tested that way)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return dist


def slowest_rank_ms(ms, dist, device=None):
    """The largest per-rank time (the job's time: every rank's replica must finish)."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import numpy as np
    import torch

    import datagen
    import paper_1306_4080_gb300 as pk

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = init_replicas()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pk.load()

    if not args.main:
        line = {"metric": METRIC, "n_gpus": world, "config": {}}
        if rank == 0:
            add_extra_legs(args, pk, line)
            print(json.dumps(line), flush=True)
        return 0

    wl = workload(args)
    prob = datagen.generate(wl.spec, with_csr=False)
    stream = torch.cuda.Stream(device=dev)
    t_cp = torch.from_numpy(prob.col_ptr).to(dev)
    t_ri = torch.from_numpy(prob.row_idx).to(dev)
    t_v = torch.from_numpy(prob.val).to(dev)
    t_y = torch.from_numpy(prob.y).to(dev)
    torch.cuda.synchronize()
    P = pk.Problem.from_device(t_cp, t_ri, t_v, t_y, wl.C, wl.loss, stream=stream)

    def timed(prec, steps, warmup, shrink=0):
        opts = pk.pcdn_default_opts(prec=prec, max_epochs=args.max_epochs, grid_ctas=args.grid, shrink=shrink,
                                    layout=args.layout)
        for _ in range(warmup):
            P.solve(wl.P, wl.eps, wl.solver_seed, opts, want_w=False)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        sts = []
        with ClockSampler(gpu_uuid(dev)) as clk:
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(steps):
                _, _, st, _ = P.solve(wl.P, wl.eps, wl.solver_seed, opts, want_w=False)
                sts.append(st)
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        if dist:
            ms = slowest_rank_ms(ms, dist, dev)
            dist.barrier()
        return ms, sts, clk.summary()

    ms, sts, clocks = timed(args.prec, args.steps, args.warmup)
    st0 = sts[-1]
    walk_s = sum(s["walk_s"] for s in sts)
    walk_launches = sum(s["epochs"] for s in sts)
    bytes_model = sum(s["bytes_model"] for s in sts)
    launches = sum(s["kernel_launches"] for s in sts)
    peak, peak_src = measured_peak()
    achieved = bytes_model / walk_s / 1e9 if walk_s > 0 else 0.0
    layout = walker_layout(args.layout, args.prec, int(st0["walk_grid"]))
    tr = walker_traffic(layout)
    ms_launch = walk_s / walk_launches * 1e3
    traffic = (tr["dram_bytes_per_launch"] * (bytes_model / walk_launches) / tr["bytes_model_per_launch"]) if tr else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic,
            # DRAM bytes the kernel really moved (ncu, scaled to this launch) per launch time, of peak
            "dram_frac": (traffic / (ms_launch * 1e-3) / 1e9 / peak) if traffic else None,
            "kernel": WALKERS[layout] + " (one launch per outer iteration)", "layout": layout,
            "peak_source": f"{peak_src} HBM copy bandwidth",
            "bytes_per_launch": bytes_model / walk_launches, "ms_per_launch": ms_launch,
            "walk_share_of_step": walk_s / (ms * 1e-3 * len(sts))}
    if tr:
        roof["traffic_source"] = tr.get("source")

    extra = {}
    if args.also_fp64 and args.prec != "fp64":
        ms64, sts64, clk64 = timed("fp64", max(1, min(args.steps, 3)), 1)
        s64 = sts64[-1]
        lay64 = walker_layout(args.layout, "fp64", int(s64["walk_grid"]))
        ach64 = sum(s["bytes_model"] for s in sts64) / sum(s["walk_s"] for s in sts64) / 1e9
        tr64 = walker_traffic(lay64)
        bpl64 = sum(s["bytes_model"] for s in sts64) / sum(s["epochs"] for s in sts64)
        mpl64 = sum(s["walk_s"] for s in sts64) / sum(s["epochs"] for s in sts64) * 1e3
        traf64 = tr64["dram_bytes_per_launch"] * bpl64 / tr64["bytes_model_per_launch"] if tr64 else None
        extra["fp64"] = {"value": ms64 * 1e-3 / world, "unit": UNIT, "ms_per_step": ms64, "epochs": s64["epochs"],
                         "F_final": s64["F_final"], "kkt_rel": s64["kkt_rel"], "layout": lay64,
                         "kernel": WALKERS[lay64],
                         "walk_ms_per_launch": mpl64,
                         "achieved_GBps": ach64, "frac": ach64 / peak, "traffic": traf64,
                         "dram_frac": (traf64 / (mpl64 * 1e-3) / 1e9 / peak) if traf64 else None, "clocks": clk64,
                         "note": "like-for-like with the FP64 reference arm: every quantity in FP64"}

    if args.also_shrink:
        # the same solve with shrinking between outer iterations (an option; the headline solve visits
        # every feature in every outer iteration, as Algorithm 3 does)
        mss, stss, clks = timed(args.prec, max(1, min(args.steps, 3)), 1, shrink=1)
        ss = stss[-1]
        _, _, _, trs = P.solve(wl.P, wl.eps, wl.solver_seed,
                               pk.pcdn_default_opts(prec=args.prec, max_epochs=args.max_epochs, grid_ctas=args.grid,
                                                    shrink=1, layout=args.layout), want_w=False, trace_epochs=200)
        extra["shrinking"] = {"value": mss * 1e-3 / world, "unit": UNIT, "ms_per_step": mss,
                              "speedup_vs_plain": ms / mss, "epochs": ss["epochs"], "bundles": ss["bundles"],
                              "coord_updates": ss["coord_updates"], "nnz_visited": ss["nnz_visited"],
                              "features_first_outer_iterations": [int(x) for x in trs["epoch_features"][:6]],
                              "F_final": ss["F_final"], "F_plain": st0["F_final"], "kkt_rel": ss["kkt_rel"],
                              "walk_ms": ss["walk_s"] * 1e3, "clocks": clks}

    e2e = None
    if not args.no_e2e:
        cp, ri, vv, yy = prob.col_ptr, prob.row_idx, prob.val, prob.y
        pin = [torch.from_numpy(a).pin_memory().numpy() for a in (cp, ri, vv, yy)]
        opts = pk.pcdn_default_opts(prec=args.prec, max_epochs=args.max_epochs, grid_ctas=args.grid,
                                    layout=args.layout)
        times = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = pk.pcdn_create(*pin, wl.C, wl.loss)
            _, w, _, _ = pk.pcdn_solve(h, wl.P, wl.eps, wl.solver_seed, opts, prob.n_features)
            pk.pcdn_destroy(h)
            t1 = time.perf_counter()
            if i > 0:
                times.append(t1 - t0)
        h2d = cp.nbytes + ri.nbytes + vv.nbytes + yy.nbytes
        e2e = {"value": statistics.mean(times) / world, "unit": UNIT, "min": min(times), "max": max(times),
               "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(8 * prob.n_features + 8), "steps": len(times),
               "includes": "pcdn_create from pinned host CSC + row-mirror build + solve + w to host + destroy"}

    cpu = cpu_omp = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nbun = args.cpu_bundles or max(8, min(200, (prob.n_features + wl.P - 1) // wl.P))
        cpu = cpu_sample(prob, wl, int(st0["bundles"]), int(st0["epochs"]), nbun)
        cpu.pop("per_bundle_s", None)
        cpu.pop("setup_s", None)
        cpu_omp = cpu_sample(prob, wl, int(st0["bundles"]), int(st0["epochs"]), nbun, openmp=True)
        cpu_omp.pop("per_bundle_s", None)
        cpu_omp.pop("setup_s", None)

    P.close()
    if rank == 0:
        line = {"metric": METRIC, "value": ms * 1e-3 / world, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32/f64 mixed" if args.prec == "mixed" else "f64",
                "data": "synthetic (seeded generator, shapes of the paper's sparse text workloads)",
                "config": config_of(wl, prob, args.prec)}
        # the FP64 solve right after the headline, so that both precisions lead the line
        if "fp64" in extra:
            line["fp64"] = extra.pop("fp64")
        line.update({"roofline": roof, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
                     "cpu_baseline": cpu, "cpu_baseline_openmp": cpu_omp,
                     "solve": {"epochs": st0["epochs"], "bundles": st0["bundles"], "F_final": st0["F_final"],
                               "kkt_rel": st0["kkt_rel"], "coord_updates_per_s": st0["coord_updates"] / (ms * 1e-3),
                               "ls_steps": st0["ls_steps"], "ls_cap_hits": st0["ls_cap_hits"],
                               "rows_touched": st0["rows_touched"]}})
        line.update(extra)
        if world == 1:
            add_extra_legs(args, pk, line)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def add_extra_legs(args, pk, line):
    """The batched and serving workloads (one GPU), added to the JSON line."""
    if not (args.batched or args.serving):
        return
    pool = batch_pool(args)
    # serving requests use the bundle size the batch's autotuner chose for their problem
    P_of = [min(64, p.n_features) for _, p in pool]
    if args.batched:
        line["batched"], P_of = run_batched(args, pk, pool)
    if args.serving:
        line["serving"] = run_serving(args, pk, pool, P_of)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
