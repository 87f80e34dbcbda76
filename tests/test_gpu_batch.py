"""Many solves on one GPU, through the C ABI: the batch solver, the bundle-size autotuner and the
request server (continuous batching).  Every result is checked twice: against the same solve run
alone (pcdn_solve with a one-block walker, warm-started along the same C path), and against the
FP64 oracle run along the same path (each C warm-started from the oracle's previous solution,
Algorithm 3 with the same partitions and stop rule).

Tolerances: the final objective of every solve within 1e-6 relative of the oracle's (the bar of the
single solves); batched vs alone within 1e-9 relative in FP64 mode (the same kernels on the same
problem; only the order of the floating-point atomic adds of d^T x_i differs) and 1e-6 in mixed
mode.
"""
import threading
import time

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_4080_gb300 import build
    build.build()
    import paper_1306_4080_gb300 as m
    m.load()
    return m


_CACHE = {}


def batch(count, seed, scale, n_C, C_range=(0.05, 5.0)):
    key = (count, seed, scale, n_C, C_range)
    if key not in _CACHE:
        jobs = datagen.batch_jobs(count, seed=seed, scale=scale, n_C=n_C, C_range=C_range)
        _CACHE[key] = [(j, datagen.generate(j.spec, with_csr=False)) for j in jobs]
    return _CACHE[key]


def oracle_path(p, job, P, eps, seed, max_epochs=400):
    """The oracle along the job's C path, each C warm-started from the previous solution."""
    w, out = None, []
    for C in job.C_path:
        orc = oracle.Oracle.from_problem(p, C, job.loss)
        w, st = orc.solve(P, eps=eps, seed=seed, w0=w, max_epochs=max_epochs)
        assert st["converged"], st
        out.append((w.copy(), st))
    return out


def solo_path(pk, h, m, job, P, eps, seed, prec):
    """The same path with pcdn_solve, one solve at a time, one-block walker."""
    out = []
    for k, C in enumerate(job.C_path):
        pk.pcdn_set_C(h, C)
        opts = pk.pcdn_default_opts(prec=prec, grid_ctas=1, warm_start=1 if k else 0, max_epochs=400)
        rc, w, st, _ = pk.pcdn_solve(h, P, eps, seed, opts, m)
        out.append((w, st))
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_path_matches_solo_and_oracle(pk, prec):
    items = batch(6, seed=1, scale=0.05, n_C=4)
    probs = [pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, j.C_path[0], j.loss) for j, p in items]
    try:
        Ps = [min(64, p.n_features) for _, p in items]
        seeds = [3 + k for k in range(len(items))]
        opts = pk.pcdn_default_opts(prec=prec, max_epochs=400)
        # fewer slots than jobs and two host threads: slots are refilled as jobs finish
        bo = pk.pcdn_default_batch_opts(max_inflight=4, threads=2)
        rc, res, bs = pk.pcdn_solve_batch([q.handle for q in probs], [q.n_features for q in probs],
                                          [j.C_path for j, _ in items], Ps, eps=1e-3, seed=seeds, opts=opts, bopts=bo)
        assert rc == pk.PCDN_OK
        assert bs["solves"] == sum(len(j.C_path) for j, _ in items) and bs["probe_solves"] == 0
        # every solve with an outer iteration replayed them from a captured CUDA graph (a solve that
        # starts at the optimum, e.g. w = 0 at a small C, has none)
        assert bs["graph_solves"] == sum(st["epochs"] > 0 for r in res for st in r["stats"])
        tol_solo = 1e-9 if prec == "fp64" else 1e-6
        for k, ((job, p), q) in enumerate(zip(items, probs)):
            r = res[k]
            assert r["status"] == pk.PCDN_OK and r["P_used"] == Ps[k]
            solo = solo_path(pk, q.handle, q.n_features, job, Ps[k], 1e-3, seeds[k], prec)
            orc = oracle_path(p, job, Ps[k], 1e-3, seeds[k])
            for ci in range(len(job.C_path)):
                st = r["stats"][ci]
                assert st["converged"] and st["walk_grid"] == 1
                Fb, Fs, Fo = st["F_final"], solo[ci][1]["F_final"], orc[ci][1]["F_final"]
                assert abs(Fb - Fs) <= tol_solo * abs(Fs), (k, ci, Fb, Fs)
                assert abs(Fb - Fo) <= 1e-6 * abs(Fo), (k, ci, Fb, Fo)
                if prec == "fp64":
                    assert st["epochs"] == orc[ci][1]["epochs"], (k, ci)
                    wo = orc[ci][0]
                    np.testing.assert_allclose(r["w"][ci], wo, rtol=0, atol=1e-6 * max(1.0, np.abs(wo).max()))
    finally:
        for q in probs:
            q.close()


def test_autotune_picks_a_candidate_and_the_path_still_matches(pk):
    items = batch(4, seed=2, scale=0.05, n_C=3)
    probs = [pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, j.C_path[0], j.loss) for j, p in items]
    try:
        cand = [16, 64, 256]
        opts = pk.pcdn_default_opts(prec="mixed", max_epochs=400)
        bo = pk.pcdn_default_batch_opts(n_candidates=3)  # one probe per size (no layout tuning)
        arr = np.array(cand, dtype=np.int32)
        bo.candidates = arr.ctypes.data
        rc, res, bs = pk.pcdn_solve_batch([q.handle for q in probs], [q.n_features for q in probs],
                                          [j.C_path for j, _ in items], 0, eps=1e-3, seed=5, opts=opts, bopts=bo)
        assert rc == pk.PCDN_OK
        assert bs["probe_solves"] == sum(len([c for c in cand if c <= p.n_features]) for _, p in items)
        for k, (job, p) in enumerate(items):
            P_used = res[k]["P_used"]
            assert P_used in cand and P_used <= p.n_features
            orc = oracle_path(p, job, P_used, 1e-3, 5)
            for ci in range(len(job.C_path)):
                Fb, Fo = res[k]["stats"][ci]["F_final"], orc[ci][1]["F_final"]
                assert abs(Fb - Fo) <= 1e-6 * abs(Fo), (k, ci, Fb, Fo)
        # the single-problem autotuner
        Pb, scores = pk.pcdn_autotune(probs[0].handle, cand, probe_eps=0.1, probe_epochs=3, seed=5, opts=opts)
        assert Pb in cand and np.all(scores[:3] >= 0)
        assert scores[cand.index(Pb)] == scores[:3].min()
    finally:
        for q in probs:
            q.close()


def test_batch_multiblock_walkers(pk):
    """A job with large bundles (svm_20k_100k at P = 1024, about 20k nonzeros per bundle) gets a
    multi-block (cooperative) walker from the block budget, captured in its graph, next to
    one-block jobs; its path matches the oracle's and pcdn_solve's."""
    wl = datagen.workload("svm_20k_100k")
    p_big = datagen.generate(wl.spec, with_csr=False)
    small = batch(3, seed=6, scale=0.03, n_C=2, C_range=(0.5, 1.0))
    path = [0.5, 1.0]
    probs = [pk.Problem.from_csc(p_big.col_ptr, p_big.row_idx, p_big.val, p_big.y, path[0], wl.loss)]
    probs += [pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, j.C_path[0], j.loss) for j, p in small]
    try:
        Ps = [1024] + [min(32, p.n_features) for _, p in small]
        opts = pk.pcdn_default_opts(prec="fp64", max_epochs=400)
        rc, res, bs = pk.pcdn_solve_batch([q.handle for q in probs], [q.n_features for q in probs],
                                          [path] + [j.C_path for j, _ in small], Ps, eps=1e-3, seed=1, opts=opts)
        assert rc == pk.PCDN_OK and bs["solves"] == 2 * len(probs)
        assert bs["graph_solves"] == sum(st["epochs"] > 0 for r in res for st in r["stats"])
        big = res[0]
        assert all(st["walk_grid"] > 1 for st in big["stats"]), [st["walk_grid"] for st in big["stats"]]
        w = None
        for ci, C in enumerate(path):
            orc = oracle.Oracle.from_problem(p_big, C, wl.loss)
            w, so = orc.solve(1024, eps=1e-3, seed=1, w0=w, max_epochs=400)
            Fb = big["stats"][ci]["F_final"]
            assert abs(Fb - so["F_final"]) <= 1e-6 * abs(so["F_final"]), (ci, Fb, so["F_final"])
        solo = solo_path(pk, probs[0].handle, probs[0].n_features, datagen.PathJob("big", wl.spec, wl.loss, path),
                         1024, 1e-3, 1, "fp64")
        for ci in range(len(path)):
            Fb, Fs = big["stats"][ci]["F_final"], solo[ci][1]["F_final"]
            assert abs(Fb - Fs) <= 1e-9 * abs(Fs), (ci, Fb, Fs)
    finally:
        for q in probs:
            q.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_autotune_tries_both_layouts_for_multiblock_sizes(pk, prec):
    """With tune_layout a candidate size whose walker spans several blocks is probed
    with both walker layouts; the job keeps the faster one (layout_used) and its path still matches
    the oracle (the layouts differ only in how d^T x_i reaches the samples)."""
    wl = datagen.workload("svm_20k_100k")
    p = datagen.generate(wl.spec, with_csr=False)
    path = [0.5, 1.0]
    q = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, path[0], wl.loss)
    try:
        arr = np.array([1024], dtype=np.int32)
        bo = pk.pcdn_default_batch_opts(n_candidates=1, tune_layout=1)
        bo.candidates = arr.ctypes.data
        opts = pk.pcdn_default_opts(prec=prec, max_epochs=400)
        rc, res, bs = pk.pcdn_solve_batch([q.handle], [q.n_features], [path], 0, eps=1e-3, seed=1, opts=opts, bopts=bo)
        assert rc == pk.PCDN_OK
        assert bs["probe_solves"] == 2  # P = 1024 with each layout
        other = "rows" if prec == "mixed" else "scatter"
        assert res[0]["P_used"] == 1024 and res[0]["layout_used"] in ("auto", other)
        w = None
        for ci, C in enumerate(path):
            orc = oracle.Oracle.from_problem(p, C, wl.loss)
            w, so = orc.solve(1024, eps=1e-3, seed=1, w0=w, max_epochs=400)
            Fb = res[0]["stats"][ci]["F_final"]
            assert abs(Fb - so["F_final"]) <= 1e-6 * abs(so["F_final"]), (ci, Fb, so["F_final"])
    finally:
        q.close()


def test_batch_rejects_bad_jobs(pk):
    (job, p), = batch(1, seed=3, scale=0.02, n_C=2)
    q = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, 1.0, job.loss)
    try:
        with pytest.raises(pk.PcdnError) as ei:  # the same problem twice
            pk.pcdn_solve_batch([q.handle, q.handle], [q.n_features] * 2, [job.C_path] * 2, 8)
        assert ei.value.code == pk.PCDN_EINVAL
        with pytest.raises(pk.PcdnError) as ei:  # C <= 0
            pk.pcdn_solve_batch([q.handle], [q.n_features], [[1.0, -1.0]], 8)
        assert ei.value.code == pk.PCDN_EINVAL
        with pytest.raises(pk.PcdnError) as ei:  # autotuning from a warm start
            pk.pcdn_solve_batch([q.handle], [q.n_features], [[1.0]], 0, opts=pk.pcdn_default_opts(warm_start=1))
        assert ei.value.code == pk.PCDN_EINVAL
        # a solve that hits max_epochs reports it and still writes its result
        rc, res, _ = pk.pcdn_solve_batch([q.handle], [q.n_features], [[1.0]], 8, eps=1e-12,
                                         opts=pk.pcdn_default_opts(max_epochs=2))
        assert rc == pk.PCDN_ENOTCONVERGED and res[0]["status"] == pk.PCDN_ENOTCONVERGED
        assert res[0]["stats"][0]["epochs"] == 2 and np.all(np.isfinite(res[0]["w"]))
    finally:
        q.close()


class StatsPoller:
    """Samples the server's counters while requests run."""

    def __init__(self, srv):
        self.srv, self.stop, self.max_inflight, self.max_bytes = srv, False, 0, 0
        self.t = threading.Thread(target=self.run)

    def run(self):
        while not self.stop:
            s = self.srv.stats()
            self.max_inflight = max(self.max_inflight, s["in_flight"])
            self.max_bytes = max(self.max_bytes, s["bytes_in_use"])
            time.sleep(0.0005)

    def __enter__(self):
        self.t.start()
        return self

    def __exit__(self, *a):
        self.stop = True
        self.t.join()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_server_result_is_the_same_alone_and_in_the_mix(pk, prec):
    items = batch(12, seed=4, scale=0.04, n_C=1, C_range=(0.5, 0.5))
    P, eps, seed = 32, 1e-3, 7
    target = 5
    opts = pk.pcdn_default_opts(prec=prec, max_epochs=400)
    srv = pk.Server(slots=4, opts=opts)
    try:
        job, p = items[target]
        Pt = min(P, p.n_features)
        t = srv.submit(p.col_ptr, p.row_idx, p.val, p.y, 0.5, job.loss, Pt, eps, seed)
        rc, w_alone, info_alone = srv.wait(t, timeout_s=120)
        assert rc == pk.PCDN_OK
        assert info_alone["t_submit"] <= info_alone["t_admit"] <= info_alone["t_start"] <= info_alone["t_done"]
        tickets = []
        with StatsPoller(srv) as poll:
            for job_k, p_k in items:
                tickets.append(srv.submit(p_k.col_ptr, p_k.row_idx, p_k.val, p_k.y, 0.5, job_k.loss,
                                          min(P, p_k.n_features), eps, seed))
            out = [srv.wait(tk, timeout_s=300) for tk in tickets]
        assert all(o[0] == pk.PCDN_OK for o in out)
        assert 1 < poll.max_inflight <= 4  # requests overlapped, never more than the slots
        rc, w_mix, info_mix = out[target]
        F_alone, F_mix = info_alone["stats"]["F_final"], info_mix["stats"]["F_final"]
        tol = 1e-9 if prec == "fp64" else 1e-6
        assert abs(F_mix - F_alone) <= tol * abs(F_alone), (F_mix, F_alone)
        if prec == "fp64":
            assert info_mix["stats"]["epochs"] == info_alone["stats"]["epochs"]
            np.testing.assert_allclose(w_mix, w_alone, rtol=0, atol=1e-7 * max(1.0, np.abs(w_alone).max()))
        # every request against the oracle
        for (job_k, p_k), (_, w_k, info_k) in zip(items, out):
            orc = oracle.Oracle.from_problem(p_k, 0.5, job_k.loss)
            _, so = orc.solve(min(P, p_k.n_features), eps=eps, seed=seed, max_epochs=400)
            Fk = info_k["stats"]["F_final"]
            assert abs(Fk - so["F_final"]) <= 1e-6 * abs(so["F_final"]), (Fk, so["F_final"])
            assert abs(orc.objective(w_k) - Fk) <= 1e-9 * abs(Fk)
        s = srv.stats()
        assert s["submitted"] == s["finished"] == len(items) + 1
    finally:
        srv.close()


def test_server_admission_respects_the_memory_budget(pk):
    items = batch(8, seed=5, scale=0.03, n_C=1, C_range=(1.0, 1.0))
    P, eps = 16, 1e-3
    # a budget that holds two of the largest of these requests at a time (none exceeds it alone)
    sizes = []
    srv = pk.Server(slots=8, hbm_budget=1 << 40)
    try:
        for job, p in items:
            t = srv.submit(p.col_ptr, p.row_idx, p.val, p.y, 1.0, job.loss, min(P, p.n_features), eps, 0, borrow=True)
            sizes.append(srv.wait(t, 120)[2]["bytes"])
    finally:
        srv.close()
    budget = int(2.2 * max(sizes))
    srv = pk.Server(slots=8, hbm_budget=budget)
    try:
        with StatsPoller(srv) as poll:
            tickets = [srv.submit(p.col_ptr, p.row_idx, p.val, p.y, 1.0, job.loss, min(P, p.n_features), eps, 0)
                       for job, p in items]
            out = [srv.wait(tk, 300) for tk in tickets]
        assert all(o[0] == pk.PCDN_OK for o in out)
        assert poll.max_bytes <= budget, (poll.max_bytes, budget)
        # finished requests release their device memory right after they are collected
        t_end = time.time() + 10
        while srv.stats()["in_flight"] and time.time() < t_end:
            time.sleep(0.001)
        assert srv.stats()["bytes_in_use"] == 0 and srv.stats()["in_flight"] == 0
        # admission in arrival order: no request admitted before an earlier one
        admits = [o[2]["t_admit"] for o in out]
        assert admits == sorted(admits)
    finally:
        srv.close()


def test_server_error_paths(pk):
    """A malformed request finishes with PCDN_EINVAL while the others complete; a wait that times
    out can be repeated; an unknown ticket is an error; destroying a server with requests queued
    and in flight leaves the GPU usable."""
    items = batch(4, seed=7, scale=0.03, n_C=1, C_range=(1.0, 1.0))
    wl = datagen.workload("svm_20k_100k")
    p_big = datagen.generate(wl.spec, with_csr=False)
    srv = pk.Server(slots=2, opts=pk.pcdn_default_opts(max_epochs=300))
    try:
        job, p = items[0]
        bad_rows = p.row_idx.copy()
        bad_rows[len(bad_rows) // 2] = p.n_samples  # row index out of range: caught at admission
        t_bad = srv.submit(p.col_ptr, bad_rows, p.val, p.y, 1.0, job.loss, 8, 1e-3, 0)
        t_ok = [srv.submit(q.col_ptr, q.row_idx, q.val, q.y, 1.0, j.loss, 8, 1e-3, 0) for j, q in items[1:]]
        # a long solve (tight tolerance on a 2M-nonzero problem): its first wait times out
        t_long = srv.submit(p_big.col_ptr, p_big.row_idx, p_big.val, p_big.y, wl.C, wl.loss, 64, 1e-9, 0)
        rc, _, info = srv.wait(t_bad, 120)
        assert rc == pk.PCDN_EINVAL and info["status"] == pk.PCDN_EINVAL
        for t in t_ok:
            assert srv.wait(t, 120)[0] == pk.PCDN_OK
        with pytest.raises(pk.PcdnError) as ei:
            srv.wait(t_long, 0.001)
        assert ei.value.code == pk.PCDN_ETIMEOUT
        rc, w, info = srv.wait(t_long, 600)
        assert rc in (pk.PCDN_OK, pk.PCDN_ENOTCONVERGED) and np.all(np.isfinite(w))
        lib = pk.load()
        assert lib.pcdn_server_wait(srv.handle, 987654, 0.0, None, None) == pk.PCDN_EINVAL
        # requests left queued and in flight when the server is destroyed
        for _ in range(3):
            srv.submit(p_big.col_ptr, p_big.row_idx, p_big.val, p_big.y, wl.C, wl.loss, 64, 1e-9, 0)
        time.sleep(0.2)
    finally:
        srv.close()
    # the device is intact
    q = pk.Problem.from_csc(items[1][1].col_ptr, items[1][1].row_idx, items[1][1].val, items[1][1].y, 1.0, items[1][0].loss)
    try:
        assert q.solve(8, 1e-3, 0)[2]["converged"]
    finally:
        q.close()


def test_server_burst_all_ok_and_matching_the_oracle(pk):
    """A burst of 120 requests submitted at once (ten problems of uneven sizes, both losses, two C
    values each, every pair six times) into a server with the default slots, in mixed precision:
    every request returns PCDN_OK, and its objective is within 1e-6 of the FP64 oracle's at the same
    tolerance (the bar of the single solves); the copies of one pair agree with each other."""
    items = batch(10, seed=11, scale=0.05, n_C=1, C_range=(1.0, 1.0))
    P, eps, seed = 32, 1e-3, 3
    combos = [(k, C) for k in range(len(items)) for C in (0.3, 3.0)]
    opts = pk.pcdn_default_opts(prec="mixed", max_epochs=1000)
    srv = pk.Server(opts=opts)
    try:
        tickets = []
        for rep in range(6):
            for k, C in combos:
                job, p = items[k]
                tickets.append(((k, C), srv.submit(p.col_ptr, p.row_idx, p.val, p.y, C, job.loss,
                                                   min(P, p.n_features), eps, seed, borrow=True)))
        out = [(kc, srv.wait(t, 600)) for kc, t in tickets]
    finally:
        srv.close()
    bad = [(kc, r[0], r[2]["message"]) for kc, r in out if r[0] != pk.PCDN_OK]
    assert not bad, bad
    F_or = {}
    for k, C in combos:
        job, p = items[k]
        orc = oracle.Oracle.from_problem(p, C, job.loss)
        _, so = orc.solve(min(P, p.n_features), eps=eps, seed=seed, max_epochs=1000)
        assert so["converged"]
        F_or[(k, C)] = so["F_final"]
    for kc, (rc, w, info) in out:
        F = info["stats"]["F_final"]
        assert abs(F - F_or[kc]) <= 1e-6 * abs(F_or[kc]), (kc, F, F_or[kc])


def test_server_request_that_stalls_goes_on_with_a_smaller_bundle(pk):
    """A request whose solve reaches max_epochs with P above 16 is continued from the w it reached
    with the next smaller default bundle size (256 -> 64 -> 16): info reports the retries and the
    size used, and its relative KKT value is still measured from w = 0 (checked against the
    oracle's KKT measure at the returned w)."""
    job, p = batch(1, seed=5, scale=0.2, n_C=1, C_range=(2.0, 2.0))[0]
    P0 = 256
    assert p.n_features > P0
    srv = pk.Server(slots=1, opts=pk.pcdn_default_opts(max_epochs=2))
    try:
        t = srv.submit(p.col_ptr, p.row_idx, p.val, p.y, 2.0, job.loss, P0, 1e-9, 0)
        rc, w, info = srv.wait(t, 300)
    finally:
        srv.close()
    assert rc == pk.PCDN_ENOTCONVERGED  # 1e-9 is out of reach in 2 outer iterations per size
    assert info["retries"] == 2 and info["P_used"] == 16
    orc = oracle.Oracle.from_problem(p, 2.0, job.loss)
    k0 = orc.kkt_l1(np.zeros(p.n_features))
    assert info["stats"]["kkt0"] == pytest.approx(k0, rel=1e-9)
    assert info["stats"]["kkt_rel"] == pytest.approx(orc.kkt_l1(w) / k0, rel=1e-6)
