"""Parity at the benchmark's full size: 2,000,000 x 3,000,000 logistic, ~300M nonzeros, P = 4096,
in the launch configuration bench.py times (default options: all blocks of the GPU).

Checked one by one against the FP64 oracle: the partition of two outer iterations (bitwise);
bundle steps sampled from w = 0 and from the state after one outer iteration (both precisions);
and the final objective of whole solves against the oracle's own recorded full solve
(tests/golden/oracle_records.json, written by make_oracle_records.py from the oracle alone).
"""
import json
import os

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_4080_gb300 import build
    build.build()
    import paper_1306_4080_gb300 as pk
    pk.load()
    wl = datagen.workload("lr_2m_3m")
    p = datagen.generate(wl.spec, with_csr=False)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    orc = oracle.Oracle.from_problem(p, wl.C, wl.loss)
    yield pk, wl, p, P, orc
    P.close()


def test_partition_fullsize(env):
    pk, wl, p, P, orc = env
    for epoch in (0, 3):
        np.testing.assert_array_equal(P.permutation(wl.solver_seed, epoch),
                                      oracle.permutation(wl.solver_seed, epoch, p.n_features))


def _compare(r, ro, prec):
    tol = 1e-9 if prec == "fp64" else 1e-5
    gs = max(1e-300, np.abs(ro["g"]).max())
    assert np.abs(r["g"] - ro["g"]).max() <= tol * gs
    assert np.abs(r["h"] - ro["h"]).max() <= tol * np.abs(ro["h"]).max()
    dscale = np.abs(ro["g"]) / ro["h"] + np.abs(ro["d"])
    assert np.all(np.abs(r["d"] - ro["d"]) <= tol * dscale + 1e-300)
    assert abs(r["Delta"] - ro["Delta"]) <= tol * abs(ro["Delta"])
    assert r["q"] == ro["q"] and r["alpha"] == ro["alpha"]
    assert abs(r["dF"] - ro["dF"]) <= (1e-7 if prec == "fp64" else 1e-4) * abs(ro["dF"])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bundle_steps_fullsize(env, prec):
    pk, wl, p, P, orc = env
    opts = pk.pcdn_default_opts(prec=prec)
    # from w = 0: the first two bundles of outer iteration 0
    w0 = np.zeros(p.n_features)
    mq0 = np.ones(p.n_samples)
    perm = oracle.permutation(wl.solver_seed, 0, p.n_features)
    for t in (0, 1):
        B = perm[t * wl.P:(t + 1) * wl.P]
        _compare(P.bundle_step(w0, B, opts), orc.bundle_step(w0, mq0, B)[2], prec)
    # from the state after one outer iteration of the GPU's FP64 solve: a bundle of iteration 1
    _, w1, _, _ = P.solve(wl.P, wl.eps, wl.solver_seed, pk.pcdn_default_opts(max_epochs=1))
    mq1 = orc.maintained(w1)
    perm1 = oracle.permutation(wl.solver_seed, 1, p.n_features)
    B = perm1[5 * wl.P:6 * wl.P]
    _compare(P.bundle_step(w1, B, opts), orc.bundle_step(w1, mq1, B)[2], prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_fullsize_matches_recorded_oracle_solve(env, prec):
    pk, wl, p, P, orc = env
    rec = json.load(open(os.path.join(HERE, "golden", "oracle_records.json")))["lr_2m_3m"]
    assert rec["nnz"] == p.nnz
    _, w, st, tr = P.solve(wl.P, wl.eps, wl.solver_seed, pk.pcdn_default_opts(prec=prec), trace_bundles=4000,
                           trace_epochs=20)
    assert st["converged"]
    rel = abs(st["F_final"] - rec["F_final"]) / abs(rec["F_final"])
    if prec == "fp64":
        assert st["epochs"] == rec["epochs"] and st["bundles"] == rec["bundles"]
        assert rel <= 1e-9, rel
    else:
        assert abs(st["epochs"] - rec["epochs"]) <= 1
        assert rel <= 1e-6, rel
    # Lemma 1(c): no accepted bundle step increases the objective
    assert np.all(tr["dF"] <= 1e-9 * abs(rec["F_final"]))
