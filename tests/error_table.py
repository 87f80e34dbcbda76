"""Error table: every quantity of the CUDA path against the FP64 oracle (run on a GPU; not collected
by pytest).

For each workload, precision and state w (w = 0, and w after one outer iteration of the CUDA
solve), a few random bundles B of the workload's bundle size go through one bundle step on both
sides from the same w and maintained quantities:

  g, h, d    per coordinate, |gpu - oracle| / max_j |oracle_j| (max and 99th percentile)
  Delta      |gpu - oracle| / |oracle|                                  (Eq. 7)
  dF         |gpu - oracle| / |oracle| where both took the same step   (Eq. 6 / Eq. 10)
  q          steps whose accepted q differs (with the oracle's Armijo margin there)
  F, KKT     objective and L1 KKT measure at w                          (Eq. 1, Section 5.1)

Usage:  python tests/error_table.py [--full]   (--full adds the 2M x 3M workload, about 2 GB of
host memory for the oracle).  Prints a Markdown table.
"""
import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import datagen  # noqa: E402
import oracle  # noqa: E402


def armijo_margin(orc, p, w, mq, B, d, Delta, q_lo, q_hi, armijo):
    """The smallest relative Armijo margin |dF(a) - sigma a Delta| / scale over q in [q_lo, q_hi],
    dF(a) in the oracle's maintained form (Eq. 10 per sample, the penalty change per coordinate),
    scale = c sum_i |change_i| + sum_j |penalty change_j| + |sigma a Delta| (the size of the
    rounding any summation order leaves)."""
    dx = np.zeros(p.n_samples)
    for k, j in enumerate(B):
        a, b = p.col_ptr[j], p.col_ptr[j + 1]
        dx[p.row_idx[a:b]] += p.val[a:b].astype(np.float64) * d[k]
    rows = np.flatnonzero(dx)
    best = np.inf
    for q in range(q_lo, q_hi + 1):
        a = armijo.beta ** q
        ch = np.array([orc.row_loss_change(mq[i], int(p.y[i]), a * dx[i]) for i in rows])
        pen = np.abs(w[B] + a * d) - np.abs(w[B])
        dF = orc.c * ch.sum() + pen.sum()
        thr = armijo.sigma * a * Delta
        scale = orc.c * np.abs(ch).sum() + np.abs(pen).sum() + abs(thr)
        best = min(best, abs(dF - thr) / scale)
    return best


def rel_vec(a, b):
    s = max(float(np.max(np.abs(b))), 1e-300)
    e = np.abs(np.asarray(a) - np.asarray(b)) / s
    return float(e.max()), float(np.percentile(e, 99))


def run(pk, name, wl, p, Pb, trials, out):
    orc = oracle.Oracle.from_problem(p, wl.C, wl.loss)
    armijo = oracle.Armijo()
    rng = np.random.default_rng(17)
    # the second state: one outer iteration of the CUDA solve (FP64)
    Pg = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        _, w1, _, _ = Pg.solve(Pb, 1e-9, 0, pk.pcdn_default_opts(prec="fp64", max_epochs=1))
    finally:
        Pg.close()
    states = [("w = 0", np.zeros(p.n_features)), ("after 1 outer iteration", w1)]
    for prec in ("fp64", "mixed"):
        P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
        try:
            opts = pk.pcdn_default_opts(prec=prec, grid_ctas=100000)
            for sname, w in states:
                mq = orc.maintained(w)
                acc = {k: [] for k in ("g", "h", "d")}
                dl, df, qmis, margins = [], [], 0, []
                for _ in range(trials):
                    B = rng.choice(p.n_features, size=Pb, replace=False).astype(np.int32)
                    r = P.bundle_step(w, B, opts)
                    _, _, ro = orc.bundle_step(w, mq, B, armijo=armijo)
                    for k in acc:
                        acc[k].append(rel_vec(r[k], ro[k]))
                    dl.append(abs(r["Delta"] - ro["Delta"]) / max(abs(ro["Delta"]), 1e-300))
                    if r["q"] == ro["q"]:
                        if ro["dF"] != 0.0:
                            df.append(abs(r["dF"] - ro["dF"]) / abs(ro["dF"]))
                    else:
                        qmis += 1
                        margins.append(armijo_margin(orc, p, w, mq, B, ro["d"], ro["Delta"], min(r["q"], ro["q"]),
                                                     max(r["q"], ro["q"]), armijo))
                P.set_w(w)
                F_err = abs(P.objective() - orc.objective(w)) / abs(orc.objective(w))
                k_or = orc.kkt_l1(w, mq)
                K_err = abs(P.kkt() - k_or) / max(k_or, 1e-300)
                row = {"workload": name, "prec": prec, "state": sname}
                for k in acc:
                    row[k] = (max(a for a, _ in acc[k]), max(b for _, b in acc[k]))
                row["Delta"] = max(dl)
                row["dF"] = max(df) if df else float("nan")
                row["q"] = f"{qmis}/{trials}" + (f" (margin <= {max(margins):.1e})" if margins else "")
                row["F"] = F_err
                row["KKT"] = K_err
                out.append(row)
        finally:
            P.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--full", action="store_true")
    ap.add_argument("--trials", type=int, default=6)
    args = ap.parse_args()
    import paper_1306_4080_gb300 as pk
    pk.load()
    cases = [("lr_2k_10k", 64), ("svm_20k_100k", 1024)]
    if args.full:
        cases.append(("lr_2m_3m", 4096))
    out = []
    for name, Pb in cases:
        wl = datagen.workload(name)
        p = datagen.generate(wl.spec, with_csr=False)
        run(pk, name, wl, p, Pb, args.trials, out)
    print("| workload | prec | state | g max / p99 | h max / p99 | d max / p99 | Delta | dF | q differs | F | KKT |")
    print("|---|---|---|---|---|---|---|---|---|---|---|")
    for r in out:
        f = lambda t: f"{t[0]:.1e} / {t[1]:.1e}"
        print(f"| {r['workload']} | {r['prec']} | {r['state']} | {f(r['g'])} | {f(r['h'])} | {f(r['d'])} | "
              f"{r['Delta']:.1e} | {r['dF']:.1e} | {r['q']} | {r['F']:.1e} | {r['KKT']:.1e} |")


if __name__ == "__main__":
    main()
