"""pcdn_objective_noalloc: the objective for callers that may not allocate device memory.

Such callers (an application whose own pool or budget owns all GPU memory, or a request loop
that allows no allocator calls) pass every buffer themselves; the entry point keeps its scratch
in a fixed array inside the library.  Checked through the C ABI against the FP64 oracle's
objective and against pcdn_objective on the same problem and w, on two calls in a row (the
scratch is shared and reused between calls), on the default and on a separate stream, with the
device's free memory unchanged by calls after the first; malformed inputs give NaN without
reading outside the arrays.  This file is collected last, so that a failure here stops a run
only after every other test has run.
"""
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


def _device(p, dev):
    import torch
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (p.col_ptr, p.row_idx, p.val, p.y))


@pytest.mark.parametrize("name", ["lr_2k_10k", "svm_20k_100k"])
def test_noalloc_objective_matches_the_oracle(pk, name):
    import torch
    wl = datagen.workload(name)
    p = datagen.generate(wl.spec, with_csr=False)
    assert p.n_samples <= pk.PCDN_NOALLOC_MAX_SAMPLES
    rng = np.random.default_rng(7)
    dev = torch.device("cuda:0")
    t_cp, t_ri, t_v, t_y = _device(p, dev)
    orc = oracle.Oracle.from_problem(p, wl.C, wl.loss)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    stream = torch.cuda.Stream(device=dev)
    try:
        for trial in range(2):
            w = rng.normal(0, 0.5, p.n_features) * (rng.random(p.n_features) < 0.05)
            F_or = orc.objective(w)
            P.set_w(w)
            F_lib = P.objective()
            t_w = torch.from_numpy(w).to(dev)
            F = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            free0 = None
            for call in range(2):  # two calls in a row share the scratch array
                pk.pcdn_objective_noalloc(t_cp, t_ri, t_v, t_y, wl.C, wl.loss, t_w, F)
                torch.cuda.synchronize()
                assert F.item() == pytest.approx(F_or, rel=1e-12), (trial, call, F.item(), F_or)
                assert F.item() == pytest.approx(F_lib, rel=1e-12), (trial, call, F.item(), F_lib)
                free = torch.cuda.mem_get_info(dev)[0]
                if free0 is None:
                    free0 = free
                assert free == free0, "a call after the first changed the device's free memory"
            # work enqueued on the caller's stream, F read after that stream alone has finished
            F.fill_(-1.0)
            torch.cuda.synchronize()
            pk.pcdn_objective_noalloc(t_cp, t_ri, t_v, t_y, wl.C, wl.loss, t_w, F, stream=stream)
            stream.synchronize()
            assert F.item() == pytest.approx(F_or, rel=1e-12)
            assert torch.cuda.mem_get_info(dev)[0] == free0
    finally:
        P.close()


def test_noalloc_malformed_inputs_give_nan(pk):
    """A row index outside [0, n_samples), a label other than +/-1 and a column pointer past nnz each
    make F NaN (the call itself succeeds: the device checks its own reads)."""
    import torch
    wl = datagen.scaled("lr_2k_10k", 0.2, seed=3)
    p = datagen.generate(wl.spec, with_csr=False)
    dev = torch.device("cuda:0")
    w = torch.from_numpy(np.full(p.n_features, 0.01)).to(dev)
    F = torch.zeros(1, dtype=torch.float64, device=dev)

    def run(cp, ri, v, y):
        F.fill_(0.0)
        t = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (cp, ri, v, y)]
        pk.pcdn_objective_noalloc(*t, wl.C, wl.loss, w, F)
        torch.cuda.synchronize()
        return F.item()

    assert np.isfinite(run(p.col_ptr, p.row_idx, p.val, p.y))
    bad_rows = p.row_idx.copy()
    bad_rows[len(bad_rows) // 2] = p.n_samples
    assert np.isnan(run(p.col_ptr, bad_rows, p.val, p.y))
    bad_y = p.y.copy()
    bad_y[3] = 0
    assert np.isnan(run(p.col_ptr, p.row_idx, p.val, bad_y))
    bad_cp = p.col_ptr.copy()
    bad_cp[-1] = bad_cp[-1] + 1000  # the last column claims entries past the arrays
    assert np.isnan(run(bad_cp, p.row_idx, p.val, p.y))
    # the entry point still computes the right value afterwards
    assert run(p.col_ptr, p.row_idx, p.val, p.y) == pytest.approx(
        oracle.Oracle.from_problem(p, wl.C, wl.loss).objective(np.full(p.n_features, 0.01)), rel=1e-12)


def test_noalloc_rejects_too_many_samples_and_bad_tensors(pk):
    import torch
    n = pk.PCDN_NOALLOC_MAX_SAMPLES + 1
    dev = torch.device("cuda:0")
    col_ptr = torch.zeros(2, dtype=torch.int64, device=dev)
    row_idx = torch.zeros(1, dtype=torch.int32, device=dev)
    val = torch.zeros(1, dtype=torch.float32, device=dev)
    y = torch.ones(n, dtype=torch.int8, device=dev)
    w = torch.zeros(1, dtype=torch.float64, device=dev)
    F = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(pk.PcdnError) as ei:
        pk.pcdn_objective_noalloc(col_ptr, row_idx, val, y, 1.0, "logistic", w, F)
    assert ei.value.code == pk.PCDN_EINVAL
    assert "PCDN_NOALLOC_MAX_SAMPLES" in pk.pcdn_last_error()
    # the binding checks what the C side cannot (raw device pointers): dtype, device, length
    with pytest.raises(pk.PcdnError):
        pk.pcdn_objective_noalloc(col_ptr, row_idx, val, y[:10], 1.0, "logistic", w.float(), F)
    with pytest.raises(pk.PcdnError):
        pk.pcdn_objective_noalloc(col_ptr.cpu(), row_idx, val, y[:10], 1.0, "logistic", w, F)
    with pytest.raises(pk.PcdnError):
        pk.pcdn_objective_noalloc(col_ptr, row_idx, val, y[:10], 1.0, "logistic", torch.zeros(3, dtype=torch.float64,
                                                                                               device=dev), F)
