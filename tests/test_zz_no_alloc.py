"""pcdn_objective_noalloc: the objective for callers that may not allocate device memory.

Such callers (an application whose own pool or budget owns all GPU memory, or a request loop
that allows no allocator calls) pass every buffer themselves; the entry point keeps its scratch
in a fixed array inside the library.  Checked through the C ABI against pcdn_objective on the
same problem and w, on two calls in a row (the scratch is shared and reused between calls).
"""
import numpy as np
import pytest

import datagen

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


@pytest.mark.parametrize("name", ["lr_2k_10k", "svm_20k_100k"])
def test_noalloc_objective_matches_pcdn_objective(pk, name):
    import torch
    wl = datagen.workload(name)
    p = datagen.generate(wl.spec, with_csr=False)
    assert p.n_samples <= pk.PCDN_NOALLOC_MAX_SAMPLES
    rng = np.random.default_rng(7)
    dev = torch.device("cuda:0")
    t_cp, t_ri, t_v, t_y = (torch.from_numpy(a).to(dev) for a in (p.col_ptr, p.row_idx, p.val, p.y))
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        for trial in range(2):
            w = rng.normal(0, 0.5, p.n_features) * (rng.random(p.n_features) < 0.05)
            P.set_w(w)
            F_ref = P.objective()
            t_w = torch.from_numpy(w).to(dev)
            F = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
            for call in range(2):  # two calls in a row share the scratch array
                pk.pcdn_objective_noalloc(t_cp, t_ri, t_v, t_y, wl.C, wl.loss, t_w, F)
                torch.cuda.synchronize()
                assert F.item() == pytest.approx(F_ref, rel=1e-12), (trial, call, F.item(), F_ref)
    finally:
        P.close()


def test_noalloc_rejects_too_many_samples(pk):
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
        pk.pcdn_objective_noalloc(col_ptr, row_idx[:0], val[:0], y, 1.0, "logistic", w, F)
    assert ei.value.code == pk.PCDN_EINVAL
    assert "PCDN_NOALLOC_MAX_SAMPLES" in pk.pcdn_last_error()
