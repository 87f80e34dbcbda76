"""Synthetic input generator: shape, layout and label recipe (CPU)."""
import numpy as np
import pytest

import datagen


@pytest.mark.parametrize("name", ["lr_2k_10k", "svm_20k_100k"])
def test_preset_layout(name):
    wl = datagen.workload(name)
    p = datagen.generate(wl.spec)
    n, m = p.n_samples, p.n_features
    assert p.col_ptr.shape == (m + 1,) and p.col_ptr[0] == 0 and np.all(np.diff(p.col_ptr) >= 0)
    assert p.row_idx.dtype == np.int32 and p.val.dtype == np.float32 and p.y.dtype == np.int8
    assert set(np.unique(p.y).tolist()) <= {-1, 1}
    # rows ascending inside every column, indices in range
    d = np.diff(p.row_idx.astype(np.int64))
    starts = p.col_ptr[1:-1]
    mask = np.ones(d.shape[0], dtype=bool)
    mask[starts[(starts > 0) & (starts < p.nnz)] - 1] = False
    assert np.all(d[mask] > 0)
    assert p.row_idx.min() >= 0 and p.row_idx.max() < n
    # rows L2-normalised (non-empty rows)
    rn = np.zeros(n)
    np.add.at(rn, p.row_idx, p.val.astype(np.float64) ** 2)
    nz = np.diff(p.row_ptr) > 0
    np.testing.assert_allclose(rn[nz], 1.0, rtol=1e-5)
    # CSR mirror holds the same entries
    assert p.nnz == int(p.row_ptr[-1])
    # labels: sign(X w*) with exactly round(frac * n) flips
    wd = np.zeros(m)
    wd[p.wstar_idx] = p.wstar_val
    z = np.zeros(n)
    np.add.at(z, p.row_idx, p.val.astype(np.float64) * wd[np.repeat(np.arange(m), np.diff(p.col_ptr))])
    clean = np.where(z >= 0, 1, -1)
    assert int((clean != p.y).sum()) == int(np.floor(wl.spec.flip_frac * n + 0.5))


def test_deterministic():
    s = datagen.scaled("svm_20k_100k", 0.05).spec
    a, b = datagen.generate(s), datagen.generate(s)
    for f in ("col_ptr", "row_idx", "val", "y"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_batch_jobs_follow_their_recipe():
    jobs = datagen.batch_jobs(64)
    again = datagen.batch_jobs(64)
    assert [j.spec for j in jobs] == [j.spec for j in again]  # seeded
    assert len(jobs) == 64 and len({j.spec.seed for j in jobs}) == 64
    for k, j in enumerate(jobs):
        assert 1000 <= j.spec.n_samples <= 50000 and 5000 <= j.spec.n_features <= 200000
        dens = j.spec.row_mean / j.spec.n_features
        assert 1e-3 - 1e-9 <= dens <= 1e-2 + 1e-9
        assert j.loss == ("logistic" if k % 2 == 0 else "l2svm")
        assert len(j.C_path) == 16 and j.C_path[0] == pytest.approx(1e-2) and j.C_path[-1] == pytest.approx(10.0)
        assert all(a < b for a, b in zip(j.C_path, j.C_path[1:]))
    # a generated problem has about its expected number of nonzeros (Poisson row lengths, also for
    # means above 500, drawn as sums of pieces)
    big = max(jobs, key=lambda j: j.spec.row_mean)
    assert big.spec.row_mean > 500
    small = datagen.Spec(400, big.spec.n_features, "zipf", row_mean=big.spec.row_mean, zipf_s=1.1, values="tfidf",
                         wstar_nnz=10, flip_frac=0.03, seed=3)
    p = datagen.generate(small, with_csr=False)
    assert p.nnz == pytest.approx(400 * big.spec.row_mean, rel=0.02)
