"""Shapes and invariants of the seeded synthetic inputs."""
import numpy as np

import emd_synth


def _check_hist(h: emd_synth.Histograms, v: int):
    assert h.row_ptr[0] == 0 and np.all(np.diff(h.row_ptr) >= 1)
    assert h.col.dtype == np.int32 and h.val.dtype == np.float32
    assert h.col.min() >= 0 and h.col.max() < v
    for i in range(0, h.n, max(1, h.n // 50)):
        c, w = h.row(i)
        assert np.all(np.diff(c) > 0)
        assert np.all(w > 0)
        assert abs(float(w.astype(np.float64).sum()) - 1.0) < 1e-6


def test_tiny_text():
    w = emd_synth.config(1)
    assert w.emb.shape == (2000, 64) and w.db.n == 1000 and w.queries.n == 10
    _check_hist(w.db, 2000); _check_hist(w.queries, 2000)
    lens = np.diff(w.db.row_ptr)
    assert lens.min() >= 10 and lens.max() <= 40
    np.testing.assert_allclose(np.linalg.norm(w.emb.astype(np.float64), axis=1), 1.0, atol=1e-6)


def test_seeded_and_reproducible():
    a = emd_synth.config(1)
    b = emd_synth.config(1)
    np.testing.assert_array_equal(a.db.col, b.db.col)
    np.testing.assert_array_equal(a.emb, b.emb)


def test_image_shape_and_fill():
    w = emd_synth.config(3, query_limit=4, n_docs=500)
    _check_hist(w.db, 784)
    frac = w.db.nnz / w.db.n / 784
    assert 0.15 <= frac <= 0.25
    assert np.all(np.diag(w.cost) == 0) and w.cost.shape == (784, 784)
    assert w.cost[0, 29] == np.float32(np.sqrt(2.0))


def test_mixed_query_lengths_are_log_uniform():
    rng = np.random.Generator(np.random.PCG64(5))
    L = emd_synth._lengths(rng, 20000, emd_synth.QUERY_LEN_MIXED)
    assert L.min() >= 5 and L.max() <= 2000
    assert 250 < L.mean() < 420 and 80 < np.median(L) < 120


def test_c_row_selection_equals_numpy_form():
    """The C helper and the numpy form of the successive-sampling step give the same
    histograms from the same seed (including rows that need a second round of draws)."""
    for V, n, law in ((60, 300, ("uniform", 40, 60)), (5000, 700, ("loguniform", 5, 2000)),
                      (100000, 2000, ("lognormal", 100.0, 0.5, 10, 1000))):
        lens = np.minimum(emd_synth._lengths(np.random.Generator(np.random.PCG64(3)), n, law), V)
        a = emd_synth.zipf_histograms(np.random.Generator(np.random.PCG64(9)), V, lens, chunk=257, use_c=False)
        b = emd_synth.zipf_histograms(np.random.Generator(np.random.PCG64(9)), V, lens, chunk=257, use_c=True)
        assert np.array_equal(a.row_ptr, b.row_ptr)
        assert np.array_equal(a.col, b.col)
        assert np.array_equal(a.val, b.val)
