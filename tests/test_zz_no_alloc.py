"""emd_topk_select_static: top-K selection with its scratch in a fixed device array, for
callers that may not allocate device memory (a host framework's allocator owns it all,
or a serving loop cannot absorb cudaMalloc's synchronisation).

Its output must equal what the regular entry point (emd_topk_device, same selection
kernels, library-allocated scratch) returns for the same distances, on two calls in a
row (the array keeps the previous call's contents).  This file is collected last so a
run that stops at the first failure has already run every other test."""
import numpy as np
import pytest

import emd_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch

    import paper_1812_02091_gb300 as emd
    from paper_1812_02091_gb300 import _build
    _build.build()
    emd.load()
    # 20000 documents: the selection runs on several blocks per row, so the block
    # partials really go through the scratch array
    w = emd_synth.small_text(2468, V=3000, m=16, n=20000, n_queries=5, lo=4, hi=24)
    db = emd.emd_db_create(w.emb, None, w.db.row_ptr, w.db.col, w.db.val,
                           emd.emd_db_options_default(max_query_h=32))
    q = w.queries
    qi = torch.from_numpy(q.col).cuda()
    qw = torch.from_numpy(q.val).cuda()
    s = torch.cuda.current_stream().cuda_stream
    t = torch.empty((q.n, w.db.n), dtype=torch.float32, device="cuda")
    emd.emd_query_batch_device(db, q.row_ptr, qi, qw, t, "act", 2, "max", stream=s)
    yield emd, db, w, q, qi, qw, t, s
    torch.cuda.synchronize()
    emd.emd_db_destroy(db)


@pytest.mark.parametrize("K", [16, 64])
def test_static_scratch_topk_matches_regular_entry_point(setup, K):
    import torch
    emd, db, w, q, qi, qw, t, s = setup
    ref_i = torch.empty((q.n, K), dtype=torch.int64, device="cuda")
    ref_d = torch.empty((q.n, K), dtype=torch.float32, device="cuda")
    emd.emd_topk_device(db, q.row_ptr, qi, qw, ref_i, ref_d, "act", 2, "max", K, stream=s)
    for call in range(2):
        oi = torch.full((q.n, K), -7, dtype=torch.int64, device="cuda")
        od = torch.full((q.n, K), -7.0, dtype=torch.float32, device="cuda")
        emd.emd_topk_select_static(t, K, oi, od, stream=s)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(oi.cpu().numpy(), ref_i.cpu().numpy(), err_msg=f"call {call}")
        np.testing.assert_allclose(od.cpu().numpy(), ref_d.cpu().numpy(), rtol=1e-5, atol=1e-7)


def test_static_scratch_rejects_sizes_beyond_its_limit(setup):
    import torch
    emd, *_ = setup
    big = torch.zeros((65, 100), dtype=torch.float32, device="cuda")
    oi = torch.empty((65, 4), dtype=torch.int64, device="cuda")
    od = torch.empty((65, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(emd.EmdError) as e:
        emd.emd_topk_select_static(big, 4, oi, od)
    assert e.value.name == "INVALID_ARG" and "64 rows" in str(e.value)
    with pytest.raises(emd.EmdError):
        emd.emd_topk_select_static(big[:2], 65, oi, od)


def test_static_scratch_after_a_larger_call(setup):
    """Calls that use fewer rows or fewer blocks than the previous one must ignore what
    that call left in the shared array: 5 rows over 20000 values (several blocks per
    row), then 1 row over 4096 values (two blocks) and 1 row over 1500 values (one
    block), each against a stable numpy argsort."""
    import torch
    emd, db, w, q, qi, qw, t, s = setup
    K = 16
    oi = torch.empty((q.n, K), dtype=torch.int64, device="cuda")
    od = torch.empty((q.n, K), dtype=torch.float32, device="cuda")
    emd.emd_topk_select_static(t, K, oi, od, stream=s)
    rng = np.random.default_rng(17)
    for n in (4096, 1500):
        x = rng.uniform(0.0, 1.0, n).astype(np.float32)
        x[rng.integers(0, n, 8)] = 0.25  # repeated values: ties go to the lower index
        xt = torch.from_numpy(x).cuda()
        oi1 = torch.full((1, K), -7, dtype=torch.int64, device="cuda")
        od1 = torch.full((1, K), -7.0, dtype=torch.float32, device="cuda")
        emd.emd_topk_select_static(xt, K, oi1, od1, stream=s)
        torch.cuda.synchronize()
        want = np.argsort(x, kind="stable")[:K]
        np.testing.assert_array_equal(oi1.cpu().numpy()[0], want, err_msg=f"n={n}")
        np.testing.assert_array_equal(od1.cpu().numpy()[0], x[want])


def test_static_wrapper_rejects_bad_shapes(setup):
    import torch
    emd, *_ = setup
    t3 = torch.zeros((2, 3, 100), dtype=torch.float32, device="cuda")
    oi = torch.empty((2, 4), dtype=torch.int64, device="cuda")
    od = torch.empty((2, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        emd.emd_topk_select_static(t3, 4, oi, od)
    with pytest.raises(ValueError):
        emd.emd_topk_select_static(t3[0], 8, oi, od)  # outputs hold 8 < 3 x 8 elements
