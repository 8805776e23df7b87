"""cf_score_tuples_noalloc against cf_score_tuples.

The no-allocation entry point serves callers that may not allocate device
memory while scoring (a fixed memory budget on a shared GPU, a control loop
that must not block or fail on an allocation).  It must give the same tuples,
fingers, margins and accept flags as the allocating entry point, call after
call, and it must not allocate: neither the library's own device pool nor
torch's caching allocator nor the CUDA driver may see a new allocation during the
calls.  The first call runs in this module, so the test also covers the
per-device set-up.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _inputs(cf, name, P, seed):
    w = synth.workload(name, P=P, S=8192, seed=seed)
    field = cf.build(w.hand, w.inv_h, w.bins, torch.from_numpy(w.q).cuda())
    soa = torch.from_numpy(w.obj.soa()).cuda()
    masks, counts = cf.query_domains(field, soa, torch.from_numpy(w.poses).cuda())
    prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed)
    return w, field, soa, masks, counts, prm


def _close(a_margin, b_margin, eps):
    a = a_margin.cpu().numpy().astype(np.float64)
    b = b_margin.cpu().numpy().astype(np.float64)
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    assert np.all(np.abs(a[fin] - b[fin]) <= 1e-4 * np.maximum(np.abs(b[fin]), eps))


def _sentinels(w):
    shape = (w.P, w.T, w.k)
    return (torch.full(shape, -7, dtype=torch.int32, device="cuda"),
            torch.full(shape, 77, dtype=torch.uint8, device="cuda"),
            torch.full((w.P, w.T), -1.0, device="cuda"),
            torch.full((w.P, w.T), 9, dtype=torch.uint8, device="cuda"))


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    for name, P, seed in [("hand16_superquadric", 64, 3), ("tiny_sphere", 48, 4)]:
        w, _field, soa, masks, counts, prm = _inputs(cf, name, P, seed)
        ref_t, ref_f, ref_m, ref_a = cf.score_tuples(soa, w.hand.F, masks, counts, prm)
        torch.cuda.synchronize()
        outs = [_sentinels(w), _sentinels(w)]
        # two calls in a row on one stream, into separate outputs: the second
        # starts from whatever the first left in the shared scratch
        for t, f, m, a in outs:
            cf.score_tuples_noalloc(soa, w.hand.F, masks, counts, prm, t, f, m, a)
        torch.cuda.synchronize()
        for t, f, m, a in outs:
            assert torch.equal(t, ref_t)
            assert torch.equal(f, ref_f)
            assert torch.equal(a, ref_a)
            _close(m, ref_m, w.eps)
        assert int(ref_a.sum()) > 0
    assert cf.device_status() == 0


def test_noalloc_calls_allocate_nothing():
    """After one warm-up call, repeated calls leave the library pool's
    high-water mark, torch's allocated and reserved bytes and the device's
    free memory exactly where they were."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    w, _field, soa, masks, counts, prm = _inputs(cf, "hand16_superquadric", 32, 5)
    t, f, m, a = _sentinels(w)
    cf.score_tuples_noalloc(soa, w.hand.F, masks, counts, prm, t, f, m, a)  # warm-up (per-device set-up)
    torch.cuda.synchronize()
    before_pool = cf.pool_usage(reset_high=True)
    before_torch = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
    before_free = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        cf.score_tuples_noalloc(soa, w.hand.F, masks, counts, prm, t, f, m, a)
    torch.cuda.synchronize()
    after_pool = cf.pool_usage()
    assert after_pool["high"] <= before_pool["used"], (before_pool, after_pool)
    assert after_pool["used"] == before_pool["used"]
    assert after_pool["reserved"] == before_pool["reserved"]
    assert (torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == before_torch
    assert torch.cuda.mem_get_info()[0] == before_free


def test_noalloc_rejects_bad_arguments_without_touching_outputs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    w = synth.workload("tiny_sphere", P=4, S=512)
    soa = torch.from_numpy(w.obj.soa()).cuda()
    # k = 9 exceeds the library's contact limit: refused on the host
    prm = cf.score_params(w.T, 9, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, 0, tuples_given=True)
    t = torch.full((w.P, w.T, 9), -7, dtype=torch.int32, device="cuda")
    m = torch.full((w.P, w.T), -1.0, device="cuda")
    a = torch.full((w.P, w.T), 9, dtype=torch.uint8, device="cuda")
    with pytest.raises(cf.CfError):
        cf.score_tuples_noalloc(soa, w.hand.F, None, None, prm, t, None, m, a)
    torch.cuda.synchronize()
    assert bool((t == -7).all()) and bool((m == -1.0).all()) and bool((a == 9).all())
