"""Served form: requests with different objects and hands share rounds on the
GPU (continuous batching); each result must be the same alone and in the mix,
admission must respect the HBM budget and the slots, and a request's first
chunk must equal the plain per-object calls."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HANDS = ["tiny_sphere", "hand16_superquadric", "hand20_tool"]


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    ws, fields = [], []
    for name in HANDS:
        w = synth.workload(name, P=1, N=64, S=4096)
        ws.append(w)
        fields.append(cf.build(w.hand, w.inv_h, w.bins, torch.from_numpy(w.q).cuda()))
    torch.cuda.synchronize()
    reqs = []
    rng = np.random.default_rng(9)
    for j, sp in enumerate(synth.batch_objects(8, seed=13, n_range=(1024, 8192), p_range=(512, 2048))):
        hi = HANDS.index(sp["hand"])
        w = ws[hi]
        obj, poses = synth.batch_object_inputs(sp, w.hand)
        prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, obj.centroid, obj.rho, 500 + j)
        reqs.append(dict(field=hi, soa=obj.soa(), poses=poses, prm=prm, n_grasps=int(rng.integers(50, 400)), tag=j))
    return cf, ws, fields, reqs


def _collect(eng, n):
    out = []
    eng.drain(120000)
    while len(out) < n:
        out += eng.poll()
    return {r["tag"]: r for r in out}


def _same(a, b):
    assert a["status"] == b["status"] == 0
    assert a["n_accepted"] == b["n_accepted"] and a["n_poses_used"] == b["n_poses_used"]
    assert np.array_equal(a["pose"], b["pose"]) and np.array_equal(a["tuples"], b["tuples"])
    assert np.array_equal(a["margin"], b["margin"])


def test_results_are_the_same_alone_and_in_the_mix(setup):
    cf, ws, fields, reqs = setup
    eng = cf.Engine(fields, max_active=16, pose_chunk=128)
    alone = {}
    for q in reqs:
        eng.submit(q["field"], q["soa"], q["poses"], q["prm"], q["n_grasps"], q["tag"])
        alone.update(_collect(eng, 1))
    for q in reqs:
        eng.submit(q["field"], q["soa"], q["poses"], q["prm"], q["n_grasps"], q["tag"])
    mixed = _collect(eng, len(reqs))
    st = eng.stats()
    eng.close()
    assert st["peak_active"] > 1          # requests really shared rounds
    for q in reqs:
        a, b = alone[q["tag"]], mixed[q["tag"]]
        _same(a, b)
        assert a["n_accepted"] >= q["n_grasps"] or a["partial"]
        assert a["t_submit"] <= a["t_admit"] <= a["t_done"]
    assert cf.device_status() == 0


def test_admission_respects_budget_and_slots(setup):
    cf, ws, fields, reqs = setup
    eng0 = cf.Engine(fields, max_active=16, pose_chunk=128)
    for q in reqs:
        eng0.submit(q["field"], q["soa"], q["poses"], q["prm"], q["n_grasps"], q["tag"])
    ref = _collect(eng0, len(reqs))
    eng0.close()
    budget = 24 << 20
    eng = cf.Engine(fields, hbm_budget_bytes=budget, max_active=3, pose_chunk=128)
    for q in reqs:
        eng.submit(q["field"], q["soa"], q["poses"], q["prm"], q["n_grasps"], q["tag"])
    got = _collect(eng, len(reqs))
    st = eng.stats()
    eng.close()
    assert st["peak_bytes_in_use"] <= budget and st["peak_active"] <= 3
    assert st["completed"] == len(reqs) and st["bytes_in_use"] == 0
    for q in reqs:
        if got[q["tag"]]["status"] == 0:
            _same(got[q["tag"]], ref[q["tag"]])
    # a request larger than the whole budget ends at once with CF_ENOMEM (2)
    eng = cf.Engine(fields, hbm_budget_bytes=1 << 16, max_active=2, pose_chunk=128)
    q = reqs[0]
    eng.submit(q["field"], q["soa"], q["poses"], q["prm"], q["n_grasps"], 99)
    r = _collect(eng, 1)[99]
    eng.close()
    assert r["status"] == 2 and r["n_accepted"] == 0


def test_first_chunk_equals_plain_calls(setup):
    cf, ws, fields, reqs = setup
    q = reqs[1]
    chunk = 64
    eng = cf.Engine(fields, max_active=4, pose_chunk=chunk)
    eng.submit(q["field"], q["soa"], q["poses"], q["prm"], 10 ** 9, q["tag"])  # runs until the pose list ends
    r = _collect(eng, 1)[q["tag"]]
    eng.close()
    assert r["partial"]
    w = ws[q["field"]]
    soa = torch.from_numpy(q["soa"]).cuda()
    pz = torch.from_numpy(q["poses"][:chunk]).cuda()
    m, c = cf.query_domains(fields[q["field"]], soa, pz)
    t, f, mar, acc = cf.score_tuples(soa, w.hand.F, m, c, q["prm"])
    torch.cuda.synchronize()
    acc = acc.cpu().numpy().astype(bool)
    sel = r["pose"] < chunk
    pose_idx, tup_idx = np.nonzero(acc)
    assert np.array_equal(r["pose"][sel], pose_idx)
    assert np.array_equal(r["tuples"][sel], t.cpu().numpy()[acc])
    assert np.array_equal(r["margin"][sel], mar.cpu().numpy()[acc])


def test_adaptive_chunks(setup):
    """Adaptive chunks (after the first round a request takes the poses its acceptance says it
    still needs): results the same alone and in the mix; on the poses both forms processed,
    the same accepted tuples as fixed chunks; never more rounds per request, fewer overall."""
    cf, ws, fields, reqs = setup
    fixed = cf.Engine(fields, max_active=16, pose_chunk=64)
    for q in reqs:
        fixed.submit(q["field"], q["soa"], q["poses"], q["prm"], q["n_grasps"], q["tag"])
    ref = _collect(fixed, len(reqs))
    fixed.close()
    eng = cf.Engine(fields, max_active=16, pose_chunk=64, pose_chunk_max=1024)
    alone = {}
    for q in reqs:
        eng.submit(q["field"], q["soa"], q["poses"], q["prm"], q["n_grasps"], q["tag"])
        alone.update(_collect(eng, 1))
    for q in reqs:
        eng.submit(q["field"], q["soa"], q["poses"], q["prm"], q["n_grasps"], q["tag"])
    mixed = _collect(eng, len(reqs))
    eng.close()
    for q in reqs:
        a, f = mixed[q["tag"]], ref[q["tag"]]
        _same(alone[q["tag"]], a)
        assert a["n_accepted"] >= q["n_grasps"] or a["partial"]
        assert a["n_rounds"] <= f["n_rounds"]
        lim = min(a["n_poses_used"], f["n_poses_used"])
        sa, sf = a["pose"] < lim, f["pose"] < lim
        assert np.array_equal(a["pose"][sa], f["pose"][sf]) and np.array_equal(a["tuples"][sa], f["tuples"][sf])
        assert np.array_equal(a["margin"][sa], f["margin"][sf])
    assert sum(mixed[q["tag"]]["n_rounds"] for q in reqs) < sum(ref[q["tag"]]["n_rounds"] for q in reqs)
    # a pair cap that never lets a chunk pass pose_chunk (every object has n >= 1,024): fixed chunks exactly
    assert min(q["soa"].shape[1] for q in reqs) >= 1024
    capped = cf.Engine(fields, max_active=16, pose_chunk=64, pose_chunk_max=1024, chunk_pairs_max=64 * 1024)
    for q in reqs:
        capped.submit(q["field"], q["soa"], q["poses"], q["prm"], q["n_grasps"], q["tag"])
    got = _collect(capped, len(reqs))
    capped.close()
    for q in reqs:
        _same(got[q["tag"]], ref[q["tag"]])
        assert got[q["tag"]]["n_rounds"] == ref[q["tag"]]["n_rounds"]
    assert cf.device_status() == 0


def test_reserve_grows_the_pool(setup):
    """reserve_bytes grows the library's pool at creation; freed memory stays reserved."""
    cf, ws, fields, reqs = setup
    r = 96 << 20
    eng = cf.Engine(fields, max_active=2, pose_chunk=64, reserve_bytes=r)
    reserved = cf.pool_usage()["reserved"]
    eng.close()
    assert reserved >= r
    with pytest.raises(cf.CfError):
        cf.Engine(fields, max_active=2, pose_chunk=64, reserve_bytes=-1)


def test_drain_is_a_bounded_wait(setup):
    """The engine's waits are on the host and bounded: a drain whose limit runs
    out while requests remain returns CF_ETIMEOUT (the engine keeps working), and
    a later drain completes every request.  No kernel waits on another block or
    on the host, so nothing on the GPU can hang."""
    cf, ws, fields, reqs = setup
    eng = cf.Engine(fields, max_active=2, pose_chunk=64)
    for q in reqs:
        eng.submit(q["field"], q["soa"], q["poses"], q["prm"], 10 ** 9, q["tag"])  # run to the pose limit
    with pytest.raises(cf.CfError) as ei:
        eng.drain(0)
    assert ei.value.code == cf.CF_ETIMEOUT
    got = _collect(eng, len(reqs))
    assert sorted(got) == [q["tag"] for q in reqs]
    assert all(r["status"] == 0 and r["partial"] for r in got.values())
    eng.close()
