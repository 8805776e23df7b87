"""GPU-vs-oracle parity of the whole hot path, through the C ABI.

Acceptance (the rule and its counts are in parity_checks): field codes and
domain masks are compared with the FP64 oracle's; an entry may differ only
inside the 1e-5 m / 1e-6 band, and the entries that differ stay below 1e-4 of
the total.  Sampled tuples and finger ids are bit-exact on every pose whose
mask rows equal the oracle's.  Margins agree within 1e-4 * max(t*, eps); accept
decisions are equal except where |t*_oracle - eps| <= 1e-4, and those too stay
below 1e-4 of all tuples.  Every check prints its counts.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_checks import AMB_BOUND, bits as _bits, check_field, check_masks, check_scores, u32 as _u32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    return cf


def _gpu_path(cf, w, poses=None):
    q = torch.from_numpy(w.q).cuda()
    field = cf.build(w.hand, w.inv_h, w.bins, q)
    soa = torch.from_numpy(w.obj.soa()).cuda()
    pz = torch.from_numpy(w.poses if poses is None else poses).cuda()
    masks, counts = cf.query_domains(field, soa, pz)
    prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed)
    tup, fing, margin, accept = cf.score_tuples(soa, w.hand.F, masks, counts, prm)
    torch.cuda.synchronize()
    return dict(field=field, soa=soa, poses=pz, masks=masks, counts=counts, tuples=tup, fingers=fing,
                margin=margin, accept=accept, prm=prm)


def check_sampling(g_tuples, g_fingers, g_masks, o_masks, o_counts, N, T, k, seed):
    """The oracle samples from its OWN masks; the GPU's tuples must equal them on
    every pose whose mask rows agree (all but ambiguous entries).  Returns the
    oracle's tuples and the agreeing poses."""
    ot, of = oracle.sample_tuples(o_masks, o_counts, N, T, k, seed)
    same = np.all(g_masks.reshape(g_masks.shape[0], -1) == o_masks.reshape(o_masks.shape[0], -1), axis=1)
    # a pose whose rows differ holds at least one in-band entry that the mask check already counted
    assert same.mean() >= 0.95, f"{int((~same).sum())} poses with differing (ambiguous) mask rows"
    assert np.array_equal(g_tuples[same], ot[same])
    assert np.array_equal(g_fingers[same], of[same])
    return ot, of, same


def _full_check(cf, w, band=True):
    r = _gpu_path(cf, w)
    ofd = oracle.Field(w.hand, w.q, w.inv_h, w.bins, band=band)
    check_field(r["field"], ofd, w.hand.F, w.name)
    soa = w.obj.soa()
    om, oc, amb = ofd.query(soa, w.poses, amb=True)
    gm, gc = _u32(r["masks"]), _u32(r["counts"])
    check_masks(gm, gc, om, oc, amb, w.obj.N, AMB_BOUND.get(w.name), label=w.name)
    # sampling and scoring: the oracle works from its own masks and tuples
    ot, of, same = check_sampling(r["tuples"].cpu().numpy(), r["fingers"].cpu().numpy(), gm, om, oc, w.obj.N, w.T,
                                  w.k, w.seed)
    omar, oacc, _ = oracle.score_tuples(soa, ot[same], w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps)
    check_scores(r["margin"].cpu().numpy()[same], r["accept"].cpu().numpy()[same], omar, w.eps, label=w.name)
    return r, ofd


def test_tiny_sphere_full_parity(cf):
    w = synth.workload("tiny_sphere")
    r, _ = _full_check(cf, w)
    acc = r["accept"].cpu().numpy()
    assert 0 < acc.sum() < acc.size
    assert cf.device_status() == 0


def test_hand16_superquadric_parity_pose_subset(cf):
    w = synth.workload("hand16_superquadric", P=96)
    r, _ = _full_check(cf, w)
    assert r["accept"].cpu().numpy().mean() > 0.2
    assert cf.device_status() == 0


def test_hand20_tool_parity_pose_subset(cf):
    w = synth.workload("hand20_tool", P=20)
    _full_check(cf, w)
    assert cf.device_status() == 0


@pytest.mark.parametrize("name", ["hand16_superquadric", "hand20_tool"])
def test_full_size_launch_sampled_outputs(cf, name):
    """The benchmark's launch configuration at full size; the oracle checks a
    random set of pose rows of the masks, the first 48 poses' tuples and a
    random sample of the scored tuples."""
    w = synth.workload(name)
    r = _gpu_path(cf, w)
    rng = np.random.default_rng(11)
    ofd = oracle.Field(w.hand, w.q, w.inv_h, w.bins, band=True)
    check_field(r["field"], ofd, w.hand.F, w.name)
    soa = w.obj.soa()
    idx = np.sort(rng.choice(w.P, 24, replace=False))
    om, oc, amb = ofd.query(soa, w.poses[idx], amb=True)
    gm_all, gc_all = _u32(r["masks"]), _u32(r["counts"])
    check_masks(gm_all[idx], gc_all[idx], om, oc, amb, w.obj.N, AMB_BOUND.get(name), label=f"{name} full size")
    # the first 48 poses: the oracle's own masks -> its tuples -> its scores of a random sample of them
    om48, oc48 = ofd.query(soa, w.poses[:48])
    ot, of, same = check_sampling(r["tuples"][:48].cpu().numpy(), r["fingers"][:48].cpu().numpy(), gm_all[:48], om48,
                                  oc48, w.obj.N, w.T, w.k, w.seed)
    flat = ot[same].reshape(-1, w.k)
    pick = rng.choice(flat.shape[0], min(3000, flat.shape[0]), replace=False)
    omar, _, _ = oracle.score_tuples(soa, flat[pick], w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps)
    g_mar = r["margin"][:48].cpu().numpy()[same].ravel()[pick]
    g_acc = r["accept"][:48].cpu().numpy()[same].ravel()[pick]
    check_scores(g_mar, g_acc, omar, w.eps, label=f"{name} full size")
    assert cf.device_status() == 0


def test_ragged_sizes_and_degenerate_cases(cf):
    base = synth.workload("tiny_sphere", P=5, S=512)
    ofd = oracle.Field(base.hand, base.q, base.inv_h, base.bins, band=True)
    q = torch.from_numpy(base.q).cuda()
    field = cf.build(base.hand, base.inv_h, base.bins, q)
    far = base.poses.copy()
    far[2, [3, 7, 11]] += 10.0  # pose 2: object far from the hand -> empty domains
    prm = cf.score_params(base.T, base.k, base.mu, base.K, base.eps, base.obj.centroid, base.obj.rho, 5)
    for N in [1, 31, 33, 100, 1000]:
        soa_h = np.ascontiguousarray(base.obj.soa()[:, :N])
        soa = torch.from_numpy(soa_h).cuda()
        masks, counts = cf.query_domains(field, soa, torch.from_numpy(far).cuda())
        tup, fing, mar, acc = cf.score_tuples(soa, base.hand.F, masks, counts, prm)
        torch.cuda.synchronize()
        om, oc, amb = ofd.query(soa_h, far, amb=True)
        check_masks(_u32(masks), _u32(counts), om, oc, amb, N)
        assert int(counts[2].sum()) == 0
        ot, of, same = check_sampling(tup.cpu().numpy(), fing.cpu().numpy(), _u32(masks), om, oc, N, base.T, base.k, 5)
        assert np.all(ot[2] == -1) and np.all(fing[2].cpu().numpy() == 255)
        om_, _, _ = oracle.score_tuples(soa_h, ot[same], base.mu, base.K, base.obj.centroid, base.obj.rho, base.eps)
        check_scores(mar.cpu().numpy()[same], acc.cpu().numpy()[same], om_, base.eps)
        assert np.all(np.isinf(mar[2].cpu().numpy())) and not acc[2].any()
    # a field built from zero samples holds nothing
    empty = cf.build(base.hand, base.inv_h, base.bins, torch.zeros((base.hand.F, base.hand.J, 0), device="cuda"))
    assert empty.info().table_words == 0
    m0, c0 = cf.query_domains(empty, torch.from_numpy(base.obj.soa()).cuda(), torch.from_numpy(base.poses).cuda())
    torch.cuda.synchronize()
    assert int(c0.abs().sum()) == 0 and int(m0.abs().sum()) == 0


def test_scoring_given_tuples_and_invalid_ids(cf):
    w = synth.workload("hand16_superquadric", P=8, S=4096)
    rng = np.random.default_rng(2)
    tup = rng.integers(0, w.obj.N, size=(w.P, w.T, w.k)).astype(np.int32)
    tup[0, :3, 1] = -1
    tup[1, 5, 2] = w.obj.N  # out of range -> invalid
    soa_h = w.obj.soa()
    soa = torch.from_numpy(soa_h).cuda()
    prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, 0, tuples_given=True)
    t_d = torch.from_numpy(tup).cuda()
    _, _, mar, acc = cf.score_tuples(soa, w.hand.F, None, None, prm, tuples=t_d)
    torch.cuda.synchronize()
    assert np.array_equal(t_d.cpu().numpy(), tup)  # tuples untouched
    om, _, _ = oracle.score_tuples(soa_h, tup, w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps)
    check_scores(mar.cpu().numpy(), acc.cpu().numpy(), om, w.eps)
    assert np.all(np.isinf(mar.cpu().numpy()[0, :3]))


@pytest.mark.parametrize("k,K", [(4, 8), (3, 9), (2, 13), (4, 6), (2, 4), (1, 16), (3, 3)])
def test_lp_shapes_parity(cf, k, K):
    """Closure margins for (k, K) shapes beyond the workloads' (3, 8): the LP's
    columns fill one slot per lane when k K + 6 <= 32 ((2, 13) is the edge) and
    two slots otherwise ((4, 8), (3, 9)); every margin matches the oracle."""
    w = synth.workload("hand16_superquadric", P=4, S=4096)
    rng = np.random.default_rng(100 + 10 * k + K)
    tup = np.stack([rng.choice(w.obj.N, k, replace=False) for _ in range(4 * 48)]).astype(np.int32).reshape(4, 48, k)
    soa_h = w.obj.soa()
    soa = torch.from_numpy(soa_h).cuda()
    prm = cf.score_params(48, k, w.mu, K, w.eps, w.obj.centroid, w.obj.rho, 0, tuples_given=True)
    _, _, mar, acc = cf.score_tuples(soa, w.hand.F, None, None, prm, tuples=torch.from_numpy(tup).cuda())
    torch.cuda.synchronize()
    om, _, _ = oracle.score_tuples(soa_h, tup, w.mu, K, w.obj.centroid, w.obj.rho, w.eps)
    check_scores(mar.cpu().numpy(), acc.cpu().numpy(), om, w.eps)
    assert cf.device_status() == 0


def test_plan_host_path_equals_device_path(cf):
    """4,096 poses from host buffers, the tuples copied back while scoring
    runs: tuples, margins, accepts and the device-side accept count equal
    those of the device-resident path.  A second run without outputs still
    returns the count."""
    w = synth.workload("tiny_sphere", P=4096)
    r = _gpu_path(cf, w)
    plan = cf.Plan(w.hand.F, w.obj.N, w.P, r["prm"])
    pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory().numpy()
    soa_h, poses_h = pin((6, w.obj.N), torch.float32), pin((w.P, 12), torch.float32)
    soa_h[:] = w.obj.soa()
    poses_h[:] = w.poses
    ht, hm, ha = pin((w.P, w.T, w.k), torch.int32), pin((w.P, w.T), torch.float32), pin((w.P, w.T), torch.uint8)
    nacc = plan.run_host(r["field"], soa_h, poses_h, ht, hm, ha)
    assert np.array_equal(ht, r["tuples"].cpu().numpy())
    assert np.array_equal(hm, r["margin"].cpu().numpy())
    assert np.array_equal(ha, r["accept"].cpu().numpy())
    assert nacc == int(r["accept"].sum()) > 0
    assert plan.run_host(r["field"], soa_h, poses_h) == nacc  # outputs optional, count still returned
    # the accepted tuples only, gathered on the device in (pose, tuple) order
    g = torch.empty(nacc * 24, dtype=torch.uint8, pin_memory=True).numpy().view(cf.GRASP_DTYPE)
    assert plan.run_host_accepted(r["field"], soa_h, poses_h, g) == nacc
    pose_idx, tup_idx = np.nonzero(ha)
    assert np.array_equal(g["pose"], pose_idx)
    assert np.array_equal(g["margin"], hm[pose_idx, tup_idx])
    assert np.array_equal(g["point"][:, :w.k], ht[pose_idx, tup_idx])
    assert (g["point"][:, w.k:] == -1).all()
    short = np.zeros(3, cf.GRASP_DTYPE)  # too small: the first 3, and the full count
    assert plan.run_host_accepted(r["field"], soa_h, poses_h, short) == nacc
    assert np.array_equal(short, g[:3])
    # a ragged request (15 gather chunks of 4,096 tuples and 2,560 more) and an empty one
    n2 = 4000
    n_rag = plan.run_host(r["field"], soa_h, poses_h[:n2], ht[:n2], hm[:n2], ha[:n2])
    g2 = np.zeros(n_rag + 1, cf.GRASP_DTYPE)
    assert plan.run_host_accepted(r["field"], soa_h, poses_h[:n2], g2) == n_rag
    pose_idx, tup_idx = np.nonzero(ha[:n2])
    assert np.array_equal(g2["pose"][:n_rag], pose_idx)
    assert np.array_equal(g2["point"][:n_rag, :w.k], ht[pose_idx, tup_idx])
    assert plan.run_host_accepted(r["field"], soa_h, poses_h[:0], g2) == 0


def test_far_and_non_finite_points_hit_nothing(cf):
    """Object points far outside the field (|x / h| far beyond 2^22 cells),
    infinite or NaN hit no finger, and the other points' mask bits and the
    counts are those of the object without them."""
    w = synth.workload("tiny_sphere", P=32)
    q = torch.from_numpy(w.q).cuda()
    field = cf.build(w.hand, w.inv_h, w.bins, q)
    soa = w.obj.soa()
    extra = np.zeros((6, 6), np.float32)
    extra[0] = [1e30, -1e30, np.inf, -np.inf, np.nan, 3e5]
    extra[1] = [0.0, 2e9, 0.0, np.nan, 0.0, -3e5]
    extra[2] = [0.0, 0.0, -np.inf, 0.0, 1.0, 0.0]
    extra[5] = 1.0
    both = np.ascontiguousarray(np.concatenate([soa, extra], axis=1))
    pz = torch.from_numpy(w.poses).cuda()
    m0, c0 = cf.query_domains(field, torch.from_numpy(soa).cuda(), pz)
    m1, c1 = cf.query_domains(field, torch.from_numpy(both).cuda(), pz)
    torch.cuda.synchronize()
    N = soa.shape[1]
    b0, b1 = _bits(_u32(m0), N), _bits(_u32(m1), N + 6)
    assert np.array_equal(b1[:, :, :N], b0)
    assert not b1[:, :, N:].any()
    assert torch.equal(c0, c1)


def test_closure_closed_forms_on_gpu(cf):
    """Antipodal pair on a sphere -> margin 0; a single axis-aligned contact
    (k = 1) -> margin 1 (Eq. GSWO with alpha_j = 1)."""
    r = 0.04
    u = np.array([0.3, -0.5, 0.8])
    u /= np.linalg.norm(u)
    pts = np.array([r * u, -r * u, [0.0, 0.0, -r]])
    nrm = np.array([u, -u, [0.0, 0.0, -1.0]])
    soa = torch.from_numpy(np.ascontiguousarray(np.concatenate([pts.T, nrm.T]), dtype=np.float32)).cuda()
    prm2 = cf.score_params(1, 2, 0.5, 8, 0.01, [0, 0, 0], r, 0, tuples_given=True)
    _, _, m2, a2 = cf.score_tuples(soa, 1, None, None, prm2, tuples=torch.tensor([[[0, 1]]], dtype=torch.int32).cuda())
    prm1 = cf.score_params(1, 1, 0.5, 8, 0.01, [0, 0, 0], r, 0, tuples_given=True)
    _, _, m1, _ = cf.score_tuples(soa, 1, None, None, prm1, tuples=torch.tensor([[[2]]], dtype=torch.int32).cuda())
    torch.cuda.synchronize()
    assert float(m2) <= 1e-6 and int(a2) == 1
    assert abs(float(m1) - 1.0) <= 1e-5


def test_field_save_load_and_plan_host_path(cf, tmp_path):
    w = synth.workload("tiny_sphere", P=64)
    r = _gpu_path(cf, w)
    path = str(tmp_path / "f.cff")
    r["field"].save(path)
    f2 = cf.Field.load(path)
    assert np.array_equal(f2.table(), r["field"].table())
    m2, c2 = cf.query_domains(f2, r["soa"], r["poses"])
    torch.cuda.synchronize()
    assert np.array_equal(_u32(m2), _u32(r["masks"]))
    plan = cf.Plan(w.hand.F, w.obj.N, w.P, r["prm"])
    ht = np.zeros((w.P, w.T, w.k), np.int32)
    hm = np.zeros((w.P, w.T), np.float32)
    ha = np.zeros((w.P, w.T), np.uint8)
    nacc = plan.run_host(r["field"], w.obj.soa(), w.poses, ht, hm, ha)
    assert np.array_equal(ht, r["tuples"].cpu().numpy())
    assert np.array_equal(hm, r["margin"].cpu().numpy())
    assert np.array_equal(ha, r["accept"].cpu().numpy())
    assert nacc == int(ha.sum())


def test_field_with_ragged_link_point_counts(cf):
    """Links holding point counts that are not multiples of the binning pass's 4-point batches (and
    of its 16-point groups): the tail batches have empty slots.  The field equals the oracle's."""
    import dataclasses
    w = synth.workload("hand16_superquadric", P=8, N=512, S=3001)
    h = w.hand
    keep = []
    for l in np.unique(h.surf_link[0]):
        idx = np.nonzero(h.surf_link[0] == l)[0]
        keep.extend(idx[: len(idx) - 1 - int(l) % 3].tolist())  # 31 / 29 / 47-style counts
    keep = np.array(keep)
    assert any(int(np.sum(h.surf_link[0][keep] == l)) % 4 for l in np.unique(h.surf_link[0]))
    hr = dataclasses.replace(h, surf_p=np.ascontiguousarray(h.surf_p[:, keep]),
                             surf_n=np.ascontiguousarray(h.surf_n[:, keep]),
                             surf_link=np.ascontiguousarray(h.surf_link[:, keep]))
    field = cf.build(hr, w.inv_h, w.bins, torch.from_numpy(w.q).cuda())
    torch.cuda.synchronize()
    check_field(field, oracle.Field(hr, w.q, w.inv_h, w.bins, band=True), hr.F, w.name)
    assert cf.device_status() == 0


def test_repeatable_bits(cf):
    w = synth.workload("hand16_superquadric", P=32, S=8192)
    a = _gpu_path(cf, w)
    b = _gpu_path(cf, w)
    assert np.array_equal(a["field"].table(), b["field"].table())
    for key in ["masks", "counts", "tuples", "fingers", "margin", "accept"]:
        assert torch.equal(a[key], b[key]), key
    cnt = cf.device_counters()
    assert cnt["lps"] > 0 and cnt["lp_pivots"] >= 2 * cnt["lps"]
    assert cf.device_status() == 0


def test_split_sampling_and_scoring_equal_the_fused_call(cf):
    w = synth.workload("hand16_superquadric", P=40, S=8192)
    r = _gpu_path(cf, w)
    t2, f2 = cf.sample_tuples(r["soa"], w.hand.F, r["masks"], r["counts"], r["prm"])
    pg = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed, tuples_given=True)
    _, _, m2, a2 = cf.score_tuples(r["soa"], w.hand.F, None, None, pg, tuples=t2)
    torch.cuda.synchronize()
    assert torch.equal(t2, r["tuples"]) and torch.equal(f2, r["fingers"])
    assert torch.equal(m2, r["margin"]) and torch.equal(a2, r["accept"])
