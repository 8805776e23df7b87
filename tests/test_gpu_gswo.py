"""GPU-vs-oracle parity of the paper's own metric, Eq. GSWO with true friction
cones (Sec. 3.2), through the C ABI.  Both sides run the same accelerated
projected-gradient iteration (the kernel in FP32, the oracle in FP64) on the
oracle's sampled tuples.

Acceptance rule: values agree within 1e-3 max(J, eps_g) (the iteration is a
non-expansive map composed with momentum; FP32 rounding of ~1e-7 per step
stays below that after 256 steps), and accept flags are equal unless the oracle
value lies within that band of eps_g."""
import numpy as np
import pytest

import oracle
import synth
from oracle import gswo as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS_G = 1e-4
REL = 1e-3


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    return cf


@pytest.mark.parametrize("name,P,S,n_iter", [("hand16_superquadric", 2, 4096, 256), ("tiny_sphere", 8, 2048, 256),
                                             ("hand20_tool", 1, 4096, 256), ("tiny_sphere", 2, 1024, 32)])
def test_gswo_parity(cf, name, P, S, n_iter):
    w = synth.workload(name, P=P, S=S)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
    soa = w.obj.soa()
    m, c = fd.query(soa, w.poses)
    tup, _ = oracle.sample_tuples(m, c, w.obj.N, w.T, w.k, w.seed)
    prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed, tuples_given=True)
    gv, ga = cf.score_gswo(torch.from_numpy(soa).cuda(), prm, torch.from_numpy(tup).cuda(), n_iter, EPS_G)
    torch.cuda.synchronize()
    gv, ga = gv.cpu().numpy().astype(np.float64), ga.cpu().numpy()
    ov = G.score_gswo(soa, tup, w.mu, w.obj.centroid, w.obj.rho, n_iter)
    fin = np.isfinite(ov)
    assert np.array_equal(np.isfinite(gv), fin)
    err = np.abs(gv[fin] - ov[fin]) / np.maximum(ov[fin], EPS_G)
    print(f"{name}: {fin.sum()} tuples, max relative error {err.max():.3g}, accept {ga[fin].mean():.3f}")
    assert err.max() <= REL
    firm = fin & (np.abs(ov - EPS_G) > REL * np.maximum(ov, EPS_G))
    assert np.array_equal(ga[firm], (ov[firm] <= EPS_G).astype(np.uint8))
    assert np.all(ga[~fin] == 0)


def test_gswo_edge_cases(cf):
    w = synth.workload("tiny_sphere", P=1, S=64)
    soa = torch.from_numpy(w.obj.soa()).cuda()
    prm = cf.score_params(2, 2, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed, tuples_given=True)
    t = torch.tensor([[[0, 1], [-1, 3]]], dtype=torch.int32).cuda()
    v, a = cf.score_gswo(soa, prm, t, 0, EPS_G)  # no step: J_j at alpha = e_j
    v = v.cpu().numpy()
    assert np.isinf(v[0, 1]) and np.isfinite(v[0, 0])
    s = w.obj.soa().astype(np.float64)
    A = G.gswo_matrix(s[0:3, [0, 1]].T, s[3:6, [0, 1]].T, w.obj.centroid, w.obj.rho)
    ref = min(float(A[:, 0] @ A[:, 0]), float(A[:, 3] @ A[:, 3]))
    assert abs(v[0, 0] - ref) <= 1e-5 * ref
    with pytest.raises(cf.CfError):
        cf.score_gswo(soa, cf.score_params(2, 1, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, 0, True), t, 8)


def test_fswo_parity(cf):
    """Eq. FSWO is Eq. GSWO with mu = 0 (no friction: every beta is 0).  Sampled tuples against
    the oracle, plus tuples that repeat one point: three equal pushes cannot cancel (alpha >= 0),
    so J = |nu|^2 + |r x nu|^2 / rho^2 = 1 on the sphere (no torque about its centre)."""
    w = synth.workload("tiny_sphere", P=4, S=2048)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
    soa = w.obj.soa()
    m, c = fd.query(soa, w.poses)
    tup, _ = oracle.sample_tuples(m, c, w.obj.N, w.T, w.k, w.seed)
    tup = tup.copy()
    tup[0, 0] = [5, 5, 5]
    tup[1, 2] = [77, 77, 77]
    prm = cf.score_params(w.T, w.k, 0.0, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed, tuples_given=True)
    gv, ga = cf.score_gswo(torch.from_numpy(soa).cuda(), prm, torch.from_numpy(tup).cuda(), 256, EPS_G)
    torch.cuda.synchronize()
    gv, ga = gv.cpu().numpy().astype(np.float64), ga.cpu().numpy()
    ov = G.score_gswo(soa, tup, 0.0, w.obj.centroid, w.obj.rho, 256)
    fin = np.isfinite(ov)
    assert np.array_equal(np.isfinite(gv), fin)
    err = np.abs(gv[fin] - ov[fin]) / np.maximum(ov[fin], EPS_G)
    print(f"FSWO: {fin.sum()} tuples, max relative error {err.max():.3g}, accept {ga[fin].mean():.3f}")
    assert err.max() <= REL
    for i, t in ((0, 0), (1, 2)):
        r = soa[0:3, tup[i, t, 0]].astype(np.float64) - w.obj.centroid
        nu = -soa[3:6, tup[i, t, 0]].astype(np.float64)
        exact = float(nu @ nu + np.sum(np.cross(r, nu) ** 2) / w.obj.rho ** 2)
        assert abs(gv[i, t] - exact) <= 1e-4 * exact and abs(ov[i, t] - exact) <= 1e-9, (gv[i, t], ov[i, t], exact)


def test_gswo_full_size_sampled(cf):
    """The benchmark's Eq. GSWO configuration at full size (hand20_tool: the whole field, 32,768 poses x
    128 sampled tuples, 256 iterations): 1,000 tuples drawn over the whole launch against the oracle."""
    w = synth.workload("hand20_tool")
    dev = torch.device("cuda:0")
    F, W = w.hand.F, (w.obj.N + 31) // 32
    field = cf.build(w.hand, w.inv_h, w.bins, torch.from_numpy(w.q).to(dev))
    soa_h = np.ascontiguousarray(w.obj.soa())
    soa = torch.from_numpy(soa_h).to(dev)
    masks = torch.empty((w.P, F, W), dtype=torch.int32, device=dev)
    counts = torch.empty((w.P, F), dtype=torch.int32, device=dev)
    tuples = torch.empty((w.P, w.T, w.k), dtype=torch.int32, device=dev)
    fingers = torch.empty((w.P, w.T, w.k), dtype=torch.uint8, device=dev)
    cf.query_domains(field, soa, torch.from_numpy(w.poses).to(dev), masks, counts)
    prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed)
    cf.sample_tuples(soa, F, masks, counts, prm, tuples, fingers)
    prm_g = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed, tuples_given=True)
    gv, ga = cf.score_gswo(soa, prm_g, tuples, 256, EPS_G)
    torch.cuda.synchronize()
    assert cf.device_status() == 0
    idx = np.random.default_rng(5).choice(w.P * w.T, 1000, replace=False)
    tup = tuples.reshape(-1, w.k)[torch.from_numpy(idx).to(dev)].cpu().numpy()
    gv = gv.reshape(-1)[torch.from_numpy(idx).to(dev)].cpu().numpy().astype(np.float64)
    ga = ga.reshape(-1)[torch.from_numpy(idx).to(dev)].cpu().numpy()
    ov = G.score_gswo(soa_h, tup, w.mu, w.obj.centroid, w.obj.rho, 256)
    fin = np.isfinite(ov)
    assert np.array_equal(np.isfinite(gv), fin)
    err = np.abs(gv[fin] - ov[fin]) / np.maximum(ov[fin], EPS_G)
    print(f"hand20_tool full size: {fin.sum()} sampled tuples, max relative error {err.max():.3g}, "
          f"accept {ga[fin].mean():.3f}")
    assert err.max() <= REL
    firm = fin & (np.abs(ov - EPS_G) > REL * np.maximum(ov, EPS_G))
    assert np.array_equal(ga[firm], (ov[firm] <= EPS_G).astype(np.uint8))
