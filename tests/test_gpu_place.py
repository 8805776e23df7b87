"""GPU-vs-oracle parity of object placement (Sec. 5.2) and the small-box
concave-point removal (Sec. 5.1), through the C ABI.  Placement runs in FP64
on both sides and rounds to FP32, so poses agree within a few FP32 ulps; the
concave test agrees except where the oracle flags a sample within its band of
-tau (or on a sign-ambiguous SDF node)."""
import numpy as np
import pytest

import oracle
import synth
from parity_checks import GivenCodes
from oracle import kinematics as K
from oracle import placement as PL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    return cf


def test_canonical_placement(cf):
    c, g, up = [0.01, -0.02, 0.005], [0.0, 0.02, 0.0], [0.0, 0.0, 1.0]
    gp = cf.place_canonical(4096, c, g, up, 0.08, 0.12, seed=17, pose_base=100).cpu().numpy()
    op = PL.place_canonical(4096, c, g, up, 0.08, 0.12, seed=17, pose_base=100)
    assert np.abs(gp - op).max() <= 4e-7
    assert np.mean(gp == op) > 0.99


@pytest.mark.parametrize("name", ["tiny_sphere", "hand16_superquadric"])
def test_exhaustive_placement(cf, name):
    w = synth.workload(name, P=1, S=2048)
    field = cf.build(w.hand, w.inv_h, w.bins, torch.from_numpy(w.q).cuda())
    # placement draws a code by its rank in the table, so it is checked given the GPU's own table
    # (the table itself is checked against the FP64 field in the parity tests)
    fd = GivenCodes(field, w.hand.F)
    soa = torch.from_numpy(w.obj.soa()).cuda()
    P = 512
    gp = cf.place_exhaustive(field, soa, P, seed=3)
    op, chosen, x = PL.place_exhaustive(fd, w.bins, w.inv_h, w.obj.soa(), P, seed=3)
    g = gp.cpu().numpy()
    assert np.abs(g - op).max() <= 4e-6
    # every placed pose makes the chosen point a contact of the chosen finger in the GPU's own query
    masks, _ = cf.query_domains(field, soa, gp)
    m = masks.cpu().numpy().view(np.uint32)
    f = chosen[:, 3]
    bits = (m[np.arange(P), f, x >> 5] >> (x & 31).astype(np.uint32)) & 1
    assert bits.mean() > 0.99  # a handful may sit on a bin tie after FP32 rounding of the pose
    assert cf.device_status() == 0


@pytest.mark.parametrize("name,side", [("hand20_tool", 0.006), ("hand16_superquadric", 0.004)])
def test_concave_filter(cf, name, side):
    w = synth.workload(name, P=1, N=4096, S=64)
    soa_h = w.obj.soa()
    lo, h, dims = cf.sdf_box(soa_h, 0.002, 0.02)
    soa = torch.from_numpy(soa_h).cuda()
    sdf = cf.Sdf(soa, lo, h, dims)
    keep, out, n = cf.concave_filter(soa, sdf, side, 0.001)
    torch.cuda.synchronize()
    gk = keep.cpu().numpy()
    grid, amb = K.sdf_grid(soa_h, lo, h, dims)
    ok, oamb = PL.concave_keep(soa_h, grid, amb, lo, h, side, 0.001)
    assert oamb.mean() < 0.01
    assert np.array_equal(gk[~oamb], ok[~oamb])
    nk = int(n.item())
    assert nk == int(gk.sum())
    assert np.array_equal(out.cpu().numpy()[:, :nk], soa_h[:, gk.astype(bool)])  # kept points, original order
    if name == "hand20_tool":
        assert 0 < nk < soa_h.shape[1]  # the composite has concave seams and a torus hole


@pytest.mark.parametrize("name", ["hand16_superquadric", "hand20_tool"])
def test_static_link_placement(cf, name):
    """Sec. 5.2 static links: poses against the palm and the penetration filter
    match the FP64 oracle (poses within FP32 rounding of FP64, flags equal off
    the oracle's band); the static contact then joins sampled finger tuples and
    the (k+1)-contact closure margins match the oracle's LPs."""
    w = synth.workload(name, P=1, S=4096)
    soa_h = w.obj.soa()
    soa = torch.from_numpy(soa_h).cuda()
    P = 384
    gp, gx, gv = cf.place_static(w.hand.palm_lo, w.hand.palm_hi, soa, P, seed=21, pose_base=5)
    torch.cuda.synchronize()
    op, ox, ov, amb = PL.place_static(w.hand.palm_lo, w.hand.palm_hi, soa_h, P, seed=21, pose_base=5)
    assert np.array_equal(gx.cpu().numpy(), ox)
    assert np.abs(gp.cpu().numpy() - op).max() <= 4e-6
    g_v = gv.cpu().numpy()
    assert np.array_equal(g_v[~amb], ov[~amb])
    assert amb.mean() < 0.02
    if name == "hand20_tool":
        assert 0 < ov.sum() < P  # the composite's seams and hole make some placements penetrate
    # the static contact in front of 2 sampled finger contacts: k = 3 tuples with the palm contact
    field = cf.build(w.hand, w.inv_h, w.bins, torch.from_numpy(w.q).cuda())
    masks, counts = cf.query_domains(field, soa, gp)
    prm2 = cf.score_params(8, 2, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, 4)
    t2, f2 = cf.sample_tuples(soa, w.hand.F, masks, counts, prm2)
    t3 = cf.append_contact(t2, gx, gv)
    prm3 = cf.score_params(8, 3, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, 4, tuples_given=True)
    _, _, mar, acc = cf.score_tuples(soa, w.hand.F, None, None, prm3, tuples=t3)
    torch.cuda.synchronize()
    t3h, t2h = t3.cpu().numpy(), t2.cpu().numpy()
    ok = (g_v.astype(bool)[:, None]) & np.all(t2h >= 0, axis=2)
    assert np.array_equal(t3h[..., 0][ok], np.broadcast_to(gx.cpu().numpy()[:, None], ok.shape)[ok])
    assert np.array_equal(t3h[..., 1:][ok], t2h[ok])
    assert np.all(t3h[~ok] == -1)
    om, oa, _ = oracle.score_tuples(soa_h, t3h, w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps)
    g = mar.cpu().numpy().astype(np.float64)
    fin = np.isfinite(om)
    assert np.array_equal(fin, np.isfinite(g))
    assert np.all(np.abs(g[fin] - np.maximum(om[fin], 0)) <= 1e-4 * np.maximum(om[fin], w.eps))
    assert fin.sum() > 0
    assert cf.device_status() == 0
