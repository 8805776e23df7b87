"""GPU-vs-oracle parity of theta-dilated bins (the leaf test of Sec. 4.3 read
as "the cell holds a bin within theta of the query's bin"), through the C ABI:
the field's dilation table, the domain masks (bit-exact except entries the
oracle flags as ambiguous), and the reverse lookup that IK does through the
accepted bins (Sec. 5.5).  Inputs of the oracle are its own."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import kinematics as K

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    return cf


def _deg_between_levels(bins, target_deg):
    """A dilation angle near target_deg that no pair of bins sits on."""
    d = bins.astype(np.float64)
    ang = np.unique(np.round(np.degrees(np.arccos(np.clip(d @ d.T, -1, 1))), 9))
    lo = ang[ang <= target_deg].max()
    hi = ang[ang > target_deg].min() if (ang > target_deg).any() else 180.0
    return float(np.float32(0.5 * (lo + hi)))


def _bits(m, N):
    P, F, W = m.shape
    return np.unpackbits(np.ascontiguousarray(m).view(np.uint8), bitorder="little").reshape(P, F, W * 32)[:, :, :N]


@pytest.mark.parametrize("name,P,S,deg", [("tiny_sphere", 32, 2048, 70), ("hand16_superquadric", 6, 8192, 50),
                                          ("hand20_tool", 2, 8192, 36)])
def test_dilated_masks(cf, name, P, S, deg):
    w = synth.workload(name, P=P, S=S)
    c = _deg_between_levels(w.bins, deg)
    q = torch.from_numpy(w.q).cuda()
    soa = torch.from_numpy(w.obj.soa()).cuda()
    poses = torch.from_numpy(w.poses).cuda()
    field = cf.build(w.hand, w.inv_h, w.bins, q, dilate_deg=c)
    inf = field.info()
    want = oracle.dilation_masks(w.bins, c)
    assert np.array_equal(np.array(inf.dilation[:w.B], np.uint32), want)
    gm, gc = cf.query_domains(field, soa, poses)
    plain = cf.build(w.hand, w.inv_h, w.bins, q)
    pm, _ = cf.query_domains(plain, soa, poses)
    torch.cuda.synchronize()
    gm = gm.cpu().numpy().view(np.uint32)
    gc = gc.cpu().numpy().view(np.uint32)
    pm = pm.cpu().numpy().view(np.uint32)
    ofd = oracle.Field(w.hand, w.q, w.inv_h, w.bins, band=True, dilate_deg=c)
    om, oc, amb = ofd.query(w.obj.soa(), w.poses, amb=True)
    gb, ob = _bits(gm, w.obj.N), _bits(om, w.obj.N)
    diff = gb != ob
    assert not np.any(diff & (amb == 0)), int(np.sum(diff & (amb == 0)))
    assert diff.sum() <= 1e-4 * diff.size
    assert np.array_equal(gc, gb.sum(axis=2).astype(np.uint32))
    assert np.all((pm & ~gm) == 0)          # dilation only adds hits
    assert (gm & ~pm).any()                  # and here it does add some
    assert cf.device_status() == 0


def test_dilated_reverse_lookup_ik(cf):
    """With dilated bins a domain point may hit through a neighbouring bin; the
    reverse lookup then takes the lowest accepted bin present, on both sides."""
    w = synth.workload("hand16_superquadric", P=3, S=8192)
    c = _deg_between_levels(w.bins, 50)
    field = cf.build(w.hand, w.inv_h, w.bins, torch.from_numpy(w.q).cuda(), want_rep=True, dilate_deg=c)
    ofd = oracle.Field(w.hand, w.q, w.inv_h, w.bins, dilate_deg=c)
    soa = w.obj.soa()
    m, cnt = ofd.query(soa, w.poses)
    tup, fing = oracle.sample_tuples(m, cnt, w.obj.N, w.T, w.k, w.seed)
    valid = (tup.reshape(-1, w.k)[:, 0] >= 0).astype(np.uint8)
    g = cf.ik_dls(field, torch.from_numpy(soa).cuda(), torch.from_numpy(w.poses).cuda(), w.T, w.k,
                  torch.from_numpy(tup).cuda(), torch.from_numpy(fing).cuda(), torch.from_numpy(valid).cuda(),
                  cf.ik_params())
    torch.cuda.synchronize()
    assert cf.device_status() == 0        # every contact found a representative
    rep = {f: oracle.rep_codes(w.hand, w.q, w.inv_h, w.bins, f) for f in range(w.hand.F)}
    o = K.ik_dls(w.hand, w.q, w.inv_h, w.bins, soa, w.poses, w.T, w.k, tup, fing, valid, rep=rep,
                 dilation=ofd.dilation)
    assert not o["miss"].any()
    # the starting sample (hence the contact link and the used-joint mask) is decided exactly
    # wherever the contact's code is clear of the band
    firm = ~o["start_amb"].any(axis=1)
    assert firm.mean() > 0.9
    assert np.array_equal(g["used"].cpu().numpy()[firm], o["used"][firm])
    n = valid.size
    fc = fing.reshape(n, w.k).astype(np.int64)
    gq = g["q"].cpu().numpy()
    att = np.nonzero(valid)[0]
    close = [np.abs(gq[u, fc[u]] - o["q"][u, fc[u]]).max() <= 1e-3 for u in att]
    assert np.mean(close) >= 0.95
