"""Fine-grained contact field (Sec. 4.4) on the GPU, through the C ABI: one
table slot per (finger, link) patch, queried together, then merged per
dependency group (Sec. 5.3).  The patch table and the patch domains follow the
FP64 oracle's per-patch fields under the acceptance rule of parity_checks; the
merged domains equal the per-finger field's domains bit for bit (the patches
partition each finger's samples), and so do the tuples and margins sampled
from them."""
import numpy as np
import pytest

import oracle
import synth
from parity_checks import check_field, check_masks, u32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    return cf


@pytest.mark.parametrize("name,P,S,n_slots", [("tiny_sphere", 16, 2048, 9), ("hand16_superquadric", 6, 4096, 12),
                                              ("hand20_tool", 3, 4096, 15)])
def test_patch_field_against_oracle_and_finger_field(cf, name, P, S, n_slots):
    w = synth.workload(name, P=P, S=S)
    q = torch.from_numpy(w.q).cuda()
    pfield = cf.build(w.hand, w.inv_h, w.bins, q, patches=True)
    ffield = cf.build(w.hand, w.inv_h, w.bins, q)
    inf = pfield.info()
    pf = oracle.PatchFields(w.hand, w.q, w.inv_h, w.bins, band=True)
    assert inf.n_slots == n_slots == pfield.n_slots == len(pf.slots)
    assert [(int(inf.slot_finger[s]), int(inf.slot_link[s])) for s in range(n_slots)] == pf.slots
    assert ffield.info().n_slots == w.hand.F and list(ffield.info().slot_link[:w.hand.F]) == [-1] * w.hand.F
    check_field(pfield, pf, n_slots, name)
    soa = torch.from_numpy(w.obj.soa()).cuda()
    poses = torch.from_numpy(w.poses).cuda()
    pm, pc = cf.query_domains(pfield, soa, poses)
    fm, fc = cf.query_domains(ffield, soa, poses)
    W = (w.obj.N + 31) // 32
    mm, mc = cf.merge_domains(pfield, pm, W)
    torch.cuda.synchronize()
    assert pm.shape == (P, n_slots, W)
    om, oc, amb = pf.query(w.obj.soa(), w.poses, amb=True)
    check_masks(u32(pm), u32(pc), om, oc, amb, w.obj.N, label=f"{name} patches")
    # merged patch domains = the finger field's domains, bit for bit
    assert torch.equal(mm, fm) and torch.equal(mc, fc)
    prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed)
    a = cf.score_tuples(soa, w.hand.F, mm, mc, prm)
    b = cf.score_tuples(soa, w.hand.F, fm, fc, prm)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert int(pc.sum()) >= int(fc.sum()) > 0
    assert cf.device_status() == 0


def test_patch_field_limits(cf):
    w = synth.workload("tiny_sphere", P=2, S=256)
    q = torch.from_numpy(w.q).cuda()
    with pytest.raises(cf.CfError, match="want_rep"):
        cf.build(w.hand, w.inv_h, w.bins, q, patches=True, want_rep=True)
    pfield = cf.build(w.hand, w.inv_h, w.bins, q, patches=True)
    soa = torch.from_numpy(w.obj.soa()).cuda()
    prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, 1)
    with pytest.raises(cf.CfError, match="patch field"):
        cf.Batch([cf.batch_item(pfield, soa, torch.from_numpy(w.poses).cuda(), prm)])
    # merging a plain field's rows copies them
    ffield = cf.build(w.hand, w.inv_h, w.bins, q)
    fm, fc = cf.query_domains(ffield, soa, torch.from_numpy(w.poses).cuda())
    mm, mc = cf.merge_domains(ffield, fm, (w.obj.N + 31) // 32)
    torch.cuda.synchronize()
    assert torch.equal(mm, fm) and torch.equal(mc, fc)
    assert cf.device_status() == 0
