"""Batched form: many objects (different hands, sizes and pose counts) run as
one launch per kernel variant inside a replayed CUDA graph; every output must
equal the per-object calls bit for bit, on consecutive replays."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _fields(cf, S=4096):
    out = {}
    for name in ["tiny_sphere", "hand16_superquadric", "hand20_tool"]:
        w = synth.workload(name, P=1, N=64, S=S)
        out[name] = (w, cf.build(w.hand, w.inv_h, w.bins, torch.from_numpy(w.q).cuda()))
    return out


def test_batch_equals_per_object_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    fields = _fields(cf)
    specs = synth.batch_objects(10, seed=5, scale=0.05)
    items, refs = [], []
    for j, sp in enumerate(specs):
        w, field = fields[sp["hand"]]
        obj, poses = synth.batch_object_inputs(sp, w.hand)
        soa = torch.from_numpy(obj.soa()).cuda()
        pz = torch.from_numpy(poses).cuda()
        prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, obj.centroid, obj.rho, 100 + j)
        m, c = cf.query_domains(field, soa, pz)
        t, f, mar, acc = cf.score_tuples(soa, w.hand.F, m, c, prm)
        refs.append(dict(masks=m, counts=c, tuples=t, fingers=f, margin=mar, accept=acc))
        items.append(cf.batch_item(field, soa, pz, prm))
    torch.cuda.synchronize()
    batch = cf.Batch(items)
    n_launch, n_groups = batch.launches()
    assert n_launch <= 3 + 1 + 3  # <= 3 query groups, one sampling launch, score groups by (k, K)
    for rep in range(2):
        for it in items:
            for key in ["masks", "counts", "tuples", "margin"]:
                it[key].fill_(-3)
            it["fingers"].fill_(77)
            it["accept"].fill_(7)
        batch.run()
        torch.cuda.synchronize()
        for it, ref in zip(items, refs):
            for key in ["masks", "counts", "tuples", "fingers", "margin", "accept"]:
                assert torch.equal(it[key], ref[key]), (rep, key)
    assert sum(int(r["accept"].sum()) for r in refs) > 0
    assert cf.device_status() == 0
    batch.close()


def test_batch_mixing_objects_that_fill_the_gpu_alone():
    """Two large objects (their query and scoring each fill the GPU) run the
    single-object kernels inside the graph, six small ones the grouped
    launches; every output equals the per-object calls bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    fields = _fields(cf)
    specs = synth.batch_objects(6, seed=9, scale=0.05)
    specs += [dict(kind="superquadric", hand="hand16_superquadric", N=16384, P=4096, obj_seed=77, pose_seed=78),
              dict(kind="tool", hand="hand20_tool", N=12000, P=3000, obj_seed=79, pose_seed=80)]
    items, refs = [], []
    for j, sp in enumerate(specs):
        w, field = fields[sp["hand"]]
        obj, poses = synth.batch_object_inputs(sp, w.hand)
        soa = torch.from_numpy(obj.soa()).cuda()
        pz = torch.from_numpy(poses).cuda()
        prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, obj.centroid, obj.rho, 300 + j)
        m, c = cf.query_domains(field, soa, pz)
        t, f, mar, acc = cf.score_tuples(soa, w.hand.F, m, c, prm)
        refs.append(dict(masks=m, counts=c, tuples=t, fingers=f, margin=mar, accept=acc))
        items.append(cf.batch_item(field, soa, pz, prm))
    torch.cuda.synchronize()
    assert 16384 * 4096 >= 1 << 25 and 4096 * 64 >= 1 << 17 and 12000 * 3000 >= 1 << 25
    batch = cf.Batch(items)
    n_launch, n_groups = batch.launches()
    assert n_launch >= 2 + 2 * 2  # two queries and two sampling + scoring pairs run alone
    batch.run()
    torch.cuda.synchronize()
    for it, ref in zip(items, refs):
        for key in ["masks", "counts", "tuples", "fingers", "margin", "accept"]:
            assert torch.equal(it[key], ref[key]), key
    assert cf.device_status() == 0
    batch.close()
