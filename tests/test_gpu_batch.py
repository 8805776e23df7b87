"""Batched form: many objects (different hands, sizes and pose counts) run as
one persistent launch per stage (query, sampling, scoring) inside a replayed
CUDA graph; every output must equal the per-object calls bit for bit, on
consecutive replays (the query's work counter returns to zero by itself)."""
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
    assert n_launch == 3  # one query launch for the three hands, one sampling launch, one scoring launch
    for rep in range(3):
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


def test_batch_mixing_large_and_small_objects_in_one_launch_per_stage():
    """Two large objects (each fills the GPU alone) and six small ones, one
    with a single pose and one with a pose count that leaves a ragged last
    query item, run in the same three launches; every output equals the
    per-object calls bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    fields = _fields(cf)
    specs = synth.batch_objects(4, seed=9, scale=0.05)
    specs += [dict(kind="superquadric", hand="hand16_superquadric", N=16384, P=4096, obj_seed=77, pose_seed=78),
              dict(kind="tool", hand="hand20_tool", N=12000, P=3001, obj_seed=79, pose_seed=80),
              dict(kind="tool", hand="tiny_sphere", N=100, P=1, obj_seed=81, pose_seed=82),
              dict(kind="superquadric", hand="hand20_tool", N=33, P=7, obj_seed=83, pose_seed=84)]
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
    batch = cf.Batch(items)
    n_launch, n_groups = batch.launches()
    assert n_launch == 3 and n_groups == 2
    for _ in range(2):
        batch.run()
        torch.cuda.synchronize()
        for it, ref in zip(items, refs):
            for key in ["masks", "counts", "tuples", "fingers", "margin", "accept"]:
                assert torch.equal(it[key], ref[key]), key
    assert cf.device_status() == 0
    batch.close()


def test_batch_with_two_edge_counts_scores_in_two_launches():
    """Objects whose pyramids have different edge counts K share the query and
    sampling launches and take one scoring launch per (k, K)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    fields = _fields(cf)
    specs = synth.batch_objects(4, seed=13, scale=0.05)
    items, refs = [], []
    for j, sp in enumerate(specs):
        w, field = fields[sp["hand"]]
        obj, poses = synth.batch_object_inputs(sp, w.hand)
        soa = torch.from_numpy(obj.soa()).cuda()
        pz = torch.from_numpy(poses).cuda()
        prm = cf.score_params(w.T, w.k, w.mu, 8 if j % 2 else 6, w.eps, obj.centroid, obj.rho, 500 + j)
        m, c = cf.query_domains(field, soa, pz)
        t, f, mar, acc = cf.score_tuples(soa, w.hand.F, m, c, prm)
        refs.append(dict(masks=m, counts=c, tuples=t, fingers=f, margin=mar, accept=acc))
        items.append(cf.batch_item(field, soa, pz, prm))
    torch.cuda.synchronize()
    batch = cf.Batch(items)
    assert batch.launches()[0] == 4
    batch.run()
    torch.cuda.synchronize()
    for it, ref in zip(items, refs):
        for key in ["masks", "counts", "tuples", "fingers", "margin", "accept"]:
            assert torch.equal(it[key], ref[key]), key
    assert cf.device_status() == 0
    batch.close()
