"""Launch shapes and the autotuner: every shape gives the same results bit for
bit (the kernels' outputs depend only on the inputs), the accessors check
their ranges, and cf_autotune leaves a valid tuning in force."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_07418_b300 as cf
    yield cf
    cf.set_tuning(4, 8, 0)


def _run(cf, w, field, soa, poses):
    masks, counts = cf.query_domains(field, soa, poses)
    prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed)
    tup, fing, margin, accept = cf.score_tuples(soa, w.hand.F, masks, counts, prm)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in (masks, counts, tup, fing, margin, accept)]


def test_tuning_accessors(cf):
    cf.set_tuning(16, 4, 1)
    assert cf.get_tuning() == {"query_poses_per_block": 16, "score_refill": 4, "score_blocks_per_sm": 1}
    for bad in ((17, 8, 0), (8, 3, 0), (8, 8, 4), (0, 8, 0), (8, 2, 0)):
        with pytest.raises(cf.CfError):
            cf.set_tuning(*bad)
    assert cf.get_tuning()["query_poses_per_block"] == 16
    cf.set_tuning(4, 8, 0)


@pytest.mark.parametrize("name,P", [("tiny_sphere", 37), ("hand16_superquadric", 45)])
def test_results_do_not_depend_on_shape(cf, name, P):
    w = synth.workload(name, P=P, S=4096)  # P not a multiple of any block size: ragged last block
    field = cf.build(w.hand, w.inv_h, w.bins, torch.from_numpy(w.q).cuda())
    soa = torch.from_numpy(w.obj.soa()).cuda()
    poses = torch.from_numpy(w.poses).cuda()
    ref = None
    for shape in ((8, 8, 0), (4, 4, 1), (16, 16, 2), (16, 4, 3), (6, 8, 0), (5, 16, 1), (10, 8, 0), (1, 8, 0)):
        cf.set_tuning(*shape)
        out = _run(cf, w, field, soa, poses)
        if ref is None:
            ref = out
        else:
            for a, b in zip(ref, out):
                assert np.array_equal(a, b), shape
    cf.set_tuning(4, 8, 0)


def test_autotune_and_batch_shapes(cf):
    ws = [synth.workload("tiny_sphere", P=40, S=2048), synth.workload("hand16_superquadric", P=24, S=4096)]
    items, keep, outs = [], [], []
    for w in ws:
        field = cf.build(w.hand, w.inv_h, w.bins, torch.from_numpy(w.q).cuda())
        soa = torch.from_numpy(w.obj.soa()).cuda()
        poses = torch.from_numpy(w.poses).cuda()
        it = cf.batch_item(field, soa, poses, cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho,
                                                              w.seed))
        items.append(it)
        keep.append((field, soa, poses, it))
    tuning, ms = cf.autotune(items, reps=2)
    # candidates 4, 8, 16 and 32 / slots: 10 for the 3-finger hand (8 for the 4-finger one)
    assert tuning["query_poses_per_block"] in (4, 8, 10, 16) and tuning["score_refill"] in (4, 8, 16)
    assert cf.get_tuning() == tuning and ms[0] > 0 and ms[1] > 0
    # a batch created under two different tunings gives identical outputs
    res = []
    for shape in ((4, 4, 0), (16, 16, 0)):
        cf.set_tuning(*shape)
        b = cf.Batch(items)
        b.run()
        torch.cuda.synchronize()
        res.append([it[key].cpu().numpy().copy() for it in items
                    for key in ("masks", "counts", "tuples", "fingers", "margin", "accept")])
        b.close()
    for a, c in zip(*res):
        assert np.array_equal(a, c)
    cf.set_tuning(4, 8, 0)
