"""Checks of the seeded input generators against the recipe they state: the
synthetic hands, objects, joint samples and palm poses that stand in for the
paper's assets (Sec. 6) and its canonical placement (Sec. 5.2).  The
generators hold none of the method's arithmetic; these tests only make sure
that the inputs both sides consume have the shapes, sizes, distributions and
geometry the workloads claim."""
import math

import numpy as np
import pytest
from scipy import stats

import synth


def _seg_dist(x, a, b):
    """Distance of points x [n,3] to the segment a-b."""
    ab = b - a
    t = np.clip(((x - a) @ ab) / max(ab @ ab, 1e-300), 0.0, 1.0)
    return np.linalg.norm(x - (a + t[:, None] * ab), axis=1)


def test_fibonacci_bins_are_unit_and_equal_area_bands():
    for B in (8, 16, 32, 256):
        d32 = synth.fibonacci_dirs(B)
        assert d32.shape == (B, 3) and d32.dtype == np.float32 and d32.flags.c_contiguous
        d = d32.astype(np.float64)
        assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
        # equal-area bands: z_i = 1 - (2i + 1) / B (Archimedes), all directions distinct
        assert np.allclose(d[:, 2], 1.0 - (2 * np.arange(B) + 1) / B, atol=1e-6)
        g = d @ d.T - 2 * np.eye(B)
        assert g.max() < 1 - 1e-3


@pytest.mark.parametrize("kind,F,J,lens,r,lo,hi", [
    ("three", 3, 3, [0.04, 0.03, 0.025], 0.008, [0.0] * 3, [1.6] * 3),
    ("anthro4", 4, 4, [0.0, 0.054, 0.038, 0.044], 0.009, [-0.35, 0, 0, 0], [0.35, 1.6, 1.6, 1.6]),
    ("anthro5", 5, 4, [0.0, 0.054, 0.038, 0.044], 0.009, [-0.35, 0, 0, 0], [0.35, 1.6, 1.6, 1.6]),
])
def test_hands_have_the_stated_links_limits_and_surface_points(kind, F, J, lens, r, lo, hi):
    h = synth._make_hand(kind)
    assert (h.F, h.J, h.M) == (F, J, 112)  # 3 capsule links x 4 stations x 8 angles + 16 tip points
    assert np.allclose(np.linalg.norm(h.offset, axis=2), np.asarray(lens)[None, :], atol=1e-7)
    assert np.allclose(np.linalg.norm(h.axis, axis=2), 1.0, atol=1e-7)
    assert np.allclose(h.lo, np.asarray(lo, np.float32)[None, :]) and np.allclose(h.hi, np.asarray(hi)[None, :])
    nz = np.asarray(lens) > 0
    assert np.allclose(h.radius[:, nz], r) and np.all(h.radius[:, ~nz] == 0)
    for f in range(F):
        R = h.base[f].reshape(3, 4)[:, :3].astype(np.float64)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6) and np.linalg.det(R) > 0
        for j in np.unique(h.surf_link[f]):
            assert nz[j]
            m = h.surf_link[f] == j
            p = h.surf_p[f][m].astype(np.float64)
            n = h.surf_n[f][m].astype(np.float64)
            off = h.offset[f, j].astype(np.float64)
            # every point sits on its capsule's surface, its normal points away from the axis
            assert np.allclose(_seg_dist(p, np.zeros(3), off), h.radius[f, j], atol=1e-6)
            assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-6)
            assert np.all(_seg_dist(p + 1e-3 * n, np.zeros(3), off) > h.radius[f, j] + 9e-4)
        counts = np.bincount(h.surf_link[f], minlength=J)[nz]
        assert counts.tolist() == [32, 32, 48]  # the distal link carries the tip cap
    if kind != "three":
        thumb = h.base[-1].reshape(3, 4)[:, :3]
        assert np.allclose(thumb, [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-7)  # 90 deg about the palm normal


def test_joint_samples_are_uniform_in_the_limits():
    h = synth.hand_anthropomorphic(4)
    q = synth.joint_samples(h, 20000, seed=5)
    assert q.shape == (4, 4, 20000) and q.dtype == np.float32 and q.flags.c_contiguous
    for f in range(4):
        for j in range(4):
            lo, hi = float(h.lo[f, j]), float(h.hi[f, j])
            assert q[f, j].min() >= lo and q[f, j].max() <= hi
            assert stats.kstest((q[f, j] - lo) / (hi - lo), "uniform").pvalue > 1e-4
    assert not np.array_equal(q, synth.joint_samples(h, 20000, seed=6))
    assert np.array_equal(q, synth.joint_samples(h, 20000, seed=5))


def test_sphere_points_are_area_uniform_with_radial_normals():
    o = synth.sphere(20000, 0.04, seed=1000)
    p, n = o.p.astype(np.float64), o.n.astype(np.float64)
    assert np.allclose(np.linalg.norm(p, axis=1), 0.04, atol=1e-8)
    assert np.allclose(n, p / 0.04, atol=1e-6)
    # area-uniform on a sphere <=> each coordinate uniform on [-r, r] (Archimedes)
    for a in range(3):
        assert stats.kstest((p[:, a] + 0.04) / 0.08, "uniform").pvalue > 1e-4
    assert np.isclose(o.rho, np.max(np.linalg.norm(p - o.centroid, axis=1)), rtol=1e-6)


def _superquadric_shape(seed):
    rng = np.random.default_rng(seed)  # the generator's first draws: axes, then exponents
    return rng.uniform(0.03, 0.08, 3), rng.uniform(0.3, 1.5, 2)


def test_superquadric_points_on_the_surface_with_gradient_normals():
    seed = 1000
    o = synth.superquadric(8192, seed)
    a, (e1, e2) = _superquadric_shape(seed)
    assert np.all((a >= 0.03) & (a <= 0.08)) and 0.3 <= e1 <= 1.5 and 0.3 <= e2 <= 1.5
    p, n = o.p.astype(np.float64), o.n.astype(np.float64)

    def io(x):  # inside-outside function, 1 on the surface
        u = np.abs(x / a)
        return (u[:, 0] ** (2 / e2) + u[:, 1] ** (2 / e2)) ** (e2 / e1) + u[:, 2] ** (2 / e1)

    assert np.all(np.abs(p) <= a[None, :] * (1 + 1e-6))
    ok = np.abs(io(p) - 1.0) < 1e-3
    assert ok.mean() > 0.999
    # normal = normalised gradient of the inside-outside function (central differences)
    hs = 1e-7
    g = np.stack([(io(p + hs * e) - io(p - hs * e)) / (2 * hs) for e in np.eye(3)], axis=1)
    gn = np.linalg.norm(g, axis=1)
    fine = ok & (gn > 1e-3) & np.all(np.abs(p) > 1e-4, axis=1)
    cos = np.sum(n[fine] * g[fine], axis=1) / gn[fine]
    assert fine.mean() > 0.95 and np.quantile(cos, 0.001) > 1 - 1e-3
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-6)


def test_tool_composite_points_lie_on_the_union_surface_with_outward_normals():
    o = synth.tool_composite(8192, seed=1000)
    p, n = o.p.astype(np.float64), o.n.astype(np.float64)
    assert p.shape == (8192, 3) and np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-6)
    # rebuild the union's inside test from the same seeded primitive poses
    rng = np.random.default_rng(1000)
    Rh = synth._rand_rot(rng, 0.3)
    th = np.array([0.087, 0.0, 0.0]) + rng.uniform(-0.004, 0.004, 3)
    Rt = synth._rand_rot(rng, 0.4)
    tt = np.array([-0.105, 0.0, 0.0]) + rng.uniform(-0.004, 0.004, 3)
    hb = np.array([0.01, 0.03, 0.015])

    def inside(x):
        cyl = (np.abs(x[:, 0]) <= 0.075) & (x[:, 1] ** 2 + x[:, 2] ** 2 <= 0.012 ** 2)
        box = np.all(np.abs((x - th) @ Rh) <= hb, axis=1)
        y = (x - tt) @ Rt
        tor = (np.sqrt(y[:, 0] ** 2 + y[:, 1] ** 2) - 0.03) ** 2 + y[:, 2] ** 2 <= 0.006 ** 2
        return cyl | box | tor

    # on the union's boundary: just inside behind the normal, outside in front of it
    assert inside(p - 1e-5 * n).mean() > 0.999
    assert (~inside(p + 1e-5 * n)).mean() > 0.999
    # every primitive contributes (handle, head and torus all present)
    assert (p[:, 0] > 0.08).sum() > 100 and (p[:, 0] < -0.08).sum() > 100 and (np.abs(p[:, 0]) < 0.05).sum() > 1000


def test_points_are_morton_sorted():
    o = synth.superquadric(8192, 1000)
    p = o.p.astype(np.float64)
    step = np.linalg.norm(np.diff(p, axis=0), axis=1).mean()
    shuffled = p[np.random.default_rng(0).permutation(len(p))]
    assert step < 0.1 * np.linalg.norm(np.diff(shuffled, axis=0), axis=1).mean()


def test_palm_poses_place_the_centroid_and_rotate_uniformly():
    g = np.array([0.01, 0.02, 0.0])
    c = np.array([0.005, -0.003, 0.002], np.float32)
    P = 20000
    X = synth.palm_poses(P, seed=2, grasp_centre=g, obj_centroid=c).astype(np.float64).reshape(P, 3, 4)
    R, t = X[:, :, :3], X[:, :, 3]
    assert np.allclose(np.einsum("pij,pkj->pik", R, R), np.eye(3)[None], atol=2e-6)
    assert np.allclose(np.linalg.det(R), 1.0, atol=2e-6)
    img = np.einsum("pij,j->pi", R, c.astype(np.float64)) + t
    assert np.allclose(img[:, :2], g[None, :2], atol=1e-6)
    d = img[:, 2] - g[2]
    assert d.min() >= 0.08 - 1e-6 and d.max() <= 0.12 + 1e-6
    assert stats.kstest((d - 0.08) / 0.04, "uniform").pvalue > 1e-4
    # Haar measure on SO(3): rotation angle theta has CDF (theta - sin theta) / pi
    th = np.arccos(np.clip((np.trace(R, axis1=1, axis2=2) - 1) / 2, -1, 1))
    assert stats.kstest(th, lambda x: (x - np.sin(x)) / math.pi).pvalue > 1e-4
    # and the rotation axis is isotropic: each rotated basis vector is uniform on S^2
    for col in range(3):
        assert stats.kstest((R[:, 2, col] + 1) / 2, "uniform").pvalue > 1e-4


def test_batch_objects_follow_the_log_uniform_mix():
    specs = synth.batch_objects(64, seed=0)
    assert len(specs) == 64
    assert [s["kind"] for s in specs].count("superquadric") == 32
    N = np.array([s["N"] for s in specs])
    P = np.array([s["P"] for s in specs])
    assert N.min() >= 2048 and N.max() <= 131072 and P.min() >= 4096 and P.max() <= 32768
    assert stats.kstest((np.log(N) - np.log(2048)) / np.log(64), "uniform").pvalue > 1e-3
    assert {s["hand"] for s in specs} == {"tiny_sphere", "hand16_superquadric", "hand20_tool"}
    assert len({s["obj_seed"] for s in specs}) == 64


def test_named_workloads_have_the_stated_sizes():
    w = synth.workload("tiny_sphere")
    assert (w.hand.F, w.hand.J, w.obj.N, w.S, w.B, w.P, w.T, w.k) == (3, 3, 2048, 4096, 8, 256, 16, 3)
    assert (w.h, w.mu, w.K) == (0.005, 0.5, 8) and w.inv_h == np.float32(200.0)
    for name, sizes in (("hand16_superquadric", (4, 4, 16384, 65536, 16, 8192, 64, 0.0025, 0.5)),
                        ("hand20_tool", (5, 4, 65536, 131072, 32, 32768, 128, 0.002, 0.4))):
        m = synth.WORKLOADS[name]
        got = (int(m["hand"][-1]), 4, m["N"], m["S"], m["B"], m["P"], m["T"], m["h"], m["mu"])
        assert got == sizes, name
