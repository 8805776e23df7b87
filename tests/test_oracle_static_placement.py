"""Pins of the oracle's static-link placement (Sec. 5.2, last paragraph): the
chosen object point lands on the palm's top face at the drawn point with its
outward normal facing into the palm; a convex object touching the plane there
never penetrates (closed form); a constructed two-point object is rejected
exactly when its second point sinks into the palm by more than the margin."""
import math

import numpy as np

import synth
from oracle import placement as PL


def test_contact_point_lands_on_the_palm_face_with_opposed_normal():
    w = synth.workload("hand16_superquadric", P=1, S=64)
    lo, hi = w.hand.palm_lo.astype(np.float64), w.hand.palm_hi.astype(np.float64)
    soa = w.obj.soa()
    poses, xs, valid, _ = PL.place_static(lo, hi, soa, 200, seed=3)
    for i in range(200):
        T = poses[i].astype(np.float64).reshape(3, 4)
        R, t = T[:, :3], T[:, 3]
        q = R @ soa[0:3, xs[i]].astype(np.float64) + t
        n = R @ soa[3:6, xs[i]].astype(np.float64)
        assert abs(q[2] - hi[2]) <= 1e-6
        assert lo[0] - 1e-6 <= q[0] <= hi[0] + 1e-6 and lo[1] - 1e-6 <= q[1] <= hi[1] + 1e-6
        assert np.allclose(n / np.linalg.norm(n), [0, 0, -1], atol=1e-5)
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-6)
    assert valid.all()  # the superquadric is convex: nothing crosses the face plane


def test_convex_sphere_is_never_rejected_and_draws_cover_the_face():
    w = synth.workload("tiny_sphere", P=1, S=64)
    lo, hi = w.hand.palm_lo, w.hand.palm_hi
    poses, xs, valid, amb = PL.place_static(lo, hi, w.obj.soa(), 300, seed=9)
    assert valid.all() and not amb.any()
    c = np.array([poses[i].reshape(3, 4)[:, :3].astype(np.float64) @ w.obj.soa()[0:3, xs[i]] +
                  poses[i].reshape(3, 4)[:, 3] for i in range(300)])
    # the contact points spread over the face: each quarter of the rectangle holds some
    mx, my = 0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1])
    for sx in (c[:, 0] < mx, c[:, 0] >= mx):
        for sy in (c[:, 1] < my, c[:, 1] >= my):
            assert (sx & sy).sum() > 30


def test_two_point_object_rejected_iff_the_second_point_penetrates():
    lo, hi = np.array([-0.05, -0.05, -0.02]), np.array([0.05, 0.05, 0.0])
    for dz, depth_ok in [(0.01, False), (-0.01, True), (0.0015, True), (0.0025, False)]:
        # point 0 at the origin with outward normal +z lands on the face with its normal down, so
        # object +z maps to palm -z: a second point dz above it in the object frame sinks dz below the face
        soa = np.zeros((6, 2), np.float32)
        soa[5, 0] = 1.0
        soa[2, 1] = dz
        soa[5, 1] = 1.0
        poses, xs, valid, amb = PL.place_static(lo, hi, soa, 64, seed=1, pen_margin=2e-3)
        sel = xs == 0
        assert sel.any()
        q = np.array([poses[i].reshape(3, 4)[:, :3].astype(np.float64) @ soa[0:3, 1] + poses[i].reshape(3, 4)[:, 3]
                      for i in np.nonzero(sel)[0]])
        inside = (np.abs(q[:, 0]) <= 0.05) & (np.abs(q[:, 1]) <= 0.05)
        want = np.where(inside, depth_ok, True).astype(np.uint8)
        assert np.array_equal(valid[sel], want), (dz, valid[sel], want)
        assert abs(q[:, 2] + dz).max() < 1e-6
