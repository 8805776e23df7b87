"""Pins for the oracle's forward kinematics and contact vectors
(Sec. 3.1 notation; Def. "Contact Field (Point)": FK((p, n); i, q))."""
import math

import numpy as np
import pytest

import oracle
import synth


def _planar_two_link(l1, l2):
    base = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    axis = np.array([[0, 0, 1], [0, 0, 1]], np.float32)
    off = np.array([[l1, 0, 0], [l2, 0, 0]], np.float32)
    return base, axis, off


@pytest.mark.parametrize("q1,q2", [(0.0, 0.0), (0.3, 0.7), (-1.1, 2.0), (math.pi / 2, -math.pi / 3)])
def test_planar_two_link_closed_form(q1, q2):
    l1, l2 = 0.25, 0.5  # exactly representable in FP32
    base, axis, off = _planar_two_link(l1, l2)
    R, t = oracle.fk_links(2, base, axis, off, [q1, q2])
    tip = t[1] + R[1] @ off[1].astype(np.float64)
    x = l1 * math.cos(q1) + l2 * math.cos(q1 + q2)
    y = l1 * math.sin(q1) + l2 * math.sin(q1 + q2)
    assert np.allclose(tip, [x, y, 0.0], atol=1e-15)
    # the second joint sits at the end of link 1
    assert np.allclose(t[1], [l1 * math.cos(q1), l1 * math.sin(q1), 0.0], atol=1e-15)


def test_link_frames_are_rotations_and_link_lengths_preserved():
    hand = synth.hand_anthropomorphic(5)
    rng = np.random.default_rng(3)
    for f in range(hand.F):
        q = rng.uniform(hand.lo[f], hand.hi[f])
        R, t = oracle.fk_links(hand.J, hand.base[f], hand.axis[f], hand.offset[f], q)
        for j in range(hand.J):
            assert np.allclose(R[j] @ R[j].T, np.eye(3), atol=1e-7)  # axes are FP32-unit
            assert abs(np.linalg.det(R[j]) - 1.0) < 1e-6
        for j in range(hand.J - 1):
            L = np.linalg.norm(hand.offset[f][j].astype(np.float64))
            assert abs(np.linalg.norm(t[j + 1] - t[j]) - L) < 1e-7


def test_straight_finger_tip_position():
    """q = 0: a finger of the 3-finger hand points straight up the palm normal;
    the tip-cap point on the link axis sits at base + (sum of links + r) z."""
    hand = synth.hand_three_finger()
    f = 1
    p32, n32, p64, n64 = oracle.contact_vectors(hand, f, np.zeros(hand.J))
    # the tip hemisphere point closest to the link axis has the largest z
    top = int(np.argmax(p64[:, 2]))
    base_t = hand.base[f][[3, 7, 11]].astype(np.float64)
    L = float(np.sum(hand.offset[f][:, 2].astype(np.float64)))
    r = float(hand.radius[f][-1])
    assert abs(p64[top, 2] - (L + r * n64[top, 2])) < 1e-7
    assert np.allclose(p64[top, :2], base_t[:2] + r * n64[top, :2], atol=1e-7)
    assert n64[top, 2] > 0.95


def test_contact_vectors_rigid_and_fp32_close_to_fp64():
    hand = synth.hand_anthropomorphic(4)
    rng = np.random.default_rng(5)
    q0 = rng.uniform(hand.lo[2], hand.hi[2])
    q1 = rng.uniform(hand.lo[2], hand.hi[2])
    a = oracle.contact_vectors(hand, 2, q0)
    b = oracle.contact_vectors(hand, 2, q1)
    # distances between two points of the same link are configuration independent
    link = hand.surf_link[2]
    for l in np.unique(link):
        idx = np.nonzero(link == l)[0]
        da = np.linalg.norm(a[2][idx[:, None]] - a[2][idx[None, :]], axis=2)
        db = np.linalg.norm(b[2][idx[:, None]] - b[2][idx[None, :]], axis=2)
        assert np.allclose(da, db, atol=1e-12)
    assert np.allclose(np.linalg.norm(a[3], axis=1), 1.0, atol=1e-6)
    # FP32 decision values stay within a few FP32 ulps of the FP64 values
    assert np.max(np.abs(a[0] - a[2])) < 1e-6
    assert np.max(np.abs(a[1] - a[3])) < 1e-6
