"""Pins of the placement and preprocessing oracle (Sec. 5.2, Sec. 5.1):
canonical rotations are proper and Haar-uniform, canonical centroids land on
the placement segment, an exhaustive pose puts the chosen object point on the
chosen field code (so the domain query reports the contact), and the small-box
test removes points in a slot narrower than the box and keeps them otherwise."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import kinematics as K
from oracle import placement as PL


def _R(poses):
    return poses.reshape(-1, 3, 4)[:, :, :3].astype(np.float64), poses.reshape(-1, 3, 4)[:, :, 3].astype(np.float64)


def test_canonical_rotations_uniform_and_centroid_on_segment():
    c = np.array([0.01, -0.02, 0.005])
    g = np.array([0.0, 0.02, 0.0])
    up = np.array([0.0, 0.0, 1.0])
    P = 3000
    poses = PL.place_canonical(P, c, g, up, 0.08, 0.12, seed=4)
    R, t = _R(poses)
    assert np.allclose(R @ np.transpose(R, (0, 2, 1)), np.eye(3), atol=1e-6)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-6)
    # Haar measure on SO(3): E[R] = 0 (so E[trace] = 0)
    assert np.abs(R.mean(axis=0)).max() < 0.05
    cw = np.einsum("pij,j->pi", R, c) + t
    d = cw - g
    assert np.allclose(d[:, :2], 0.0, atol=1e-6)
    assert d[:, 2].min() >= 0.08 - 1e-6 and d[:, 2].max() <= 0.12 + 1e-6
    assert abs(d[:, 2].mean() - 0.1) < 0.002  # uniform offset


@pytest.fixture(scope="module")
def small_field():
    w = synth.workload("tiny_sphere", P=4, S=512)
    return w, oracle.Field(w.hand, w.q, w.inv_h, w.bins)


def test_table_order(small_field):
    w, fd = small_field
    c = PL.table_codes(fd)
    assert len(c) == int(fd.n_codes().sum())
    lo = c[:, :3].min(axis=0)
    dims = c[:, :3].max(axis=0) - lo + 1
    cell = ((c[:, 2] - lo[2]) * dims[1] + (c[:, 1] - lo[1])) * dims[0] + (c[:, 0] - lo[0])
    key = (cell * 64 + c[:, 3]) * 64 + c[:, 4]
    assert np.all(np.diff(key) > 0)


def test_exhaustive_places_a_contact(small_field):
    w, fd = small_field
    soa = w.obj.soa()
    P = 64
    poses, chosen, x = PL.place_exhaustive(fd, w.bins, w.inv_h, soa, P, seed=9)
    R, t = _R(poses)
    assert np.allclose(R @ np.transpose(R, (0, 2, 1)), np.eye(3), atol=1e-6)
    pts = soa[0:3, x].T.astype(np.float64)
    nrm = soa[3:6, x].T.astype(np.float64)
    cell_centre = (chosen[:, :3] + 0.5) / float(np.float32(w.inv_h))
    assert np.allclose(np.einsum("pij,pj->pi", R, pts) + t, cell_centre, atol=2e-6)
    d = w.bins[chosen[:, 4]].astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    assert np.allclose(-np.einsum("pij,pj->pi", R, nrm / np.linalg.norm(nrm, axis=1, keepdims=True)), d, atol=2e-6)
    # the domain query of each placed pose reports the chosen point for the chosen finger
    masks, _ = fd.query(soa, poses)
    f = chosen[:, 3]
    bits = (masks[np.arange(P), f, x >> 5] >> (x & 31).astype(np.uint32)) & 1
    assert bits.all()


def _slot_object(gap, n=40, size=0.02):
    """Two facing planes z = 0 (normal +z) and z = gap (normal -z): a slot."""
    u = np.linspace(-size, size, n)
    X, Y = np.meshgrid(u, u)
    lower = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    upper = lower + np.array([0, 0, gap])
    p = np.concatenate([lower, upper])
    nrm = np.concatenate([np.tile([0, 0, 1.0], (X.size, 1)), np.tile([0, 0, -1.0], (X.size, 1))])
    return np.ascontiguousarray(np.concatenate([p.T, nrm.T]).astype(np.float32))


@pytest.mark.parametrize("gap,side,removed", [(0.003, 0.006, True), (0.012, 0.004, False)])
def test_small_box_test_on_a_slot(gap, side, removed):
    soa = _slot_object(gap)
    # grid nodes off the planes: on a plane a point-sampled SDF's sign is undefined
    lo = np.array([-0.0303, -0.0303, -0.0103], np.float32)
    h = 0.001
    dims = (61, 61, 10 + int(gap / h) + 12)
    grid, amb = K.sdf_grid(soa, lo, h, dims)
    keep, ambig = PL.concave_keep(soa, grid, amb, lo, h, side, 0.001)
    inner = np.abs(soa[0]) < 0.012  # away from the slot's open edges
    inner &= np.abs(soa[1]) < 0.012
    if removed:
        assert not keep[inner].any()
    else:
        assert keep[inner].all()
    assert not ambig[inner].any()


def test_small_box_keeps_a_convex_object():
    soa = synth.sphere(2048, 0.04, seed=2).soa()
    lo = np.array([-0.06, -0.06, -0.06], np.float32)
    grid, amb = K.sdf_grid(soa, lo, 0.003, (41, 41, 41))
    keep, _ = PL.concave_keep(soa, grid, amb, lo, 0.003, 0.004, 0.001)
    assert keep.mean() > 0.99
