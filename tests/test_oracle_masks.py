"""Pins for the oracle's contact field and contact-domain masks
(Def. Contact Field (Hand); Def. Contact Surface Representation; Sec. 4.2
contact domain CF(H) intersected with S(O); Sec. 4.3 Object Contact Query)."""
import math

import numpy as np

import oracle
import synth


def _bits(masks, N):
    P, F, W = masks.shape
    return np.unpackbits(masks.view(np.uint8), bitorder="little").reshape(P, F, W * 32)[:, :, :N]


def test_indexed_equals_brute_force_existential(tiny):
    S, P, N = 48, 6, 512
    w = synth.workload("tiny_sphere", P=P, N=N, S=S)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
    m_idx, counts = fd.query(w.obj.soa(), w.poses)
    m_bf = oracle.query_masks_brute(w.hand, w.q, w.inv_h, w.bins, w.obj.soa(), w.poses)
    assert np.array_equal(m_idx, m_bf)
    assert np.array_equal(counts, _bits(m_idx, N).sum(axis=2).astype(np.uint32))
    assert counts.sum() > 0


def test_bin_is_nearest_direction_and_ties_go_to_lowest_index():
    """A direction lands in its own bin; an exact tie goes to the lower index."""
    hand = synth.hand_three_finger()
    bins = synth.fibonacci_dirs(16)
    # object with one point per bin direction placed at a hand sample's position:
    # the contact-surface normal is -n, so an object normal of -d_b gives bin b.
    q = np.zeros((hand.F, hand.J, 1), np.float32)
    p32, n32, _, _ = oracle.contact_vectors(hand, 0, np.zeros(hand.J))
    # use the field's own code for point 0 and check it equals nearest-direction
    d64 = bins.astype(np.float64)
    for m in range(hand.M):
        b = int(np.argmax(d64 @ n32[m].astype(np.float64)))
        fd = oracle.Field(synth.Hand(**{**hand.__dict__}), q, np.float32(200.0), bins)
        codes = fd.codes(0)
        cell = np.floor(p32[m].astype(np.float64) * 200.0).astype(np.int64)
        hit = np.any(np.all(codes == np.array([*cell, b]), axis=1))
        assert hit, m
        break
    # ties: two identical directions -> the lower index wins
    bins2 = np.concatenate([bins[:3], bins[2:3], bins[3:]]).astype(np.float32)  # d_2 == d_3
    fd2 = oracle.Field(hand, q, np.float32(200.0), bins2)
    used = set(fd2.codes(0)[:, 3].tolist()) | set(fd2.codes(1)[:, 3].tolist()) | set(fd2.codes(2)[:, 3].tolist())
    assert 3 not in used


def test_cells_are_half_open_floor_cells():
    """A coordinate exactly on k/inv_h belongs to cell k; negatives floor down."""
    hand = synth.hand_three_finger()
    bins = synth.fibonacci_dirs(8)
    q = np.zeros((hand.F, hand.J, 1), np.float32)
    fd = oracle.Field(hand, q, np.float32(256.0), bins)  # 1/256 m cells: exact in FP32
    p32, n32, _, _ = oracle.contact_vectors(hand, 0, np.zeros(hand.J))
    cells = fd.codes(0)[:, :3]
    want = np.floor(p32.astype(np.float64) * 256.0).astype(np.int64)
    assert {tuple(c) for c in cells.tolist()} <= {tuple(c) for c in want.tolist()}
    assert {tuple(c) for c in want.tolist()} <= {tuple(c) for c in cells.tolist()}
    assert (want < 0).any()  # the hand has fingers on the negative x / y side


def test_contact_surface_flips_the_object_normal():
    """An object point placed on a hand contact vector (p, n) is in the domain
    iff its outward normal is -n (Def. Contact Surface Representation)."""
    hand = synth.hand_three_finger()
    bins = synth.fibonacci_dirs(8)
    q = np.zeros((hand.F, hand.J, 1), np.float32)
    fd = oracle.Field(hand, q, np.float32(200.0), bins)
    p32, n32, _, _ = oracle.contact_vectors(hand, 0, np.zeros(hand.J))
    ident = np.array([[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]], np.float32)
    opp = np.concatenate([p32.T, -n32.T], axis=0).astype(np.float32)
    same = np.concatenate([p32.T, n32.T], axis=0).astype(np.float32)
    m_opp, c_opp = fd.query(opp, ident)
    m_same, c_same = fd.query(same, ident)
    assert c_opp[0, 0] == hand.M          # every opposing contact vector hits
    assert c_same[0, 0] < hand.M          # the outward tip-cap normals do not
    # a point far from the hand never hits
    far = opp.copy()
    far[0:3] += 5.0
    _, c_far = fd.query(far, ident)
    assert c_far.sum() == 0


def test_rigid_pose_preserves_distances_of_transformed_points(tiny):
    """The query transform is rigid: pairwise distances of transformed points
    equal those of the object points (FP64 check of the pose convention R p + t,
    and of the [R | t] row-major layout)."""
    P = tiny.poses.reshape(-1, 3, 4).astype(np.float64)[:4]
    p = tiny.obj.p.astype(np.float64)[:64]
    d0 = np.linalg.norm(p[:, None] - p[None], axis=2)
    for T in P:
        q = p @ T[:, :3].T + T[:, 3]
        assert np.allclose(np.linalg.norm(q[:, None] - q[None], axis=2), d0, atol=1e-6)
        # the centroid lands at grasp_centre + d z with d in [0.08, 0.12]
        c = tiny.obj.centroid.astype(np.float64) @ T[:, :3].T + T[:, 3]
        assert np.allclose(c[:2], tiny.hand.grasp_centre[:2], atol=1e-6)
        assert 0.08 - 1e-6 <= c[2] - tiny.hand.grasp_centre[2] <= 0.12 + 1e-6


def test_identity_pose_on_pretransformed_points_gives_the_same_masks(tiny):
    """Moving the object by pose T and querying with T equals querying the
    pre-moved object with the identity (the transform is exact for the identity)."""
    w = synth.workload("tiny_sphere", P=3, N=256, S=512)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
    soa = w.obj.soa()
    m, _ = fd.query(soa, w.poses)
    ident = np.array([[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]], np.float32)
    for i in range(3):
        T = w.poses[i].reshape(3, 4)
        R, t = T[:, :3].astype(np.float64), T[:, 3].astype(np.float64)
        # the moved points and normals in FP64, rounded once to the FP32 inputs
        pre = np.empty_like(soa)
        pre[:3] = (R @ soa[:3].astype(np.float64) + t[:, None]).astype(np.float32)
        pre[3:] = (R @ soa[3:].astype(np.float64)).astype(np.float32)
        mi, _ = fd.query(pre, ident)
        # rounding the moved points to FP32 may move a handful across a cell face
        diff = np.unpackbits((mi[0] ^ m[i]).view(np.uint8)).sum()
        assert diff <= 2


def test_ambiguity_band_brackets_the_fp32_decision(tiny):
    """Every entry on which an FP32 evaluation of the same definition (the
    oracle's own diagnostic chain) decides otherwise than the FP64 oracle is
    flagged ambiguous; the flagged entries stay a small fraction."""
    w = synth.workload("tiny_sphere", P=32, S=1024)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins, band=True)
    m64, c64, amb, m32 = fd.query(w.obj.soa(), w.poses, amb=True, mask32=True)
    N = w.obj.N
    b32, b64 = _bits(m32, N), _bits(m64, N)
    assert np.all(amb[b32 != b64] == 1)
    assert amb.mean() < 0.05
    assert np.array_equal(c64, b64.sum(axis=2).astype(np.uint32))


def test_field_code_sets_nest():
    """The band's code sets bracket the FP64 decisions: sure <= fp64 <= possible,
    and the FP32 diagnostic codes lie within the same brackets."""
    w = synth.workload("hand16_superquadric", P=1, S=2048)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins, band=True)
    for f in range(w.hand.F):
        sets = {k: set(map(tuple, fd.codes(f, k).tolist())) for k in ("fp64", "fp32", "possible", "sure")}
        assert sets["sure"] <= sets["fp64"] <= sets["possible"]
        assert sets["sure"] <= sets["fp32"] <= sets["possible"]
        assert len(sets["possible"] - sets["sure"]) < 0.05 * len(sets["fp64"])


def test_paper_normal_bin_cone_half_angle():
    """Sec. 4.3: 256 directions give each a cone half-angle of about 7 degrees.
    The equal-area cap of 1/256 of the sphere has half-angle arccos(1 - 2/256);
    the oracle's binning of random directions onto a 256-point Fibonacci set
    stays within that scale."""
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
    B = g["normal_bins"]["B"]
    want = g["normal_bins"]["cone_half_angle_deg_about"]
    cap = math.degrees(math.acos(1 - 2 / B))
    assert round(cap) == want
    # nearest-bin angles of random directions through the oracle's field codes:
    hand = synth.hand_three_finger()
    bins = synth.fibonacci_dirs(B)
    rng = np.random.default_rng(0)
    ang = []
    q = np.zeros((hand.F, hand.J, 1), np.float32)
    fd = oracle.Field(hand, q, np.float32(100.0), bins)
    ident = np.array([[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]], np.float32)
    _, _, p64, n64 = oracle.contact_vectors(hand, 0, np.zeros(hand.J))
    codes = fd.codes(0)
    for m in range(hand.M):
        cm = codes[np.all(codes[:, :3] == np.floor(p64[m] * np.float64(np.float32(100.0))).astype(np.int64), axis=1)]
        d = bins[cm[:, 3]].astype(np.float64)
        ang.append(np.degrees(np.arccos(np.clip(d @ n64[m], -1, 1))).min())
    ang = np.array(ang)
    assert ang.max() < 1.5 * cap and np.median(ang) < cap
