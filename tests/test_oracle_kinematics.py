"""Pins of the FP64 kinematics oracle (Sec. 5.5 kinematics optimisation,
Sec. 5.6 post-processing) against closed forms, finite differences, an
independent least-squares route, brute force and analytic distance fields."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import kinematics as K


def _hand(name, base, axis, offset, lo, hi, radius, M=1):
    F, J = axis.shape[:2]
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    sp = np.zeros((F, M, 3))
    sn = np.zeros((F, M, 3))
    sn[..., 2] = 1.0
    return synth.Hand(name=name, base=f32(base), axis=f32(axis), offset=f32(offset), lo=f32(lo), hi=f32(hi),
                      radius=f32(radius), surf_p=f32(sp), surf_n=f32(sn),
                      surf_link=np.zeros((F, M), np.int32), grasp_centre=np.zeros(3))


def _planar_2link(l1=0.05, l2=0.03):
    base = np.array([[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]], np.float64)
    axis = np.array([[[0, 0, 1], [0, 0, 1]]], np.float64)
    offset = np.array([[[l1, 0, 0], [l2, 0, 0]]], np.float64)
    return _hand("planar2", base, axis, offset, [[-3, -3]], [[3, 3]], [[0.01, 0.01]])


def test_chain_planar_closed_form():
    """Two parallel axes: the tip is (l1 cos q1 + l2 cos(q1+q2), l1 sin q1 + l2 sin(q1+q2))."""
    l1, l2 = 0.05, 0.03
    hand = _planar_2link(l1, l2)
    rng = np.random.default_rng(1)
    q = rng.uniform(-3, 3, (64, 2))
    R, t, aw = K.chain(hand, np.zeros(64, np.int64), q)
    tip = t[:, 1] + np.einsum("gij,j->gi", R[:, 1], hand.offset[0, 1].astype(np.float64))
    l1f, l2f = float(np.float32(l1)), float(np.float32(l2))
    ex = l1f * np.cos(q[:, 0]) + l2f * np.cos(q[:, 0] + q[:, 1])
    ey = l1f * np.sin(q[:, 0]) + l2f * np.sin(q[:, 0] + q[:, 1])
    assert np.allclose(tip[:, 0], ex, atol=1e-15) and np.allclose(tip[:, 1], ey, atol=1e-15)
    assert np.allclose(tip[:, 2], 0.0, atol=1e-15)
    assert np.allclose(aw, [0, 0, 1])  # both joint axes stay the palm z axis


def test_chain_matches_c_fk():
    hand = synth.hand_anthropomorphic(4)
    rng = np.random.default_rng(2)
    for f in range(hand.F):
        q = rng.uniform(hand.lo[f], hand.hi[f], (8, hand.J))
        R, t, _ = K.chain(hand, np.full(8, f), q)
        for g in range(8):
            Rc, tc = oracle.fk_links(hand.J, hand.base[f], hand.axis[f], hand.offset[f], q[g])
            assert np.allclose(R[g], Rc, atol=1e-14) and np.allclose(t[g], tc, atol=1e-14)


def _attached_point(hand, f, l, pl, q):
    R, t, _ = K.chain(hand, f, q)
    g = np.arange(len(f))
    return np.einsum("gij,gj->gi", R[g, l], pl) + t[g, l]


def test_jacobian_central_differences():
    hand = synth.hand_anthropomorphic(4)
    rng = np.random.default_rng(3)
    G = 64
    f = rng.integers(0, hand.F, G)
    m = rng.integers(0, hand.M, G)
    l = hand.surf_link[f, m].astype(np.int64)
    pl = hand.surf_p[f, m].astype(np.float64)
    q = rng.uniform(hand.lo[f], hand.hi[f])
    R, t, aw = K.chain(hand, f, q)
    x = _attached_point(hand, f, l, pl, q)
    Jm = K.jacobian(aw, t, l, x)
    eps = 1e-6
    for j in range(hand.J):
        dq = np.zeros_like(q)
        dq[:, j] = eps
        fd = (_attached_point(hand, f, l, pl, q + dq) - _attached_point(hand, f, l, pl, q - dq)) / (2 * eps)
        assert np.allclose(Jm[:, :, j], fd, atol=1e-9), j
    # joints beyond the contact link do not move the point
    assert np.all(Jm[np.arange(hand.J)[None, None, :].repeat(G, 0).repeat(3, 1) > l[:, None, None]] == 0)


def test_dls_step_is_damped_least_squares():
    """dq of Eq. DLS = argmin |J dq - e|^2 + lam |dq|^2 = lstsq([J; sqrt(lam) I], [e; 0])."""
    hand = synth.hand_anthropomorphic(4)
    rng = np.random.default_rng(4)
    G = 32
    f = rng.integers(0, hand.F, G)
    m = rng.integers(0, hand.M, G)
    l = hand.surf_link[f, m].astype(np.int64)
    pl = hand.surf_p[f, m].astype(np.float64)
    nl = hand.surf_n[f, m].astype(np.float64)
    q = rng.uniform(hand.lo[f], hand.hi[f])
    p = _attached_point(hand, f, l, pl, q) + rng.normal(0, 3e-3, (G, 3))
    n = rng.normal(size=(G, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    lam = 1e-4
    qn, dq, Jm, e = K.dls_step(hand, f, l, pl, nl, p, n, q, 0.01, lam, return_parts=True)
    for g in range(G):
        A = np.vstack([Jm[g], math.sqrt(lam) * np.eye(hand.J)])
        b = np.concatenate([e[g], np.zeros(hand.J)])
        ref = np.linalg.lstsq(A, b, rcond=None)[0]
        assert np.allclose(dq[g], ref, atol=1e-10)
    assert np.allclose(qn, np.clip(q + dq, hand.lo[f], hand.hi[f]))
    # the step lowers the linearised objective below the zero step
    lin = np.linalg.norm(np.einsum("grj,gj->gr", Jm, dq) - e, axis=1) ** 2 + lam * np.sum(dq * dq, axis=1)
    assert np.all(lin <= np.linalg.norm(e, axis=1) ** 2 + 1e-15)


def test_dls_converges_to_reachable_targets():
    """Targets generated by FK at q*: DLS from a perturbed start drives both
    position and normal errors to ~0 (a sign error in e or J would diverge)."""
    hand = synth.hand_anthropomorphic(4)
    rng = np.random.default_rng(5)
    G = 64
    f = rng.integers(0, hand.F, G)
    m = rng.integers(0, hand.M, G)
    l = hand.surf_link[f, m].astype(np.int64)
    pl = hand.surf_p[f, m].astype(np.float64)
    nl = hand.surf_n[f, m].astype(np.float64)
    lo, hi = hand.lo[f].astype(np.float64), hand.hi[f].astype(np.float64)
    qs = lo + (0.2 + 0.6 * rng.random((G, hand.J))) * (hi - lo)
    R, t, _ = K.chain(hand, f, qs)
    g = np.arange(G)
    p = np.einsum("gij,gj->gi", R[g, l], pl) + t[g, l]
    n = np.einsum("gij,gj->gi", R[g, l], nl)
    q = np.clip(qs + rng.normal(0, 0.05, qs.shape), lo, hi)
    for _ in range(40):
        q = K.dls_step(hand, f, l, pl, nl, p, n, q, 0.01, 1e-4)
    R, t, _ = K.chain(hand, f, q)
    x = np.einsum("gij,gj->gi", R[g, l], pl) + t[g, l]
    nn = np.einsum("gij,gj->gi", R[g, l], nl)
    err = np.linalg.norm(x - p, axis=1)
    assert np.median(err) < 1e-7 and np.quantile(err, 0.9) < 1e-4
    assert np.median(np.sum(nn * n, axis=1)) > 1 - 1e-6


def _capsule_case(rng, G=48):
    hand = synth.hand_anthropomorphic(4)
    f = rng.integers(0, hand.F, G)
    l = rng.integers(1, hand.J, G)  # links 1..3 have length and radius
    q = rng.uniform(hand.lo[f], hand.hi[f])
    m = np.zeros(G, np.int64)
    pl = hand.surf_p[f, m].astype(np.float64)
    nl = hand.surf_n[f, m].astype(np.float64)
    R, t, _ = K.chain(hand, f, q)
    g = np.arange(G)
    a = t[g, l]
    b = a + np.einsum("gij,gj->gi", R[g, l], hand.offset[f, l].astype(np.float64))
    return hand, f, l, q, pl, nl, a, b


def test_project_capsule_optimal_over_capsule_normals():
    """The projected point lies on the capsule at the axis point nearest p, its
    normal is a capsule normal there, and no sampled capsule normal at that axis
    point gives a lower DLS objective."""
    rng = np.random.default_rng(6)
    hand, f, l, q, pl, nl, a, b = _capsule_case(rng)
    G = len(f)
    beta = 0.01
    mid = a + rng.uniform(-0.3, 1.3, (G, 1)) * (b - a)
    p = mid + rng.normal(0, 0.012, (G, 3))
    n = rng.normal(size=(G, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    _, _, xw, nw = K.project_capsule(hand, f, l, q, p, n, pl, nl, beta)
    r = hand.radius[f, l].astype(np.float64)
    dirs = rng.normal(size=(4000, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    for g in range(G):
        d = b[g] - a[g]
        s = np.clip((p[g] - a[g]) @ d / (d @ d), 0, 1)
        c = a[g] + s * d
        assert np.allclose(xw[g], c + r[g] * nw[g], atol=1e-14)
        assert abs(np.linalg.norm(nw[g]) - 1) < 1e-12
        u = d / np.linalg.norm(d)
        if 0 < s < 1:
            valid = dirs - np.outer(dirs @ u, u)
            valid /= np.linalg.norm(valid, axis=1, keepdims=True)
            assert abs(nw[g] @ u) < 1e-12
        else:
            sign = -1.0 if s == 0 else 1.0
            valid = dirs[(dirs @ u) * sign >= 0]
            assert (nw[g] @ u) * sign >= -1e-12
        obj = lambda x, v: np.sum((x - p[g]) ** 2, -1) + np.sum((x + beta * v - p[g] - beta * n[g]) ** 2, -1)
        best = obj(c[None] + r[g] * valid, valid).min()
        assert obj(xw[g], nw[g]) <= best + 1e-12


def test_project_capsule_reduces_to_nearest_point():
    """When n is the radial direction from the axis to p, the projection is the
    nearest capsule point to p (checked by dense sampling of the surface)."""
    rng = np.random.default_rng(7)
    hand, f, l, q, pl, nl, a, b = _capsule_case(rng, 24)
    G = len(f)
    p = a + rng.uniform(0.1, 0.9, (G, 1)) * (b - a) + rng.normal(0, 0.02, (G, 3))
    r = hand.radius[f, l].astype(np.float64)
    for g in range(G):
        d = b[g] - a[g]
        c = a[g] + np.clip((p[g] - a[g]) @ d / (d @ d), 0, 1) * d
        n = (p[g] - c) / np.linalg.norm(p[g] - c)
        _, _, xw, _ = K.project_capsule(hand, f[g:g + 1], l[g:g + 1], q[g:g + 1], p[g:g + 1], n[None],
                                        pl[g:g + 1], nl[g:g + 1], 0.01)
        # dense sample of the capsule surface
        s = np.linspace(0, 1, 801)
        axis_pts = a[g] + s[:, None] * d
        ax_d = np.min(np.linalg.norm(p[g] - axis_pts, axis=1))
        assert abs(np.linalg.norm(xw[0] - p[g]) - abs(ax_d - r[g])) < 1e-6


def _brute_seg(p0, p1, q0, q1, k=601):
    s = np.linspace(0, 1, k)
    P = p0[None] + s[:, None] * (p1 - p0)[None]
    Q = q0[None] + s[:, None] * (q1 - q0)[None]
    return np.min(np.linalg.norm(P[:, None, :] - Q[None, :, :], axis=2))


def test_segment_distance_cases_and_brute_force():
    z = np.zeros(3)
    ex, ey, ez = np.eye(3)
    assert K.segment_distance(z, ex, ez * 0.3, ez * 0.3 + ex) == pytest.approx(0.3, abs=1e-15)       # parallel
    assert K.segment_distance(-ex, ex, -ey, ey) == pytest.approx(0.0, abs=1e-15)                       # crossing
    assert K.segment_distance(-ex, ex, 0.2 * ez - ey, 0.2 * ez + ey) == pytest.approx(0.2, abs=1e-15)  # skew
    assert K.segment_distance(z, ex, 2 * ex, 3 * ex) == pytest.approx(1.0, abs=1e-15)                  # collinear
    rng = np.random.default_rng(8)
    for _ in range(60):
        p0, p1, q0, q1 = rng.normal(size=(4, 3))
        d = K.segment_distance(p0, p1, q0, q1)
        bf = _brute_seg(p0, p1, q0, q1)
        assert d <= bf + 1e-12
        assert bf - d < 2e-5 * (1 + np.linalg.norm(p1 - p0) + np.linalg.norm(q1 - q0))
        assert d == pytest.approx(K.segment_distance(q1, q0, p1, p0), abs=1e-14)  # symmetric


def test_sdf_grid_sphere_analytic():
    """Point-sampled sphere: the brute-force grid SDF is |x| - r up to the
    sampling gap, negative inside, positive outside."""
    r = 0.04
    soa = synth.sphere(2048, r, seed=3).soa()
    lo = np.array([-0.06, -0.06, -0.06], np.float32)
    h = 0.008
    dims = (16, 16, 16)
    grid, amb = K.sdf_grid(soa, lo, h, dims)
    iz, iy, ix = np.meshgrid(*(np.arange(d) for d in dims[::-1]), indexing="ij")
    x = np.stack([lo[0] + ix * float(np.float32(h)), lo[1] + iy * float(np.float32(h)),
                  lo[2] + iz * float(np.float32(h))], -1)
    exact = np.linalg.norm(x, axis=-1) - r
    # covering radius of the samples on the sphere: |sdf - exact| <= rho for
    # every node (nearest sample vs nearest surface point)
    dense = synth.fibonacci_dirs(20000).astype(np.float64) * r
    pts = soa[:3].T.astype(np.float64)
    rho = max(np.min(np.linalg.norm(dense[a:a + 2000, None] - pts[None], axis=2), axis=1).max()
              for a in range(0, 20000, 2000))
    assert rho < 8e-3
    assert np.max(np.abs(grid - exact)) <= rho + 1e-6
    far = np.abs(exact) > rho
    assert np.all(np.sign(grid[far]) == np.sign(exact[far]))
    assert not amb[far].any()
    # trilinear interpolation reproduces node values on the nodes
    pts = x.reshape(-1, 3)[:: 37]
    v, _ = K.sdf_trilinear(grid, amb, lo, h, pts + 1e-12)
    ins = np.isfinite(v)
    assert np.allclose(v[ins], grid.reshape(-1)[:: 37][ins], atol=1e-9)


def test_sdf_trilinear_linear_field_exact():
    lo = np.array([0.0, 0.0, 0.0], np.float32)
    h = 0.5
    dims = (5, 4, 3)
    iz, iy, ix = np.meshgrid(*(np.arange(d) for d in dims[::-1]), indexing="ij")
    grid = 0.3 * ix * h - 0.7 * iy * h + 1.1 * iz * h + 0.2
    amb = np.zeros_like(grid, bool)
    rng = np.random.default_rng(9)
    x = rng.uniform(0, [4 * h, 3 * h, 2 * h], (200, 3)) * 0.999
    v, _ = K.sdf_trilinear(grid, amb, lo, h, x)
    assert np.allclose(v, 0.3 * x[:, 0] - 0.7 * x[:, 1] + 1.1 * x[:, 2] + 0.2, atol=1e-12)
    v_out, _ = K.sdf_trilinear(grid, amb, lo, h, np.array([[-0.1, 0.2, 0.2], [0.2, 0.2, 5.0]]))
    assert np.all(np.isinf(v_out))


def test_random_joint_range():
    lo, hi = np.float32(-0.35), np.float32(1.6)
    vals = [K.random_joint(lo, hi, w) for w in (0, 255, 1 << 31, 0xFFFFFFFF)]
    assert vals[0] == lo and vals[1] == lo
    assert all(lo <= v <= hi for v in vals)
    assert vals[2] == pytest.approx(float(lo) + 0.5 * (float(hi) - float(lo)), abs=1e-6)
    rng = np.random.default_rng(10)
    u = [K.random_joint(lo, hi, int(w)) for w in rng.integers(0, 1 << 32, 4000, dtype=np.uint64)]
    assert abs(np.mean(u) - 0.5 * (float(lo) + float(hi))) < 0.03


def test_rep_codes_are_the_smallest_producer():
    """Reverse lookup table of a small field = the first (s, m) in s * M + m
    order that produces each code, by enumerating single-point fields."""
    hand = synth.hand_three_finger()
    S = 6
    q = synth.joint_samples(hand, S, seed=11)
    bins = synth.fibonacci_dirs(8)
    inv_h = np.float32(200.0)
    f = 1
    rep = oracle.rep_codes(hand, q, inv_h, bins, f)
    assert set(rep) == set(oracle.pack_code(f, *c) for c in oracle.Field(hand, q, inv_h, bins).codes(f).tolist())
    first = {}
    for s in range(S):
        for m in range(hand.M):
            single = synth.Hand(name="one", base=hand.base, axis=hand.axis, offset=hand.offset, lo=hand.lo,
                                hi=hand.hi, radius=hand.radius, surf_p=np.ascontiguousarray(hand.surf_p[:, m:m + 1]),
                                surf_n=np.ascontiguousarray(hand.surf_n[:, m:m + 1]),
                                surf_link=np.ascontiguousarray(hand.surf_link[:, m:m + 1]),
                                grasp_centre=hand.grasp_centre)
            code = oracle.Field(single, np.ascontiguousarray(q[:, :, s:s + 1]), inv_h, bins).codes(f)
            key = oracle.pack_code(f, *code[0].tolist())
            first.setdefault(key, s * hand.M + m)
    assert first == rep


def test_point_codes_agree_with_query_masks():
    w = synth.workload("tiny_sphere", P=6, S=512)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
    soa = w.obj.soa()
    masks, _ = fd.query(soa, w.poses)
    pi = np.repeat(np.arange(w.P), w.obj.N)
    xi = np.tile(np.arange(w.obj.N), w.P)
    codes = oracle.point_codes(soa, w.poses, pi, xi, w.inv_h, w.bins)
    for f in range(w.hand.F):
        keys = set(oracle.pack_code(f, *c) for c in fd.codes(f).tolist())
        hit = np.array([oracle.pack_code(f, *c) in keys for c in codes.tolist()])
        bits = (masks[pi, f, xi >> 5] >> (xi & 31)) & 1
        assert np.array_equal(hit, bits.astype(bool))


def test_ik_dls_outputs_consistent():
    w = synth.workload("hand16_superquadric", P=4, S=4096)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
    soa = w.obj.soa()
    m, c = fd.query(soa, w.poses)
    tup, fing = oracle.sample_tuples(m, c, w.obj.N, w.T, w.k, w.seed)
    acc = (tup.reshape(-1, w.k)[:, 0] >= 0).astype(np.uint8)
    out = K.ik_dls(w.hand, w.q, w.inv_h, w.bins, soa, w.poses, w.T, w.k, tup, fing, acc)
    n = acc.size
    assert not out["miss"].any()  # every domain point has a representative
    ok = out["ok"].astype(bool)
    assert ok.any() and not ok.all()
    r = out["resid"]
    okc = (r[..., 0] <= 2e-3) & (r[..., 1] >= np.float32(math.cos(math.radians(20))))
    assert np.array_equal(ok, okc.all(axis=1) & acc.astype(bool))
    tf = fing.reshape(n, w.k)
    for u in np.nonzero(acc)[0][:50]:
        for cc in range(w.k):
            fq = out["q"][u, tf[u, cc]]
            assert np.all(fq >= w.hand.lo[tf[u, cc]] - 1e-12) and np.all(fq <= w.hand.hi[tf[u, cc]] + 1e-12)
            assert out["used"][u, tf[u, cc], 0] == 1
        unused = np.setdiff1d(np.arange(w.hand.F), tf[u])
        assert np.all(out["q"][u, unused] == 0) and np.all(out["used"][u, unused] == 0)
        if ok[u]:
            assert list(out["rtuples"][u]) == [u * w.k + cc for cc in range(w.k)]
            # realised contacts sit within tol_pos of the object points (object frame)
            pts = soa[:3, tup.reshape(n, w.k)[u]].T.astype(np.float64)
            rc = out["contacts"][:3, u * w.k:(u + 1) * w.k].T
            assert np.all(np.linalg.norm(rc - pts, axis=1) <= 2e-3 + 1e-9)
            nc = out["contacts"][3:, u * w.k:(u + 1) * w.k].T
            assert np.allclose(np.linalg.norm(nc, axis=1), 1.0)
        else:
            assert np.all(out["rtuples"][u] == -1)


def _two_finger_cross():
    base = np.array([[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0],
                     [0, -1, 0, 0.02, 1, 0, 0, -0.02, 0, 0, 1, 0]], np.float64)  # finger 1 rotated 90 deg about z
    axis = np.array([[[0, 0, 1]], [[0, 0, 1]]], np.float64)
    offset = np.array([[[0.04, 0, 0]], [[0.04, 0, 0]]], np.float64)
    return _hand("cross", base, axis, offset, [[-2.0], [-2.0]], [[2.0], [2.0]], [[0.005], [0.005]])


def test_realize_self_collision_and_penetration():
    hand = _two_finger_cross()
    soa = synth.sphere(1024, 0.01, seed=4).soa()  # small ball
    lo, h, dims = np.array([-0.03, -0.03, -0.03], np.float32), 0.004, (16, 16, 16)
    grid, amb = K.sdf_grid(soa, lo, h, dims)
    n = 3
    q = np.zeros((n, 2, 1), np.float32)
    q[1, 1, 0] = -1.5708  # finger 1 swung parallel to finger 0, 20 mm away: no contact
    q[2, :, 0] = [0.0, -1.5708]
    used = np.ones((n, 2, 1), np.uint8)
    ident = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    far = ident.copy()
    far[[3, 7, 11]] = [0.5, 0.5, 0.5]        # object far from the hand
    near = ident.copy()
    near[[3, 7, 11]] = [0.03, 0.0, 0.0]      # ball centred on finger 0's axis
    poses = np.stack([far, far, near])
    qo, flags, ambig = K.realize(hand, grid, amb, lo, h, poses, 1, q, used, None, None, pen_margin=2e-3,
                                 axis_step=1e-3, seed=5)
    assert list(flags) == [4, 0, 2] and not ambig.any()
    assert np.array_equal(qo, q)  # every joint was fixed by IK
    # a gated slot is left alone
    _, flags2, _ = K.realize(hand, grid, amb, lo, h, poses, 1, q, used, np.array([1, 0, 1], np.uint8), None)
    assert flags2[1] == 1


def test_realize_fills_free_joints_only():
    hand = synth.hand_anthropomorphic(4)
    n = 5
    rng = np.random.default_rng(12)
    q = rng.uniform(hand.lo, hand.hi, (n, hand.F, hand.J)).astype(np.float32)
    used = (rng.random((n, hand.F, hand.J)) < 0.5).astype(np.uint8)
    grid = np.full((4, 4, 4), 1.0)
    amb = np.zeros_like(grid, bool)
    poses = np.tile(np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 5.0], np.float32), (n, 1))
    qo, flags, _ = K.realize(hand, grid, amb, np.zeros(3, np.float32), 0.01, poses, 1, q, used, None, None, seed=7)
    assert np.array_equal(qo[used == 1], q[used == 1])
    free = used == 0
    assert np.all(qo[free] != q[free])
    lo = np.broadcast_to(hand.lo, q.shape)[free]
    hi = np.broadcast_to(hand.hi, q.shape)[free]
    assert np.all((qo[free] >= lo) & (qo[free] <= hi))


def test_realize_slot_ids_key_the_draws():
    """Slots taken out of a launch keep their free joints when their slot indices come with them."""
    hand = synth.hand_anthropomorphic(4)
    n, T = 6, 3
    rng = np.random.default_rng(13)
    q = rng.uniform(hand.lo, hand.hi, (n, hand.F, hand.J)).astype(np.float32)
    used = (rng.random((n, hand.F, hand.J)) < 0.5).astype(np.uint8)
    grid = np.full((4, 4, 4), 1.0)
    amb = np.zeros_like(grid, bool)
    poses = np.tile(np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 5.0], np.float32), (n // T, 1))
    args = (hand, grid, amb, np.zeros(3, np.float32), 0.01)
    qa, fa, _ = K.realize(*args, poses, T, q, used, None, None, seed=7)
    sl = np.arange(T, 2 * T)  # the second pose's slots
    qs, fs, _ = K.realize(*args, poses[1:], T, q[sl], used[sl], None, None, seed=7, slot_ids=sl)
    assert np.array_equal(qs, qa[sl]) and np.array_equal(fs, fa[sl])
    qd, _, _ = K.realize(*args, poses[1:], T, q[sl], used[sl], None, None, seed=7)  # keyed as slots 0 .. T-1
    assert not np.array_equal(qd, qa[sl])
    with pytest.raises(ValueError):
        K.realize(*args, poses[1:], T, q[sl], used[sl], None, None, seed=7, slot_ids=sl[:1])
