"""Pins for the oracle's closure margin (Eq. GSWO, Sec. 2.2, linearised:
K-edge inscribed friction pyramid, torque-weighted max-norm, one LP per
j with alpha_j = 1, margin = min over j)."""
import math

import numpy as np
import pytest
from scipy.optimize import linprog

import oracle


def _onb(n):
    # Duff et al. 2017 branchless basis, restated for the check's wrench build
    s = math.copysign(1.0, n[2])
    a = -1.0 / (s + n[2])
    b = n[0] * n[1] * a
    return (np.array([1 + s * n[0] * n[0] * a, s * b, -s * n[0]]),
            np.array([b, s + n[1] * n[1] * a, -n[1]]))


def _highs_margin(p, n, mu, K, c, rho):
    """Same LPs solved by scipy's HiGHS (an independent LP library)."""
    k = len(p)
    W = []
    for i in range(k):
        nu = -np.asarray(n[i], float)
        x, y = _onb(nu)
        r = np.asarray(p[i], float) - c
        for m in range(K):
            th = 2 * math.pi * m / K
            e = nu + mu * (math.cos(th) * x + math.sin(th) * y)
            W.append(np.concatenate([e, np.cross(r, e) / rho]))
    W = np.array(W).T  # 6 x kK
    out = []
    nv = k * K + 1
    for j in range(k):
        cost = np.zeros(nv)
        cost[-1] = 1.0
        A = np.zeros((12, nv))
        A[:6, :-1] = W
        A[6:, :-1] = -W
        A[:, -1] = -1.0
        Aeq = np.zeros((1, nv))
        Aeq[0, j * K:(j + 1) * K] = 1.0
        res = linprog(cost, A_ub=A, b_ub=np.zeros(12), A_eq=Aeq, b_eq=[1.0],
                      bounds=[(0, None)] * nv, method="highs")
        assert res.status == 0
        out.append(res.fun)
    return np.array(out)


def _rand_contacts(rng, k):
    p = rng.normal(size=(k, 3)) * 0.05
    n = rng.normal(size=(k, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    return p, n


@pytest.mark.parametrize("k,K,mu", [(2, 4, 0.5), (3, 8, 0.5), (3, 8, 0.4), (4, 6, 0.8), (3, 8, 0.0)])
def test_lp_matches_highs(k, K, mu):
    rng = np.random.default_rng(100 + k * 10 + K)
    for _ in range(40):
        p, n = _rand_contacts(rng, k)
        c = p.mean(axis=0) + rng.normal(size=3) * 0.01
        rho = float(np.max(np.linalg.norm(p - c, axis=1)))
        t, tj, piv = oracle.closure_lp(p, n, mu, K, c, rho)
        ref = _highs_margin(p, n, mu, K, c, rho)
        assert np.allclose(tj, ref, atol=1e-9, rtol=1e-8)
        assert abs(t - ref.min()) <= 1e-9
        assert (piv > 0).all()


def test_antipodal_pair_on_a_sphere_balances_exactly():
    r = 0.04
    u = np.array([0.3, -0.5, 0.8])
    u /= np.linalg.norm(u)
    p = np.array([r * u, -r * u])
    n = np.array([u, -u])
    t, tj, _ = oracle.closure_lp(p, n, 0.5, 8, np.zeros(3), r)
    assert t == 0.0 or abs(t) < 1e-15


def test_single_contact_axis_aligned_normal_gives_margin_one():
    """One contact, alpha = 1: the normal component of the force is exactly 1
    along an axis, so the max-norm is at least 1; the symmetric edge mix reaches
    it (tangential part 0, torque components <= |p - c| / rho <= 1)."""
    for nrm in ([0, 0, 1], [0, -1, 0], [1, 0, 0]):
        p = np.array([[0.01, 0.02, -0.03]])
        t, _, _ = oracle.closure_lp(p, np.array([nrm], float), 0.5, 8, np.zeros(3), 0.05)
        assert abs(t - 1.0) < 1e-12


def _two_contact(phi, azim, mu, K):
    """Contact 1 at the origin with inward force direction +z; contact 2 on the
    segment direction making angle phi with +z at azimuth azim (measured in
    contact 1's Duff tangent basis), with inward direction pointing back."""
    nu1 = np.array([0.0, 0.0, 1.0])
    x, y = _onb(nu1)
    d = math.cos(phi) * nu1 + math.sin(phi) * (math.cos(azim) * x + math.sin(azim) * y)
    p = np.array([[0.0, 0.0, 0.0], 0.1 * d])
    n = np.array([-nu1, d])  # outward normals: nu = -n
    c = p.mean(axis=0)
    rho = 0.05
    return oracle.closure_lp(p, n, mu, K, c, rho)[0]


@pytest.mark.parametrize("K", [8, 6])
def test_two_contact_closure_iff_segment_inside_pyramid(K):
    """Nguyen-style criterion for two contacts: a zero wrench exists iff the
    segment between the contacts lies in both friction pyramids.  Contact 2's
    pyramid is aligned with the segment; contact 1's pyramid half-angle is
    atan(mu) toward an edge and atan(mu cos(pi/K)) toward a face midline."""
    mu = 0.5
    edge = math.atan(mu)
    face = math.atan(mu * math.cos(math.pi / K))
    d = 2e-3
    assert _two_contact(edge - d, 0.0, mu, K) < 1e-12
    assert _two_contact(edge + d, 0.0, mu, K) > 1e-4
    assert _two_contact(face - d, math.pi / K, mu, K) < 1e-12
    assert _two_contact(face + d, math.pi / K, mu, K) > 1e-4


def test_invariances_translation_permutation_and_friction_monotonicity():
    rng = np.random.default_rng(9)
    for _ in range(25):
        p, n = _rand_contacts(rng, 3)
        c = p.mean(axis=0)
        rho = float(np.max(np.linalg.norm(p - c, axis=1)))
        t0 = oracle.closure_lp(p, n, 0.5, 8, c, rho)[0]
        s = np.array([0.125, -0.25, 0.0625])  # exact shift
        t1 = oracle.closure_lp(p + s, n, 0.5, 8, c + s, rho)[0]
        assert abs(t0 - t1) < 1e-10
        perm = rng.permutation(3)
        t2 = oracle.closure_lp(p[perm], n[perm], 0.5, 8, c, rho)[0]
        assert abs(t0 - t2) < 1e-10
        # larger friction pyramid -> no larger margin; mu = 0 is the frictionless form
        tf = oracle.closure_lp(p, n, 0.0, 8, c, rho)[0]
        tm = oracle.closure_lp(p, n, 0.8, 8, c, rho)[0]
        assert tm <= t0 + 1e-12 <= tf + 2e-12


def test_score_tuples_marks_invalid_and_thresholds():
    rng = np.random.default_rng(1)
    N = 64
    pts = rng.normal(size=(N, 3)) * 0.04
    nrm = pts / np.linalg.norm(pts, axis=1, keepdims=True)
    soa = np.concatenate([pts.T, nrm.T]).astype(np.float32)
    tuples = rng.integers(0, N, size=(5, 4, 3)).astype(np.int32)
    tuples[1, 2] = -1
    c = pts.mean(0).astype(np.float32)
    m, a, piv = oracle.score_tuples(soa, tuples, 0.5, 8, c, 0.05, 0.01)
    assert np.isinf(m[1, 2]) and a[1, 2] == 0 and piv[1, 2] == 0
    fin = np.isfinite(m)
    assert np.array_equal(a[fin].astype(bool), m[fin] <= np.float32(0.01))


def test_lp_matches_highs_on_tool_faces_with_axis_aligned_normals():
    """Box faces of the tool object give normals with exact zero components;
    their wrench columns are partly collinear, a degenerate case for the
    simplex (rounding noise on structural zeros must never become a pivot)."""
    import synth
    obj = synth.tool_composite(4096, 1000)
    rng = np.random.default_rng(21)
    axis = np.sum(obj.n == 0.0, axis=1) >= 1
    pool = np.nonzero(axis)[0]
    c = obj.centroid.astype(np.float64)
    for _ in range(120):
        ids = rng.choice(pool, 3, replace=False)
        p, n = obj.p[ids].astype(np.float64), obj.n[ids].astype(np.float64)
        t, tj, piv = oracle.closure_lp(p, n, float(np.float32(0.4)), 8, c, float(obj.rho))
        ref = _highs_margin(p, n, float(np.float32(0.4)), 8, c, float(obj.rho))
        assert np.all(np.isfinite(tj))
        assert np.allclose(tj, ref, atol=1e-9, rtol=1e-8)


def test_oracle_workload_margins_are_never_nan():
    import synth
    w = synth.workload("hand20_tool", P=6, S=2048)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
    soa = w.obj.soa()
    m, cnt = fd.query(soa, w.poses)
    tup, _ = oracle.sample_tuples(m, cnt, w.obj.N, w.T, w.k, w.seed)
    mar, _, piv = oracle.score_tuples(soa, tup, w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps)
    assert not np.isnan(mar).any()
    assert (piv >= 0).all()
