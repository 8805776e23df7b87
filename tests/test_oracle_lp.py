"""Pins for the oracle's closure margin (Eq. GSWO, Sec. 3.2, linearised:
K-edge inscribed friction pyramid, torque-weighted max-norm, one LP per
j with alpha_j = 1, margin = min over j).  The LP solver is a library routine;
these tests pin the LP it is given: brute-force vertex enumeration, the
wrench columns against their definition, closed forms and invariances."""
import math

import numpy as np
import pytest

import oracle


def _onb(n):
    # Duff et al. 2017 branchless basis (used by the two-contact construction below)
    s = math.copysign(1.0, n[2])
    a = -1.0 / (s + n[2])
    b = n[0] * n[1] * a
    return (np.array([1 + s * n[0] * n[0] * a, s * b, -s * n[0]]),
            np.array([b, s + n[1] * n[1] * a, -n[1]]))


def _vertex_enumeration(W, K, j):
    """LP_j by brute force: every vertex of {(c, t): -t <= W c <= t, c >= 0,
    t >= 0, sum_m c_jm = 1} is the solution of the equality plus nv - 1 active
    inequalities; the optimum of min t is the smallest t over feasible vertices."""
    import itertools
    nc = W.shape[1]
    nv = nc + 1
    G = np.zeros((12 + nv, nv))          # G z <= 0
    G[:6, :nc] = W
    G[6:12, :nc] = -W
    G[:12, nc] = -1.0
    G[12:, :] = -np.eye(nv)
    a = np.zeros(nv)
    a[j * K:(j + 1) * K] = 1.0
    combos = np.array(list(itertools.combinations(range(G.shape[0]), nv - 1)))
    M = np.concatenate([np.broadcast_to(a, (len(combos), 1, nv)), G[combos]], axis=1)
    rhs = np.zeros((len(combos), nv))
    rhs[:, 0] = 1.0
    ok = np.abs(np.linalg.det(M)) > 1e-12
    z = np.linalg.solve(M[ok], rhs[ok][..., None])[..., 0]
    feas = np.all(z @ G.T <= 1e-9, axis=1)
    return float(z[feas, nc].min())


def _rand_contacts(rng, k, axis_aligned=False):
    p = rng.normal(size=(k, 3)) * 0.05
    if axis_aligned:
        n = np.zeros((k, 3))
        for i in range(k):
            n[i, rng.integers(3)] = rng.choice([-1.0, 1.0])
            if rng.random() < 0.5:  # a face normal with one exact zero component
                n[i] = n[i] + np.roll(n[i], 1) * rng.uniform(0.2, 1.0)
        n /= np.linalg.norm(n, axis=1, keepdims=True)
    else:
        n = rng.normal(size=(k, 3))
        n /= np.linalg.norm(n, axis=1, keepdims=True)
    return p, n


@pytest.mark.parametrize("k,K,mu,aligned,reps", [(2, 3, 0.5, False, 8), (2, 4, 0.5, False, 2),
                                                 (2, 4, 0.3, True, 2), (1, 4, 0.5, False, 6), (3, 3, 0.4, True, 1),
                                                 (2, 3, 0.0, False, 4), (2, 3, 0.8, True, 6)])
def test_lp_matches_vertex_enumeration(k, K, mu, aligned, reps):
    rng = np.random.default_rng(100 + 10 * k + K + int(aligned))
    for _ in range(reps):
        p, n = _rand_contacts(rng, k, aligned)
        c = p.mean(axis=0) + rng.normal(size=3) * 0.01
        rho = float(np.max(np.linalg.norm(p - c, axis=1)))
        t, tj, it = oracle.closure_lp(p, n, mu, K, c, rho)
        W = oracle.wrench_matrix(p, n, mu, K, c, rho)
        ref = np.array([_vertex_enumeration(W, K, j) for j in range(k)])
        assert np.allclose(tj, ref, atol=1e-8, rtol=1e-7), (tj, ref)
        assert abs(t - ref.min()) <= 1e-8


def test_wrench_columns_match_their_definition():
    """Edge m of contact i: normal component 1 along nu = -n, tangential part
    of length mu at angle 2 pi m / K in the (x, y) basis; torque = r x e / rho."""
    rng = np.random.default_rng(3)
    p, n = _rand_contacts(rng, 2)
    c = np.array([0.01, -0.02, 0.0])
    W = oracle.wrench_matrix(p, n, 0.5, 8, c, 0.1)
    for i in range(2):
        nu = -n[i]
        x, y = _onb(nu)
        assert abs(x @ nu) < 1e-12 and abs(y @ nu) < 1e-12 and abs(x @ y) < 1e-12
        assert np.allclose(np.cross(x, y), nu, atol=1e-12)  # right-handed
        for m in range(8):
            e = W[:3, 8 * i + m]
            assert abs(e @ nu - 1.0) < 1e-12
            tang = e - nu
            assert abs(np.linalg.norm(tang) - 0.5) < 1e-12
            ang = math.atan2(tang @ y, tang @ x) % (2 * math.pi)
            assert abs(ang - 2 * math.pi * m / 8) < 1e-9 or abs(ang - 2 * math.pi * m / 8 - 2 * math.pi) < 1e-9
            assert np.allclose(W[3:, 8 * i + m], np.cross(p[i] - c, e) / 0.1, atol=1e-12)


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


def test_scaled_box_form_gives_the_same_margin():
    """The GPU solves LP_j in a scaled form: with c = t c', LP_j = 1 / s_j where
    s_j = max sum_m c'_jm s.t. -1 <= (W c')_r <= 1, c' >= 0, and s_j unbounded
    exactly when LP_j = 0.  Solved here with the library LP solver on random
    tuples (both closing and non-closing), the reciprocal matches LP_j as
    defined."""
    from scipy.optimize import linprog
    rng = np.random.default_rng(21)
    n_zero = n_pos = 0
    for rep in range(60):
        k = 3 if rep % 3 else 2
        K = 8
        p = rng.normal(size=(k, 3)) * 0.03
        n = -p / np.linalg.norm(p, axis=1, keepdims=True) + 0.6 * rng.normal(size=(k, 3))
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        W = oracle.wrench_matrix(p, n, 0.5, K, np.zeros(3), 0.05)
        for j in range(k):
            t, _ = oracle.lp_subproblem(W, K, j)
            cost = np.zeros(W.shape[1])
            cost[j * K:(j + 1) * K] = -1.0  # maximise sum_m c'_jm
            res = linprog(cost, A_ub=np.vstack([W, -W]), b_ub=np.ones(12), bounds=[(0, None)] * W.shape[1],
                          method="highs")
            if res.status == 3:  # unbounded
                assert t <= 1e-9
                n_zero += 1
            else:
                assert res.status == 0
                s = -res.fun
                assert s > 0 and abs(1.0 / s - t) <= 1e-9 * max(1.0, t)
                n_pos += 1
    assert n_zero > 0 and n_pos > 0
