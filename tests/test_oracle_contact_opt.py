"""Pins of the Alg. 2 oracle (Sec. 5.4 blockwise zeroth-order contact
optimisation): the mutation draws are standard normal, projections land on the
nearest domain point, the margin never increases and is the closure margin of
the final tuple, and the degenerate settings (no iteration, no mutation) leave
tuples unchanged."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import synth
from oracle import contact_opt as CO


def test_mutation_draws_are_standard_normal():
    g = np.array([CO.mutation_normals(p, t, 0, 0, 3, 16, 5) for p in range(20) for t in range(20)]).reshape(-1, 2)
    for col in (g[:, 0], g[:, 1]):
        assert stats.kstest(col, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(g[:, 0], g[:, 1])[0, 1]) < 0.05
    # distinct blocks, candidates and seeds draw distinct values
    a = CO.mutation_normals(1, 2, 0, 0, 3, 8, 5)
    b = CO.mutation_normals(1, 2, 0, 1, 3, 8, 5)
    c = CO.mutation_normals(1, 2, 0, 0, 3, 8, 6)
    assert len(set(a)) == 8 and set(a).isdisjoint(b) and set(a).isdisjoint(c)


def test_box_muller_extremes():
    # u1 = 1 (top word) gives radius 0; the smallest u1 gives the largest radius
    assert CO.box_muller(0xFFFFFFFF, 0) == (0.0, 0.0)
    g1, g2 = CO.box_muller(0, 0)
    assert g1 == pytest.approx(math.sqrt(-2 * math.log(2.0 ** -24))) and g2 == 0.0


def test_projection_is_nearest_domain_point():
    rng = np.random.default_rng(1)
    pts = rng.normal(size=(500, 3))
    dom = np.sort(rng.choice(500, 120, replace=False))
    for _ in range(50):
        q = rng.normal(size=3)
        x, amb = CO.project_to_domain(pts, dom, q)
        assert x in dom
        d = np.linalg.norm(pts[dom] - q, axis=1)  # brute force over the domain
        assert x == dom[int(np.argmin(d))]
        assert amb == (np.sort(d)[1] - d.min() <= CO.PROJ_GAP)
    # exact copies of the nearest point: the lowest index, and no ambiguity
    # (a copy ties in every precision)
    pts2 = np.vstack([pts, pts[dom[5]][None]])
    dom2 = np.append(dom, 500)
    assert CO.project_to_domain(pts2, dom2, pts[dom[5]]) == (dom[5], False)
    # a distinct point at the same distance is ambiguous
    q = pts[dom[5]] + np.array([0.0, 0.0, 1e-3])
    pts4 = np.vstack([pts, q + np.array([0.0, 0.0, 1e-3])])
    assert CO.project_to_domain(pts4, dom2, q) == (dom[5], True)
    # a point 2e-7 m nearer than the next one is clear of the band
    q = pts[dom[7]] + np.array([1e-3, 0.0, 0.0])
    pts3 = np.vstack([pts, q + np.array([-1e-3 - 2e-7, 0.0, 0.0])])
    pts3[dom[7]] = q + np.array([-1e-3, 0.0, 0.0])
    assert CO.project_to_domain(pts3, np.append(dom, 500), q)[1] is False


def test_tangent_basis_is_orthonormal():
    rng = np.random.default_rng(2)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        x, y = CO.tangent_basis(n)
        x, y = np.array(x), np.array(y)
        assert abs(x @ y) < 1e-12 and abs(x @ n) < 1e-12 and abs(y @ n) < 1e-12
        assert abs(np.linalg.norm(x) - 1) < 1e-12 and abs(np.linalg.norm(y) - 1) < 1e-12
        # right-handed: x cross y = nu = -n
        assert np.allclose(np.cross(x, y), -n, atol=1e-12)


@pytest.fixture(scope="module")
def hand16_small():
    w = synth.workload("hand16_superquadric", P=2, S=4096)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
    soa = w.obj.soa()
    m, c = fd.query(soa, w.poses)
    tup, fing = oracle.sample_tuples(m, c, w.obj.N, w.T, w.k, w.seed)
    m0, a0, _ = oracle.score_tuples(soa, tup, w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps)
    return w, soa, m, tup, fing, m0, a0


def test_optimisation_monotone_and_consistent(hand16_small):
    w, soa, m, tup, fing, m0, a0 = hand16_small
    ot, om, oa, amb = CO.optimize_tuples(soa, m, tup, fing, w.T, w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps, w.seed)
    fin = np.isfinite(m0)
    assert np.all(om[fin] <= m0[fin] * (1 + 1e-9) + 1e-12)       # never worse
    assert np.array_equal(np.isfinite(om), fin)                    # invalid tuples stay invalid
    assert oa.sum() > a0.sum()                                     # it does improve on this workload
    # the reported margin is the closure margin of the final tuple
    m_re, _, _ = oracle.score_tuples(soa, ot, w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps)
    assert np.allclose(m_re[fin], om[fin], rtol=1e-9, atol=1e-12)
    # every contact stays in its finger's domain
    P, T, k = ot.shape
    for i in range(P):
        for t in range(T):
            if not fin[i, t]:
                continue
            for d in range(k):
                x, f = ot[i, t, d], fing[i, t, d]
                assert (m[i, f, x >> 5] >> (x & 31)) & 1
    assert amb.mean() < 0.05


def test_degenerate_settings_leave_tuples(hand16_small):
    w, soa, m, tup, fing, m0, a0 = hand16_small
    args = (soa, m, tup, fing, w.T, w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps, w.seed)
    t0, mm0, _, _ = CO.optimize_tuples(*args, n_outer=0)
    assert np.array_equal(t0, tup)
    fin = np.isfinite(m0)
    assert np.allclose(mm0[fin], m0[fin], rtol=1e-12, atol=0)
    ts, _, _, _ = CO.optimize_tuples(*args, sigma=0.0)  # every mutation projects back onto p_i (or a copy)
    assert np.array_equal(ts, tup)


def test_pose_ids_key_the_draws(hand16_small):
    """Rows taken out of a request keep their results when their pose indices come with them (the
    draws are keyed by the pose's index in its request), and differ when they do not."""
    w, soa, m, tup, fing, m0, a0 = hand16_small
    args = (w.T, w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps, w.seed)
    ot, om, _, _ = CO.optimize_tuples(soa, m, tup, fing, *args)
    rows = np.array([1, 0])
    st, sm, _, _ = CO.optimize_tuples(soa, m[rows], tup[rows], fing[rows], *args, pose_ids=rows)
    assert np.array_equal(st, ot[rows])
    assert np.array_equal(sm, om[rows])
    dt, _, _, _ = CO.optimize_tuples(soa, m[rows], tup[rows], fing[rows], *args)  # keyed as poses 0 and 1 instead
    assert not np.array_equal(dt, ot[rows])
    with pytest.raises(ValueError):
        CO.optimize_tuples(soa, m[rows], tup[rows], fing[rows], *args, pose_ids=[0])
