"""Pins of the Eq. GSWO oracle (true friction cones, squared L2, lambda = 1/rho^2;
Sec. 3.2): the cone projection against the Moreau decomposition, closed forms,
the two-contact friction criterion, and the sandwich between the LP margins of
the inscribed and circumscribed K-edge pyramids (HiGHS), which holds for the
exact optimum: t_circ^2 <= J <= 6 t_insc^2."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import gswo as G


def test_cone_projection_moreau():
    rng = np.random.default_rng(1)
    for mu in (0.0, 0.3, 1.0, 2.5):
        for t in range(200):
            a = rng.normal()
            b = rng.normal(size=2) if t % 4 else np.zeros(2)  # b = 0: the frictionless ray's edge case
            pa, pb = G.project_cone(a, b, mu)
            ra, rb = a - pa, b - pb
            assert pa >= 0.0 and np.linalg.norm(pb) <= mu * pa + 1e-12  # in the cone
            assert mu * np.linalg.norm(rb) <= -ra + 1e-12           # residual in the polar cone
            assert abs(pa * ra + pb @ rb) < 1e-12                   # orthogonal parts


def _sphere_pair(angle):
    """Contacts at +-x on a unit-radius sphere; contact 1's normal tilted by `angle`."""
    p = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    n = np.array([[1.0, 0, 0], [-math.cos(angle), math.sin(angle), 0]])
    return p, n


def test_closed_forms():
    p, n = _sphere_pair(0.0)
    J, _ = G.gswo(p, n, 0.5, np.zeros(3), 1.0, n_iter=3000)
    assert J < 1e-12  # antipodal: forces cancel, no torque
    J1, _ = G.gswo(p[:1], n[:1], 0.5, np.zeros(3), 1.0, n_iter=2000)
    assert J1 == pytest.approx(1.0, abs=1e-9)  # one contact through the centroid: |nu|^2


@pytest.mark.parametrize("mu", [0.3, 0.6])
def test_two_contact_friction_criterion(mu):
    """Two contacts close (J = 0) iff the segment between them lies inside both
    friction cones: tilt below atan(mu) -> 0, above -> bounded away from 0."""
    half = math.atan(mu)
    J_in, _ = G.gswo(*_sphere_pair(0.8 * half), mu, np.zeros(3), 1.0, n_iter=6000)
    J_out, _ = G.gswo(*_sphere_pair(1.3 * half), mu, np.zeros(3), 1.0, n_iter=6000)
    assert J_in < 1e-8
    assert J_out > 1e-4


def test_sandwich_between_pyramid_lps():
    w = synth.workload("hand16_superquadric", P=1, S=256)
    soa = w.obj.soa().astype(np.float64)
    rng = np.random.default_rng(3)
    K = w.K
    mu_c = w.mu / math.cos(math.pi / K)
    for _ in range(12):
        ids = rng.choice(w.obj.N, w.k, replace=False)
        p, n = soa[0:3, ids].T, soa[3:6, ids].T
        J, _ = G.gswo(p, n, w.mu, w.obj.centroid, w.obj.rho, n_iter=20000)
        t_in, _, _ = oracle.closure_lp(p, n, w.mu, K, w.obj.centroid, w.obj.rho)
        t_ci, _, _ = oracle.closure_lp(p, n, mu_c, K, w.obj.centroid, w.obj.rho)
        assert t_ci ** 2 - 1e-9 <= J <= 6 * t_in ** 2 + 1e-9, (J, t_ci, t_in)


def test_fixed_point_and_monotone_in_mu():
    w = synth.workload("tiny_sphere", P=1, S=64)
    soa = w.obj.soa().astype(np.float64)
    rng = np.random.default_rng(4)
    for _ in range(6):
        ids = rng.choice(w.obj.N, 3, replace=False)
        p, n = soa[0:3, ids].T, soa[3:6, ids].T
        A = G.gswo_matrix(p, n, w.obj.centroid, w.obj.rho)
        Jj, z = G.gswo_subproblem(A, 0, 0.5, 20000)
        Q = A.T @ A
        step = 1.0 / (2.0 * np.trace(Q))
        z2 = G._project(z - step * 2.0 * (Q @ z), 0, 0.5)
        assert np.linalg.norm(z2 - z) < 1e-7  # converged to a fixed point of the projected step
        Ja, _ = G.gswo(p, n, 0.3, w.obj.centroid, w.obj.rho, n_iter=8000)
        Jb, _ = G.gswo(p, n, 0.8, w.obj.centroid, w.obj.rho, n_iter=8000)
        assert Jb <= Ja + 1e-9  # wider cones cannot do worse


def _fswo_nnls(p, n, c, rho):
    """Eq. FSWO from its definition with a library solver: for each j, fix alpha_j = 1
    and minimise |a_j + sum_{i != j} alpha_i a_i|^2 over alpha >= 0 (scipy's NNLS,
    Lawson-Hanson), a_i = [nu_i ; r_i x nu_i / rho]."""
    from scipy.optimize import nnls
    p = np.asarray(p, np.float64)
    n = np.asarray(n, np.float64)
    k = p.shape[0]
    cols = [np.concatenate([-n[i], np.cross(p[i] - c, -n[i]) / rho]) for i in range(k)]
    vals = []
    for j in range(k):
        others = [cols[i] for i in range(k) if i != j]
        if others:
            _, res = nnls(np.stack(others, 1), -cols[j])
            vals.append(res * res)
        else:
            vals.append(float(cols[j] @ cols[j]))
    return min(vals)


def test_fswo_closed_forms():
    """Eq. FSWO (mu = 0): an antipodal pair closes; two contacts pushing the same way cannot
    (alpha >= 0 forbids cancelling), J = |nu|^2 = 1 with no torque; any tilt leaves J > 0."""
    c = np.zeros(3)
    p, n = _sphere_pair(0.0)
    assert G.gswo(p, n, 0.0, c, 1.0, n_iter=3000)[0] < 1e-12
    same_p = np.array([[1.0, 0, 0], [2.0, 0, 0]])
    same_n = np.array([[1.0, 0, 0], [1.0, 0, 0]])
    assert G.gswo(same_p, same_n, 0.0, c, 1.0, n_iter=3000)[0] == pytest.approx(1.0, abs=1e-12)
    J_t, _ = G.gswo(*_sphere_pair(0.05), 0.0, c, 1.0, n_iter=6000)
    assert J_t > 1e-4


def test_fswo_against_nnls_and_gswo_bound():
    """mu = 0 against NNLS written from Eq. FSWO's definition, and the paper's remark that the
    optimum of GSWO is a lower bound of FSWO (mu = 0.3, 0.6)."""
    w = synth.workload("hand16_superquadric", P=1, S=256)
    soa = w.obj.soa().astype(np.float64)
    rng = np.random.default_rng(7)
    for _ in range(16):
        ids = rng.choice(w.obj.N, w.k, replace=False)
        p, n = soa[0:3, ids].T, soa[3:6, ids].T
        J0, _ = G.gswo(p, n, 0.0, w.obj.centroid, w.obj.rho, n_iter=20000)
        ref = _fswo_nnls(p, n, w.obj.centroid, w.obj.rho)
        assert abs(J0 - ref) <= 1e-6 * max(ref, 1e-3), (J0, ref)
        for mu in (0.3, 0.6):
            Jm, _ = G.gswo(p, n, mu, w.obj.centroid, w.obj.rho, n_iter=20000)
            assert Jm <= ref + 1e-9, (mu, Jm, ref)
