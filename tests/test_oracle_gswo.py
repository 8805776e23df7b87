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
        for _ in range(200):
            a = rng.normal()
            b = rng.normal(size=2)
            pa, pb = G.project_cone(a, b, mu)
            ra, rb = a - pa, b - pb
            assert np.linalg.norm(pb) <= mu * pa + 1e-12            # in the cone
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
