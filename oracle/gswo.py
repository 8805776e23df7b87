"""FP64 oracle of the paper's own grasp metric, Eq. GSWO (Sec. 3.2) with true
quadratic friction cones -- TEST INFRASTRUCTURE ONLY (imported by tests/ and
bench.py's CPU legs, never by the GPU library).

For a tuple of k contacts with inward force directions nu_i = -n_i and the
Duff et al. 2017 tangent basis (x_i, y_i) of nu_i, contact i applies
f_i = alpha_i nu_i + bx_i x_i + by_i y_i.  With z = (alpha_i, bx_i, by_i)_i and
A the 6 x 3k matrix whose column block i is [nu_i x_i y_i ; (r_i x nu_i, r_i x x_i,
r_i x y_i) / rho] (r_i = p_i - c), the objective of Eq. GSWO with lambda = 1 /
rho^2 is |A z|^2.  Subproblem j fixes alpha_j = 1 (its friction then lies in the
disc |b_j| <= mu); every other contact lies in the cone |b_i| <= mu alpha_i.
J = min_j J_j.  Eq. FSWO (frictionless) is the case mu = 0: every b is 0 and
each subproblem is the nonnegative least-squares problem min |a_j + A' alpha'|^2,
alpha' >= 0, over the normal columns; the paper notes that GSWO's optimum is a
lower bound of FSWO's.

The paper solves the subproblems by projected gradient descent.  Reading taken
(the paper gives no schedule): projected gradient with Nesterov momentum
(FISTA: t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2), n_iter steps from
alpha = e_j, beta = 0, step 1 / (2 tr(A^T A)) (tr >= the largest eigenvalue, so
the step is safe), evaluating |A z|^2 at the last iterate.  The same iteration
runs in the kernel in FP32.

Functions:
  gswo_matrix(p, n, c, rho)          A (6 x 3k)
  project_cone(a, b, mu)             Euclidean projection onto |b| <= mu a
  gswo_subproblem(A, j, mu, n_iter)  J_j and z
  gswo(p, n, mu, c, rho, n_iter)     J = min_j J_j
  score_gswo(soa, tuples, ...)       J of many tuples
"""
from __future__ import annotations

import math

import numpy as np

from . import _onb_duff


def gswo_matrix(p, n, c, rho) -> np.ndarray:
    p = np.asarray(p, np.float64)
    n = np.asarray(n, np.float64)
    k = p.shape[0]
    A = np.zeros((6, 3 * k))
    for i in range(k):
        nu = -n[i]
        x, y = _onb_duff(nu)
        r = p[i] - np.asarray(c, np.float64)
        for col, d in enumerate((nu, x, y)):
            A[:3, 3 * i + col] = d
            A[3:, 3 * i + col] = np.cross(r, d) / rho
    return A


def project_cone(a: float, b: np.ndarray, mu: float):
    """Nearest point of {(a, b): |b| <= mu a, a >= 0} to (a, b) (second-order cone; at mu = 0 the
    ray b = 0, a >= 0 of a frictionless contact, Eq. FSWO)."""
    s = float(np.linalg.norm(b))
    if a >= 0.0 and s <= mu * a:
        return a, b
    if mu * s <= -a:
        return 0.0, np.zeros_like(b)
    a2 = (a + mu * s) / (1.0 + mu * mu)
    return a2, b * (mu * a2 / s)


def _project(z: np.ndarray, j: int, mu: float) -> np.ndarray:
    k = z.shape[0] // 3
    out = z.copy()
    for i in range(k):
        if i == j:
            out[3 * i] = 1.0
            b = z[3 * i + 1:3 * i + 3]
            s = float(np.linalg.norm(b))
            out[3 * i + 1:3 * i + 3] = b if s <= mu else b * (mu / s)
        else:
            a, b = project_cone(z[3 * i], z[3 * i + 1:3 * i + 3], mu)
            out[3 * i] = a
            out[3 * i + 1:3 * i + 3] = b
    return out


def gswo_subproblem(A: np.ndarray, j: int, mu: float, n_iter: int):
    """J_j = |A z|^2 after n_iter accelerated projected-gradient steps; returns (J_j, z)."""
    Q = A.T @ A
    step = 1.0 / (2.0 * float(np.trace(Q)))
    k = A.shape[1] // 3
    z = np.zeros(3 * k)
    z[3 * j] = 1.0
    y = z.copy()
    t = 1.0
    for _ in range(n_iter):
        z_new = _project(y - step * 2.0 * (Q @ y), j, mu)
        t_new = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        y = z_new + ((t - 1.0) / t_new) * (z_new - z)
        z, t = z_new, t_new
    v = A @ z
    return float(v @ v), z


def gswo(p, n, mu, c, rho, n_iter: int = 256):
    A = gswo_matrix(p, n, c, rho)
    k = A.shape[1] // 3
    vals = [gswo_subproblem(A, j, mu, n_iter)[0] for j in range(k)]
    return min(vals), vals


def score_gswo(soa, tuples, mu, c, rho, n_iter: int = 256):
    """J of every tuple [.., k] of point ids into soa [6, N] (+inf when invalid)."""
    soa = np.asarray(soa, np.float64)
    t = np.asarray(tuples).reshape(-1, np.asarray(tuples).shape[-1])
    out = np.full(t.shape[0], np.inf)
    N = soa.shape[1]
    for u, ids in enumerate(t):
        if np.any(ids < 0) or np.any(ids >= N):
            continue
        out[u] = gswo(soa[0:3, ids].T, soa[3:6, ids].T, mu, c, rho, n_iter)[0]
    return out.reshape(np.asarray(tuples).shape[:-1])
