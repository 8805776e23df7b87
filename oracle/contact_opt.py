"""FP64 oracle of the blockwise zeroth-order contact optimisation (Sec. 5.4,
Alg. 2) -- TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's CPU legs,
never by the GPU library).

The steps of Alg. 2 in the paper's order, for one tuple (p_1, ..., p_k):

  for it = 1 .. n_o, for i = 1 .. k:
    (x, y) = Tangent(n_i)                       Duff et al. 2017 basis of -n_i
    [dx], [dy] = Normal(n_in, sigma^2) x, y     Box-Muller pairs of Philox words
    [p_i'] = p_i + [dx] + [dy]
    [p_i', n_i'] = Project([p_i'], D_i)          nearest point of the domain

The whole iteration is FP64: the tangent basis of the (FP32-given) normal, the
Box-Muller pair, the mutated point and the distances of the projection.
    (p_i, n_i) = argmin J over the candidates     J = closure margin (closure_lp)

Readings (the paper leaves them open): the current point competes with the
candidates, which are taken in order, each replacing the best so far only when
its margin is lower by more than the relative min_gain (so J never increases,
and near-equal margins -- e.g. when contact i carries no force at the optimum
and every candidate ties -- keep the current point); margins <= zero_tol count
as 0, where the optimisation of that tuple stops (nothing beats 0); the
mutation draws are Philox4x32-10 at
counter (pose, tau, (it k + i) ceil(n_in / 2) + c / 2, 0xA162), key seed, words
(2 (c mod 2), 2 (c mod 2) + 1) -> u1 = ((w >> 8) + 1) 2^-24,
u2 = (w' >> 8) 2^-24, (g1, g2) = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).

Each decision that a correct FP32 evaluation could take differently is
recorded as ambiguous: a projection whose nearest and second-nearest domain
points lie within PROJ_GAP = 1e-7 m of the same distance from the mutated
point (far above the FP32 rounding of coordinates near 0.1 m, ~1e-8 m), a
replacement test within 2e-4 max(J, eps) of its threshold (the closure-margin
parity tolerance on each side), or a margin within a factor 2 of zero_tol.
Tests compare only tuples whose whole path is clear of those.
"""
from __future__ import annotations

import math

import numpy as np

from . import _get_pool, closure_lp, philox4x32_10

OPT_TAG = 0xA162


PROJ_GAP = 1e-7  # metres: distance gap below which a projection is ambiguous


def box_muller(w0: int, w1: int):
    """FP64 normal pair from two Philox words (u1 in (0, 1], u2 in [0, 1))."""
    u1 = ((int(w0) >> 8) + 1) * 2.0 ** -24
    u2 = (int(w1) >> 8) * 2.0 ** -24
    r = math.sqrt(-2.0 * math.log(u1))
    return r * math.cos(math.pi * (2.0 * u2)), r * math.sin(math.pi * (2.0 * u2))


def mutation_normals(pose: int, tau: int, it: int, i: int, k: int, n_in: int, seed: int):
    """(g1, g2) of candidates 0 .. n_in-1 of block (it, i), FP64."""
    per = (n_in + 1) // 2
    key = [int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF]
    out = []
    for c in range(n_in):
        w = philox4x32_10([pose, tau, (it * k + i) * per + c // 2, OPT_TAG], key)
        a, b = (w[2], w[3]) if c & 1 else (w[0], w[1])
        out.append(box_muller(a, b))
    return out


def tangent_basis(n):
    """Duff et al. 2017 branchless orthonormal basis (x, y) of nu = -n, FP64."""
    vx, vy, vz = -float(n[0]), -float(n[1]), -float(n[2])
    sgn = math.copysign(1.0, vz)
    aa = -1.0 / (sgn + vz)
    bb = vx * vy * aa
    x = (1.0 + sgn * vx * vx * aa, sgn * bb, -sgn * vx)
    y = (bb, sgn + vy * vy * aa, -vy)
    return x, y


def mutate(p, xv, yv, g1, g2, sigma):
    """p + sigma (g1 x + g2 y), FP64."""
    return tuple(float(p[d]) + float(sigma) * (g1 * xv[d] + g2 * yv[d]) for d in range(3))


def project_to_domain(pts64: np.ndarray, dom: np.ndarray, q, gap: float = PROJ_GAP):
    """Nearest domain point to q by FP64 Euclidean distance, lowest index on
    exact ties; also whether a domain point at another location lies within
    `gap` of the same distance (then an FP32 evaluation may pick it instead;
    copies of the nearest point tie in every precision and go to the lowest
    index on both sides)."""
    P = pts64[dom]
    d = np.sqrt(((P - np.asarray(q, np.float64)[None, :]) ** 2).sum(axis=1))
    j = int(np.argmin(d))
    other = np.any(P != P[j][None, :], axis=1)
    return int(dom[j]), bool(np.any(other & (d <= d[j] + gap)))


def _margin(soa64, ids, mu, K, c, rho):
    p = soa64[0:3, ids].T
    n = soa64[3:6, ids].T
    t, _, _ = closure_lp(p, n, mu, K, c, rho)
    return t


def optimize_tuple(soa, masks_pose, ids, fingers, pose, tau, mu, K, c, rho, eps, seed, n_outer, n_inner, sigma,
                   zero_tol, min_gain=1e-2):
    """One tuple through Alg. 2.  masks_pose = [F][W] mask words of its pose.
    Returns (ids, margin, ambiguous)."""
    soa64 = np.asarray(soa, np.float64)
    ids = [int(x) for x in ids]
    k = len(ids)
    N = soa64.shape[1]
    if any(x < 0 or x >= N for x in ids):
        return ids, math.inf, False
    amb = False
    pts64 = np.ascontiguousarray(soa64[0:3].T)
    nrm64 = soa64[3:6].T
    J = _margin(soa64, ids, mu, K, c, rho)

    def cls(v):
        return 0.0 if v <= zero_tol else v

    def near_zero_band(v):
        return 0.5 * zero_tol <= v <= 2.0 * zero_tol

    amb |= near_zero_band(J)
    Jc = cls(J)
    bits = [np.unpackbits(np.ascontiguousarray(masks_pose[f]).view(np.uint8), bitorder="little") for f in fingers]
    for it in range(n_outer):
        for i in range(k):
            if Jc <= 0.0:
                break
            x0 = ids[i]
            dom = np.nonzero(bits[i][:N])[0]
            xv, yv = tangent_basis(nrm64[x0])
            cands = []
            for (g1, g2) in mutation_normals(pose, tau, it, i, k, n_inner, seed):
                xc, a = project_to_domain(pts64, dom, mutate(pts64[x0], xv, yv, g1, g2, sigma))
                amb |= a
                cands.append(xc)
            best_c, best_raw, best_x = Jc, J, x0
            seen = {x0}
            for xc in cands:
                if xc in seen:
                    continue
                seen.add(xc)
                trial = list(ids)
                trial[i] = xc
                Jt = _margin(soa64, trial, mu, K, c, rho)
                amb |= near_zero_band(Jt)
                Jtc = cls(Jt)
                thr = (1.0 - min_gain) * best_c
                # the decision Jtc < thr flips if either margin moves by its parity tolerance
                if best_c > 0.0 and Jtc > 0.0 and abs(Jtc - thr) <= 2e-4 * max(Jtc, best_c, eps):
                    amb = True
                if Jtc < thr:
                    best_c, best_raw, best_x = Jtc, Jt, xc
            Jc, J = best_c, best_raw
            ids[i] = best_x
        if Jc <= 0.0:
            break
    return ids, J, amb


def _opt_chunk(args):
    (soa, masks, tuples, fingers, pose_ids, us, T, mu, K, c, rho, eps, seed, n_outer, n_inner, sigma, zero_tol,
     min_gain) = args
    out = []
    for u in us:
        row, tau = divmod(int(u), T)
        out.append(optimize_tuple(soa, masks[row], tuples[u], fingers[u], int(pose_ids[row]), tau, mu, K, c, rho, eps,
                                  seed, n_outer, n_inner, sigma, zero_tol, min_gain))
    return out


def optimize_tuples(soa, masks, tuples, fingers, T, mu, K, c, rho, eps, seed, n_outer=2, n_inner=8, sigma=0.005,
                    zero_tol=1e-6, min_gain=1e-2, workers: bool = True, pose_ids=None):
    """All tuples [P,T,k] through Alg. 2: returns (tuples [P,T,k] int32,
    margin [P,T], accept [P,T] uint8, ambiguous [P,T] bool).  pose_ids [P]: the
    index of each row's pose in its request, which keys the row's draws (default
    0 .. P-1), so that rows sampled from a larger request keep their draws."""
    P = masks.shape[0]
    pose_ids = np.arange(P) if pose_ids is None else np.asarray(pose_ids, np.int64)
    if pose_ids.shape != (P,):
        raise ValueError("pose_ids must hold one index per mask row")
    k = tuples.shape[-1]
    flat = np.asarray(tuples, np.int64).reshape(-1, k)
    ff = np.asarray(fingers, np.int64).reshape(-1, k)
    n = flat.shape[0]
    us = np.arange(n)
    soa = np.ascontiguousarray(soa, np.float32)
    masks = np.ascontiguousarray(masks, np.uint32)
    c = np.asarray(c, np.float64)
    base = (soa, masks, flat, ff, pose_ids)
    rest = (T, float(mu), int(K), c, float(rho), float(eps), int(seed), int(n_outer), int(n_inner), float(sigma),
            float(zero_tol), float(min_gain))
    if workers and n > 8:
        chunks = np.array_split(us, min(n, 4 * max(1, (_cpu_count()))))
        futs = [_get_pool().submit(_opt_chunk, (*base, ch, *rest)) for ch in chunks if len(ch)]
        res = [r for f in futs for r in f.result()]
    else:
        res = _opt_chunk((*base, us, *rest))
    out_t = np.array([r[0] for r in res], np.int32).reshape(P, T, k)
    out_m = np.array([r[1] for r in res]).reshape(P, T)
    amb = np.array([r[2] for r in res], bool).reshape(P, T)
    return out_t, out_m, (out_m <= eps).astype(np.uint8), amb


def _cpu_count():
    import os
    return os.cpu_count() or 1
