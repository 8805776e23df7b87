"""FP64 oracle of the kinematics optimisation and post-processing -- TEST
INFRASTRUCTURE ONLY (imported by tests/, smoke() and the CPU-baseline leg of
bench.py; never by the GPU library).

Plain numpy, vectorised over contacts, following the paper's steps in order:

  chain / jacobian   forward kinematics of a finger chain and the position
                     Jacobian of a point attached to link l: column j is
                     a_j x (x - o_j) for j <= l, else 0 (Sec. 5.5, the point
                     form of J_p - [p~]x J_r)
  dls_step           one damped-least-squares update: the solution of
                     (J^T J + lambda I) dq = J^T e for the two position targets
                     p~ -> p and p~ + beta n~ -> p + beta n (Eq. DLS, Sec. 5.5),
                     then clamped to the joint limits
  project_capsule    Phase II ("Finetuning" of Sec. 5.5): the contact vector
                     (p, n) projected onto the contact link's capsule -- the
                     axis point nearest p, and there the capsule normal that
                     minimises the DLS objective
  ik_dls             reverse lookup (the representative field sample of the
                     contact's code) + Phase I + Phase II + success test
  sdf_grid           signed distance of the oriented point set on a grid, by
                     brute force (nearest point; sign of (x - p) . n)
  segment_distance   distance of two segments: minimum of a convex quadratic on
                     the unit square over its stationary point and four edges
  realize            random values for free joints, capsule-vs-SDF
                     penetration and finger-finger capsule intersection
                     (Sec. 5.6 "Postprocessing")

Decisions that sit within a tolerance band of their threshold are reported as
ambiguous rather than forced, so that tests compare only what FP32 and FP64
must agree on.
"""
from __future__ import annotations

import math

import numpy as np

from . import pack_code, philox4x32_10, point_codes, rep_codes

# ---------------------------------------------------------------------------
# kinematics
# ---------------------------------------------------------------------------


def rodrigues(axis: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Rotation by angle q about unit axis (axis-angle formula), [G,3,3]."""
    x, y, z = axis[:, 0], axis[:, 1], axis[:, 2]
    s, c = np.sin(q), np.cos(q)
    v = 1.0 - c
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = c + x * x * v
    R[:, 0, 1] = x * y * v - z * s
    R[:, 0, 2] = x * z * v + y * s
    R[:, 1, 0] = y * x * v + z * s
    R[:, 1, 1] = c + y * y * v
    R[:, 1, 2] = y * z * v - x * s
    R[:, 2, 0] = z * x * v - y * s
    R[:, 2, 1] = z * y * v + x * s
    R[:, 2, 2] = c + z * z * v
    return R


def chain(hand, f, q):
    """Link frames of fingers f [G] at joint vectors q [G,J] (FP64).

    frame_{-1} = base[f]; frame_j = frame_{j-1} Trans(offset_{j-1}) Rot(axis_j, q_j).
    Returns R [G,J,3,3], t [G,J,3] (frame of link j; t_j is also the origin of
    joint j) and the palm-frame joint axes a [G,J,3] (= R_{j-1} axis_j)."""
    f = np.atleast_1d(np.asarray(f, np.int64))
    q = np.atleast_2d(np.asarray(q, np.float64))
    G, J = q.shape
    base = hand.base[f].astype(np.float64).reshape(G, 3, 4)
    axis = hand.axis[f].astype(np.float64)
    off = hand.offset[f].astype(np.float64)
    R = base[:, :, :3].copy()
    t = base[:, :, 3].copy()
    Rs = np.empty((G, J, 3, 3))
    ts = np.empty((G, J, 3))
    aw = np.empty((G, J, 3))
    for j in range(J):
        if j > 0:
            t = t + np.einsum("gij,gj->gi", R, off[:, j - 1])
        aw[:, j] = np.einsum("gij,gj->gi", R, axis[:, j])
        R = R @ rodrigues(axis[:, j], q[:, j])
        Rs[:, j] = R
        ts[:, j] = t
    return Rs, ts, aw


def jacobian(aw: np.ndarray, origins: np.ndarray, l: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Position Jacobian [G,3,J] of palm-frame point x [G,3] rigidly attached to
    link l [G]: column j = a_j x (x - o_j) for j <= l, else 0."""
    G, J, _ = aw.shape
    cols = np.cross(aw, x[:, None, :] - origins)  # [G,J,3]
    cols[np.arange(J)[None, :] > l[:, None]] = 0.0
    return np.transpose(cols, (0, 2, 1))


def _attached(R, t, l, pl, nl):
    g = np.arange(R.shape[0])
    Rl, tl = R[g, l], t[g, l]
    x1 = np.einsum("gij,gj->gi", Rl, pl) + tl
    nn = np.einsum("gij,gj->gi", Rl, nl)
    return Rl, tl, x1, nn


def dls_step(hand, f, l, pl, nl, p, n, q, beta: float, lam: float, return_parts: bool = False):
    """One DLS update (Eq. DLS): dq = (J^T J + lam I)^-1 J^T e, e = [p - p~;
    p + beta n - (p~ + beta n~)], J the stacked Jacobians of p~ and p~ + beta n~;
    q + dq clamped to [lo, hi]."""
    R, t, aw = chain(hand, f, q)
    _, _, x1, nn = _attached(R, t, l, pl, nl)
    x2 = x1 + beta * nn
    e = np.concatenate([p - x1, (p + beta * n) - x2], axis=1)                     # [G,6]
    Jm = np.concatenate([jacobian(aw, t, l, x1), jacobian(aw, t, l, x2)], axis=1)  # [G,6,J]
    Jn = Jm.shape[2]
    A = np.einsum("gri,grj->gij", Jm, Jm) + lam * np.eye(Jn)[None]
    b = np.einsum("gri,gr->gi", Jm, e)
    dq = np.linalg.solve(A, b[..., None])[..., 0]
    lo = hand.lo[f].astype(np.float64)
    hi = hand.hi[f].astype(np.float64)
    qn = np.clip(q + dq, lo, hi)
    if return_parts:
        return qn, dq, Jm, e
    return qn


def project_capsule(hand, f, l, q, p, n, pl, nl, beta: float):
    """Phase II projection of the target contact vector (p, n) onto the
    capsule of link l (axis from the link origin along its offset, radius r).
    The axis point c nearest p is the projection of p onto the link; the new
    attached normal is the outward capsule normal at c that minimises the DLS
    objective |p~ - p|^2 + |p~ + beta n~ - p - beta n|^2 with p~ = c + r n~,
    i.e. the direction of w = (2r + beta)(p - c) + beta (r + beta) n, restricted
    to the normals the capsule has at c (perpendicular to the axis inside the
    segment, the outward hemisphere at an end).  Returns the new attached
    point / normal (link frame) and the palm-frame point / normal.  A
    degenerate w keeps the attached point."""
    f = np.atleast_1d(np.asarray(f, np.int64))
    R, t, _ = chain(hand, f, q)
    Rl, tl, x_old, n_old = _attached(R, t, l, pl, nl)
    off = hand.offset[f, l].astype(np.float64)
    rad = hand.radius[f, l].astype(np.float64)
    bv = np.einsum("gij,gj->gi", Rl, off)
    L2 = np.einsum("gi,gi->g", bv, bv)
    pos_len = L2 > 0
    L2s = np.where(pos_len, L2, 1.0)
    s = np.where(pos_len, np.clip(np.einsum("gi,gi->g", p - tl, bv) / L2s, 0.0, 1.0), 0.0)
    cpt = tl + s[:, None] * bv
    w = (2.0 * rad + beta)[:, None] * (p - cpt) + (beta * (rad + beta))[:, None] * n
    u = bv / np.sqrt(L2s)[:, None]
    wu = np.einsum("gi,gi->g", w, u)
    to_perp = pos_len & (((s > 0) & (s < 1)) | ((s <= 0) & (wu > 0)) | ((s >= 1) & (wu < 0)))
    w = np.where(to_perp[:, None], w - wu[:, None] * u, w)
    wn = np.linalg.norm(w, axis=1)
    moved = wn > 1e-12
    nw = np.where(moved[:, None], w / np.where(moved, wn, 1.0)[:, None], n_old)
    xw = np.where(moved[:, None], cpt + rad[:, None] * nw, x_old)
    pl_new = np.einsum("gji,gj->gi", Rl, xw - tl)
    nl_new = np.einsum("gji,gj->gi", Rl, nw)
    return np.where(moved[:, None], pl_new, pl), np.where(moved[:, None], nl_new, nl), xw, nw


def _pose_targets(soa, poses, pose_idx, x):
    """FP64 contact-surface vector (R p + t, -(R n)) of points x under poses."""
    P = np.asarray(poses, np.float64).reshape(-1, 3, 4)[pose_idx]
    pts = np.asarray(soa, np.float64)[:3, x].T
    nrm = np.asarray(soa, np.float64)[3:, x].T
    p = np.einsum("gij,gj->gi", P[:, :, :3], pts) + P[:, :, 3]
    n = -np.einsum("gij,gj->gi", P[:, :, :3], nrm)
    return p, n, P


def ik_dls(hand, qs, inv_h, bins, soa, poses, T: int, k: int, tuples, fingers, accept, beta=0.01, lam=1e-4,
           n_phase1=16, n_rounds=4, n_phase2=4, tol_pos=2e-3, tol_cos=None, tol_deg=20.0, rep=None,
           perturb: float = 0.0, dilation=None, rep_sure=None, start_tau: float = 1e-6):
    """Kinematics optimisation of tuple slots (Sec. 5.5), same outputs as the
    library call: dict(q [n,F,J], used, contacts [6,n*k], rtuples [n,k],
    resid [n,k,2], ok [n], miss [n,k] (contact code without representative),
    start_amb [n,k] (the contact's FP64 code, or its representative, could
    change under a perturbation of start_tau metres (1e-6 in cosine on a bin
    tie), so a correct FP32 lookup may start from another sample; 1e-6 m is
    some 20 times the FP32 rounding of the kinematic chain)).
    ``rep`` maps finger -> {packed code: s*M + m}; ``rep_sure`` finger -> set
    of codes whose representative is band-stable; both computed when None.
    ``perturb`` shifts targets by that many metres and the starting joints by
    that many radians (a sensitivity probe)."""
    tuples = np.asarray(tuples, np.int64).reshape(-1, k)
    fingers = np.asarray(fingers, np.int64).reshape(-1, k)
    n = tuples.shape[0]
    F, J, M = hand.F, hand.J, hand.M
    N = np.asarray(soa).shape[1]
    if tol_cos is None:
        tol_cos = float(np.float32(math.cos(math.radians(tol_deg))))
    acc = np.ones(n, bool) if accept is None else np.asarray(accept).reshape(-1).astype(bool)
    valid = acc & np.all((tuples >= 0) & (tuples < N) & (fingers < F), axis=1)
    for a in range(k):
        for b in range(a + 1, k):
            valid &= fingers[:, a] != fingers[:, b]
    out = dict(q=np.zeros((n, F, J), np.float64), used=np.zeros((n, F, J), np.uint8),
               contacts=np.zeros((6, n * k)), rtuples=np.full((n, k), -1, np.int64),
               resid=np.tile(np.array([np.inf, -2.0]), (n, k, 1)), ok=np.zeros(n, np.uint8),
               miss=np.zeros((n, k), bool), start_amb=np.zeros((n, k), bool))
    slots = np.nonzero(valid)[0]
    if slots.size == 0:
        return out
    sl = np.repeat(slots, k)
    cc = np.tile(np.arange(k), slots.size)
    x = tuples[sl, cc]
    f = fingers[sl, cc]
    pose_idx = sl // T
    if rep is None:
        both = {ff: rep_codes(hand, qs, inv_h, bins, ff, with_sure=True, tau=start_tau)
                for ff in np.unique(f).tolist()}
        rep = {ff: v[0] for ff, v in both.items()}
        rep_sure = {ff: v[1] for ff, v in both.items()}
    codes, camb = point_codes(soa, poses, pose_idx, x, inv_h, bins, with_amb=True, tau=start_tau)

    def lookup(ff, cd):
        # the contact's own bin first; with dilated bins, then the lowest other accepted bin present
        kx, ky, kz, b = cd
        order = [b]
        if dilation is not None:
            order += [b2 for b2 in range(32) if (int(dilation[b]) >> b2) & 1 and b2 != b]
        for b2 in order:
            key = pack_code(ff, kx, ky, kz, b2)
            v = rep[int(ff)].get(key)
            if v is not None:
                return v, rep_sure is not None and key not in rep_sure[int(ff)]
        return -1, False

    found = [lookup(ff, cd) for ff, cd in zip(f.tolist(), codes.tolist())]
    v = np.array([r[0] for r in found], np.int64)
    out["start_amb"][sl, cc] = camb.astype(bool) | np.array([r[1] for r in found], bool)
    miss = v < 0
    vv = np.where(miss, 0, v)
    s_idx, m_idx = vv // M, vv % M
    q = np.asarray(qs, np.float32)[f, :, s_idx].astype(np.float64)      # [G,J]
    q[miss] = hand.lo[f[miss]].astype(np.float64)
    pl = hand.surf_p[f, m_idx].astype(np.float64)
    nl = hand.surf_n[f, m_idx].astype(np.float64)
    l = hand.surf_link[f, m_idx].astype(np.int64)
    p, nvec, P = _pose_targets(soa, poses, pose_idx, x)
    if perturb:
        p = p + perturb / math.sqrt(3.0)
        q = np.clip(q + perturb, hand.lo[f], hand.hi[f])
    for _ in range(n_phase1):
        q = dls_step(hand, f, l, pl, nl, p, nvec, q, beta, lam)
    for _ in range(n_rounds):
        pl, nl, _, _ = project_capsule(hand, f, l, q, p, nvec, pl, nl, beta)
        for _ in range(n_phase2):
            q = dls_step(hand, f, l, pl, nl, p, nvec, q, beta, lam)
    pl, nl, xw, nw = project_capsule(hand, f, l, q, p, nvec, pl, nl, beta)
    pos = np.linalg.norm(xw - p, axis=1)
    cosv = np.einsum("gi,gi->g", nw, nvec)
    # a contact whose code has no representative is not attempted: joints at
    # their lower limits, nothing used, no residual
    q[miss] = hand.lo[f[miss]].astype(np.float64)
    pos[miss] = np.inf
    cosv[miss] = -2.0
    xw[miss] = P[miss][:, :, 3]
    nw[miss] = 0.0
    l = np.where(miss, -1, l)
    okc = (pos <= tol_pos) & (cosv >= tol_cos) & ~miss
    gok = okc.reshape(-1, k).all(axis=1)
    out["ok"][slots] = gok
    out["miss"][sl, cc] = miss
    out["q"][sl, f] = q
    out["used"][sl, f] = (np.arange(J)[None, :] <= l[:, None]).astype(np.uint8)
    out["resid"][sl, cc, 0] = pos
    out["resid"][sl, cc, 1] = cosv
    e = sl * k + cc
    R = P[:, :, :3]
    xo = np.einsum("gji,gj->gi", R, xw - P[:, :, 3])
    no = -np.einsum("gji,gj->gi", R, nw)
    out["contacts"][:3, e] = xo.T
    out["contacts"][3:, e] = no.T
    okr = np.repeat(gok, k)
    out["rtuples"][sl, cc] = np.where(okr, e, -1)
    return out


# ---------------------------------------------------------------------------
# object SDF and realization checks
# ---------------------------------------------------------------------------


def sdf_grid(soa, lo, h, dims, rel_tie: float = 1e-5):
    """Signed distance of the oriented point set on the grid lo + (i,j,k) h
    (brute force, FP64).  Returns grid [dz,dy,dx] and a per-node ambiguity flag:
    the sign decision is ambiguous when points within a relative distance
    rel_tie of the nearest disagree on it, or (x - p) . n is ~0, at a node more
    than 1e-6 m from the nearest point."""
    soa = np.asarray(soa, np.float64)
    pts, nrm = soa[:3].T, soa[3:].T
    lo = np.asarray(lo, np.float32).astype(np.float64)
    h = float(np.float32(h))
    dx, dy, dz = (int(d) for d in dims)
    iz, iy, ix = np.meshgrid(np.arange(dz), np.arange(dy), np.arange(dx), indexing="ij")
    g = np.stack([lo[0] + ix.ravel() * h, lo[1] + iy.ravel() * h, lo[2] + iz.ravel() * h], axis=1)
    val = np.empty(g.shape[0])
    amb = np.zeros(g.shape[0], bool)
    N = pts.shape[0]
    if N == 0:
        val[:] = np.inf
        return val.reshape(dz, dy, dx), amb.reshape(dz, dy, dx)
    chunk = max(1, (1 << 22) // N)
    for a in range(0, g.shape[0], chunk):
        gg = g[a:a + chunk]
        diff = gg[:, None, :] - pts[None, :, :]
        d2 = np.einsum("cni,cni->cn", diff, diff)
        idx = np.argmin(d2, axis=1)
        d2m = d2[np.arange(gg.shape[0]), idx]
        side = np.einsum("cni,ni->cn", diff, nrm)
        sm = side[np.arange(gg.shape[0]), idx]
        val[a:a + chunk] = np.where(sm >= 0, np.sqrt(d2m), -np.sqrt(d2m))
        near = d2 <= d2m[:, None] * (1.0 + rel_tie) ** 2 + 1e-18
        pos_near = np.any(near & (side >= 0), axis=1)
        neg_near = np.any(near & (side < 0), axis=1)
        # a node within 1e-6 m of the surface has |value| ~ 0, so its sign cannot matter
        amb[a:a + chunk] = ((pos_near & neg_near) | (np.abs(sm) <= 1e-9)) & (d2m > 1e-12)
    return val.reshape(dz, dy, dx), amb.reshape(dz, dy, dx)


def sdf_trilinear(grid, amb, lo, h, x):
    """Trilinear SDF at points x [G,3]; +inf outside the grid.  Also returns
    whether any of the 8 nodes used is sign-ambiguous."""
    lo = np.asarray(lo, np.float32).astype(np.float64)
    h = float(np.float32(h))
    dz, dy, dx = grid.shape
    u = (x - lo) / h
    i0 = np.floor(u).astype(np.int64)
    fr = u - i0
    inside = np.all(i0 >= 0, axis=1) & (i0[:, 0] + 1 < dx) & (i0[:, 1] + 1 < dy) & (i0[:, 2] + 1 < dz)
    out = np.full(x.shape[0], np.inf)
    a_out = np.zeros(x.shape[0], bool)
    if not inside.any():
        return out, a_out
    ii = i0[inside]
    ff = fr[inside]
    acc = np.zeros(ii.shape[0])
    aa = np.zeros(ii.shape[0], bool)
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                w = (ff[:, 0] if cx else 1 - ff[:, 0]) * (ff[:, 1] if cy else 1 - ff[:, 1]) * \
                    (ff[:, 2] if cz else 1 - ff[:, 2])
                acc += w * grid[ii[:, 2] + cz, ii[:, 1] + cy, ii[:, 0] + cx]
                aa |= amb[ii[:, 2] + cz, ii[:, 1] + cy, ii[:, 0] + cx]
    out[inside] = acc
    a_out[inside] = aa
    return out, a_out


def segment_distance(p0, p1, q0, q1) -> float:
    """min over s, t in [0,1] of |p0 + s (p1 - p0) - q0 - t (q1 - q0)|: the
    convex quadratic's minimum is at its stationary point (when inside) or on
    one of the four edges, where each 1-D minimum is a clamped projection."""
    p0, p1, q0, q1 = (np.asarray(v, np.float64) for v in (p0, p1, q0, q1))
    d1, d2, r = p1 - p0, q1 - q0, p0 - q0
    a, e, b = d1 @ d1, d2 @ d2, d1 @ d2
    c, f = d1 @ r, d2 @ r

    def dist(s, t):
        return float(np.linalg.norm(r + s * d1 - t * d2))

    cands = []
    den = a * e - b * b
    if den > 0:
        s = (b * f - c * e) / den
        t = (f + s * b) / e if e > 0 else 0.0
        if 0 <= s <= 1 and 0 <= t <= 1:
            cands.append(dist(s, t))
    for s in (0.0, 1.0):
        t = min(max(((r + s * d1) @ d2) / e, 0.0), 1.0) if e > 0 else 0.0
        cands.append(dist(s, t))
    for t in (0.0, 1.0):
        s = min(max(-((r - t * d2) @ d1) / a, 0.0), 1.0) if a > 0 else 0.0
        cands.append(dist(s, t))
    return min(cands)


def capsules(hand, axis_step: float):
    """Capsule links in (finger, link) order: (f, j, radius, ns) with
    ns = max(1, ceil(length / axis_step)) axis intervals."""
    out = []
    step = float(np.float32(axis_step))
    for f in range(hand.F):
        for j in range(hand.J):
            o = hand.offset[f, j]
            ln = math.sqrt(float(o[0]) * float(o[0]) + float(o[1]) * float(o[1]) + float(o[2]) * float(o[2]))
            r = float(hand.radius[f, j])
            if r > 0 and ln > 0:
                out.append((f, j, r, int(max(1.0, math.ceil(ln / step)))))
    return out


def random_joint(lo, hi, word):
    """lo + (u24 * 2^-24) * (hi - lo), every operation rounded to FP32."""
    u = np.float32(int(word) >> 8) * np.float32(2.0 ** -24)
    return np.float32(np.float32(lo) + np.float32(u * np.float32(np.float32(hi) - np.float32(lo))))


def realize(hand, sdf, sdf_amb, sdf_lo, sdf_h, poses, T: int, q, used, gate_a, gate_b, pen_margin=2e-3,
            axis_step=1.25e-3, seed=0, band=1e-5, slot_ids=None):
    """Post-processing of tuple slots (Sec. 5.6).  Returns (q [n,F,J] float32
    with free joints filled, flags [n] uint8 (1 gated out, 2 penetration,
    4 self-collision), ambiguous [n] bool).  Slot u takes pose u // T; its
    draws are keyed by slot_ids[u], its index in its launch (default u), so
    that slots taken out of a larger launch keep their draws."""
    q = np.array(q, np.float32, copy=True)
    used = np.asarray(used)
    n = q.shape[0]
    slot_ids = np.arange(n) if slot_ids is None else np.asarray(slot_ids, np.int64)
    if slot_ids.shape != (n,):
        raise ValueError("slot_ids must hold one index per slot")
    F, J = hand.F, hand.J
    ga = np.ones(n, bool) if gate_a is None else np.asarray(gate_a).astype(bool)
    gb = np.ones(n, bool) if gate_b is None else np.asarray(gate_b).astype(bool)
    flags = np.ones(n, np.uint8)
    ambig = np.zeros(n, bool)
    caps = capsules(hand, axis_step)
    key = [int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF]
    Pz = np.asarray(poses, np.float64).reshape(-1, 3, 4)
    for u in np.nonzero(ga & gb)[0].tolist():
        for f in range(F):
            words = None
            for j in range(J):
                if j % 4 == 0:
                    words = philox4x32_10([int(slot_ids[u]), f, j // 4, 0x7EA1], key)
                if not used[u, f, j]:
                    q[u, f, j] = random_joint(hand.lo[f, j], hand.hi[f, j], words[j % 4])
        R, t, _ = chain(hand, np.arange(F), q[u].astype(np.float64))
        segs = []
        for (f, j, r, ns) in caps:
            a = t[f, j]
            b = a + R[f, j] @ hand.offset[f, j].astype(np.float64)
            segs.append((f, a, b, r, ns))
        Pu = Pz[u // T]
        pen_sure = pen_poss = False
        for (f, a, b, r, ns) in segs:
            s = np.arange(ns + 1, dtype=np.float64) / ns
            x = a[None, :] + s[:, None] * (b - a)[None, :]
            xo = (x - Pu[:, 3]) @ Pu[:, :3]
            v, va = sdf_trilinear(sdf, sdf_amb, sdf_lo, sdf_h, xo)
            thr = r - pen_margin
            pen_sure |= bool(np.any((v < thr - band) & ~va))
            pen_poss |= bool(np.any((v < thr + band) | va))
        col_sure = col_poss = False
        for i1 in range(len(segs)):
            for i2 in range(i1 + 1, len(segs)):
                f1, a1, b1, r1, _ = segs[i1]
                f2, a2, b2, r2, _ = segs[i2]
                if f1 == f2:
                    continue
                d = segment_distance(a1, b1, a2, b2)
                col_sure |= d < r1 + r2 - band
                col_poss |= d < r1 + r2 + band
        flags[u] = (2 if pen_sure else 0) | (4 if col_sure else 0)
        ambig[u] = (pen_sure != pen_poss) or (col_sure != col_poss)
    return q, flags, ambig
