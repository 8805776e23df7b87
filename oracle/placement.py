"""FP64 oracle of object placement (Sec. 5.2) and object preprocessing (Sec.
5.1) -- TEST INFRASTRUCTURE ONLY (imported by tests/, never by the GPU
library).

  place_canonical   the object's centroid at g + d up (d uniform in [d_lo, d_hi])
                    under a uniform rotation (Shoemake's quaternion)
  table_codes       the field's codes in table order (cell z-major, x fastest;
                    then finger; then bin)
  place_exhaustive  a random field code's cell centre and bin direction aligned
                    with a random object point and its flipped normal, spun by a
                    random angle about the normal
  place_static      the object against the palm (a static link): a random point
                    of the palm's top face meets a random object point whose
                    outward normal faces into the palm, spun by a random angle
                    about the palm normal; rejected when some object point sinks
                    into the palm deeper than the penetration margin
  concave_keep      the small-box test: a cube of side s resting on the tangent
                    plane outside each point; the point goes when the SDF at the
                    cube's centre or a corner of its upper half is below -tau
The draws are Philox4x32-10 words at counter (pose + pose_base, tag, 0, 0), key
seed, with u = (w >> 8) 2^-24; poses are rounded to FP32.
"""
from __future__ import annotations

import math

import numpy as np

from . import _onb_duff, philox4x32_10
from .kinematics import sdf_trilinear

TAG_CANONICAL = 0x91AC
TAG_EXHAUSTIVE = 0xE7A1
TAG_STATIC = 0x57A7


def _words(i, tag, seed):
    return philox4x32_10([i, tag, 0, 0], [int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF])


def _u(w):
    return (int(w) >> 8) * 2.0 ** -24


def _rodrigues(k, ang):
    k = np.asarray(k, np.float64)
    s, c = math.sin(ang), math.cos(ang)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return c * np.eye(3) + s * K + (1 - c) * np.outer(k, k)


def _pose32(R, t):
    return np.concatenate([np.asarray(R, np.float64), np.asarray(t, np.float64)[:, None]], axis=1).reshape(12) \
        .astype(np.float32)


def place_canonical(P, centroid, g, up, d_lo, d_hi, seed, pose_base=0):
    c = np.asarray(centroid, np.float32).astype(np.float64)
    g = np.asarray(g, np.float32).astype(np.float64)
    up = np.asarray(up, np.float32).astype(np.float64)
    d_lo, d_hi = float(np.float32(d_lo)), float(np.float32(d_hi))
    out = np.zeros((P, 12), np.float32)
    for i in range(P):
        w = _words(i + pose_base, TAG_CANONICAL, seed)
        u1, u2, u3, u4 = (_u(x) for x in w)
        s1, s2 = math.sqrt(1 - u1), math.sqrt(u1)
        x, y, z, qw = (s1 * math.sin(2 * math.pi * u2), s1 * math.cos(2 * math.pi * u2),
                       s2 * math.sin(2 * math.pi * u3), s2 * math.cos(2 * math.pi * u3))
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * qw), 2 * (x * z + y * qw)],
                      [2 * (x * y + z * qw), 1 - 2 * (x * x + z * z), 2 * (y * z - x * qw)],
                      [2 * (x * z - y * qw), 2 * (y * z + x * qw), 1 - 2 * (x * x + y * y)]])
        d = d_lo + u4 * (d_hi - d_lo)
        out[i] = _pose32(R, g + d * up - R @ c)
    return out


def slot_bits(B: int) -> int:
    return 8 if B <= 8 else (16 if B <= 16 else 32)


def table_codes(field) -> np.ndarray:
    """All (kx, ky, kz, finger, bin) codes of an oracle Field, in table order."""
    codes = [np.concatenate([field.codes(f), np.full((len(field.codes(f)), 1), f)], axis=1)
             for f in range(field.F)]
    c = np.concatenate(codes)[:, [0, 1, 2, 4, 3]]  # kx ky kz f b
    lo = c[:, :3].min(axis=0)
    dims = c[:, :3].max(axis=0) - lo + 1
    cell = ((c[:, 2] - lo[2]) * dims[1] + (c[:, 1] - lo[1])) * dims[0] + (c[:, 0] - lo[0])
    order = np.lexsort((c[:, 4], c[:, 3], cell))
    return c[order]


def place_exhaustive(field, bins, inv_h, soa, P, seed, pose_base=0):
    """Returns (poses [P,12] float32, chosen (code [P,5], point [P]))."""
    codes = table_codes(field)
    n = codes.shape[0]
    soa = np.asarray(soa, np.float32)
    N = soa.shape[1]
    ih = float(np.float32(inv_h))
    dirs = np.asarray(bins, np.float32).astype(np.float64)
    out = np.zeros((P, 12), np.float32)
    chosen = np.zeros((P, 5), np.int64)
    pts = np.zeros(P, np.int64)
    for i in range(P):
        w = _words(i + pose_base, TAG_EXHAUSTIVE, seed)
        r = (int(w[0]) * n) >> 32
        kx, ky, kz, f, b = (int(v) for v in codes[r])
        cpos = np.array([(kx + 0.5) / ih, (ky + 0.5) / ih, (kz + 0.5) / ih])
        d = dirs[b] / np.linalg.norm(dirs[b])
        x = (int(w[1]) * N) >> 32
        a = soa[3:6, x].astype(np.float64)
        a = a / np.linalg.norm(a)
        bv = -d
        v = np.cross(a, bv)
        s = float(np.linalg.norm(v))
        cdot = float(a @ bv)
        if s > 1e-12:
            Ra = _rodrigues(v / s, math.atan2(s, cdot))
        elif cdot < 0:
            e = np.array([1.0, 0.0, 0.0]) if abs(a[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
            k = np.cross(a, e)
            Ra = _rodrigues(k / np.linalg.norm(k), math.pi)
        else:
            Ra = np.eye(3)
        R = _rodrigues(d, 2 * math.pi * _u(w[2])) @ Ra
        t = cpos - R @ soa[0:3, x].astype(np.float64)
        out[i] = _pose32(R, t)
        chosen[i] = (kx, ky, kz, f, b)
        pts[i] = x
    return out, chosen, pts


def place_static(palm_lo, palm_hi, soa, P, seed, pose_base=0, pen_margin=2e-3, band=1e-6):
    """Sec. 5.2, static links.  Returns (poses [P,12] float32, static point [P],
    valid [P] uint8, ambiguous [P] bool).  The penetration test uses the stored
    FP32 pose evaluated in FP64; a pose is ambiguous when a point's depth below
    the face, or its distance to the rectangle's edges, is within `band` of a
    decision boundary."""
    lo = np.asarray(palm_lo, np.float32).astype(np.float64)
    hi = np.asarray(palm_hi, np.float32).astype(np.float64)
    soa = np.asarray(soa, np.float32)
    N = soa.shape[1]
    pts = soa[0:3].T.astype(np.float64)
    top = float(np.float32(np.float32(hi[2]) - np.float32(pen_margin)))  # the kernel's threshold, in FP32
    out = np.zeros((P, 12), np.float32)
    xs = np.zeros(P, np.int64)
    valid = np.zeros(P, np.uint8)
    amb = np.zeros(P, bool)
    z = np.array([0.0, 0.0, 1.0])
    for i in range(P):
        w = _words(i + pose_base, TAG_STATIC, seed)
        x = (int(w[0]) * N) >> 32
        c = np.array([lo[0] + _u(w[1]) * (hi[0] - lo[0]), lo[1] + _u(w[2]) * (hi[1] - lo[1]), hi[2]])
        a = soa[3:6, x].astype(np.float64)
        a = a / np.linalg.norm(a)
        b = -z
        v = np.cross(a, b)
        sv = float(np.linalg.norm(v))
        cdot = float(a @ b)
        if sv > 1e-12:
            Ra = _rodrigues(v / sv, math.atan2(sv, cdot))
        elif cdot < 0:  # n_x = +z
            Ra = _rodrigues(np.array([0.0, 1.0, 0.0]), math.pi)
        else:
            Ra = np.eye(3)
        R = _rodrigues(z, 2 * math.pi * _u(w[3])) @ Ra
        t = c - R @ soa[0:3, x].astype(np.float64)
        out[i] = _pose32(R, t)
        xs[i] = x
        T = out[i].astype(np.float64).reshape(3, 4)
        q = pts @ T[:, :3].T + T[:, 3]
        inside = np.all((q[:, :2] >= lo[:2]) & (q[:, :2] <= hi[:2]), axis=1) & (q[:, 2] >= lo[2])
        pen = inside & (q[:, 2] < top)
        valid[i] = 0 if pen.any() else 1
        # decisions within the band of a boundary: depth at the threshold, or a rectangle / bottom edge
        near = (np.abs(q[:, 2] - top) <= band) | np.any(np.abs(q[:, :2] - lo[:2]) <= band, axis=1) | \
            np.any(np.abs(q[:, :2] - hi[:2]) <= band, axis=1) | (np.abs(q[:, 2] - lo[2]) <= band)
        close = near & (q[:, 2] < top + band) & (q[:, 2] >= lo[2] - band) & \
            np.all((q[:, :2] >= lo[:2] - band) & (q[:, :2] <= hi[:2] + band), axis=1)
        # firm when some penetrating point is clear of the band; otherwise a close point may flip it
        amb[i] = bool(close.any()) and not bool((pen & ~close).any())
    return out, xs, valid, amb


def concave_keep(soa, grid, amb, lo, h, side, tau, band=1e-6):
    """Keep flags [N] and an ambiguity flag per point (a sample within `band` of
    -tau, or on a sign-ambiguous SDF node)."""
    soa = np.asarray(soa, np.float32)
    p = soa[0:3].T.astype(np.float64)
    n = soa[3:6].T.astype(np.float64)
    hs = 0.5 * float(np.float32(side))
    c = p + hs * n
    # the cube rests on the tangent plane: axes (t1, t2, n), t1, t2 the Duff et al. 2017 basis of n
    t1 = np.zeros_like(n)
    t2 = np.zeros_like(n)
    for i in range(n.shape[0]):
        t1[i], t2[i] = _onb_duff(n[i])
    # the centre and the corners of the cube's upper half (heights s/2 and s above the tangent plane)
    offs = [np.zeros_like(n)] + [hs * ((1 if k & 1 else -1) * t1 + (1 if k & 2 else -1) * t2 +
                                       (1 if k & 4 else 0) * n) for k in range(8)]
    vals, ambs = [], []
    for o in offs:
        v, a = sdf_trilinear(grid, amb, lo, h, c + o)
        vals.append(v)
        ambs.append(a)
    V = np.stack(vals, axis=1)
    A = np.stack(ambs, axis=1)
    m = V.min(axis=1)
    keep = ~(m < -tau)
    ambiguous = np.any(np.abs(V + tau) <= band, axis=1) | np.any(A & (V < 0), axis=1)
    return keep.astype(np.uint8), ambiguous
