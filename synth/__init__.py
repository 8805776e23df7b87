"""Seeded synthetic inputs for the Contact-Field grasp path.

This module only *produces inputs*: hand descriptors (capsule-chain kinematics plus
a fixed set of hand surface points in link frames), object surface points with
outward normals, palm poses, joint-space samples and the fixed normal-bin
direction set.  It holds none of the method's arithmetic (no forward
kinematics, no binning, no lookup, no sampling of tuples, no scoring).  Both the
CUDA path and the CPU oracle consume exactly the arrays produced here.

Geometry units are metres; every array handed out is contiguous float32 (or
int32) so that both sides see bit-identical inputs.

The paper's hands (Allegro, LEAP, Shadow, DClaw) and objects (YCB / Sketchfab
meshes) are not available; the generators below stand in for them with the
shapes, sizes and structure of the paper's workloads (Sec. 6, Table 1):
3/4/5-finger capsule hands, a sphere, a superquadric and an irregular
tool-like composite, poses in a canonical placement box above the palm
(Sec. 5.2, "Canonical Placement").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Hand", "Obj", "Workload",
    "fibonacci_dirs", "hand_three_finger", "hand_anthropomorphic",
    "joint_samples", "sphere", "superquadric", "tool_composite",
    "palm_poses", "workload", "WORKLOADS", "batch_objects", "batch_object_inputs",
]

# ---------------------------------------------------------------------------
# normal-bin directions (the fixed direction set that quantises normals;
# Sec. 4.4 "Memory Consumption": normals become an index on a fixed sphere set)
# ---------------------------------------------------------------------------

def fibonacci_dirs(B: int) -> np.ndarray:
    """B unit vectors on a spherical Fibonacci lattice (float64 -> float32)."""
    i = np.arange(B, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / B
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return np.ascontiguousarray(d.astype(np.float32))


# ---------------------------------------------------------------------------
# hands
# ---------------------------------------------------------------------------

@dataclass
class Hand:
    """Capsule-chain hand: F fingers, each a serial chain of J revolute joints.

    Chain convention (shared by every consumer): frame_{-1} = base[f];
    frame_j = frame_{j-1} * Trans(offset[f][j-1]) * Rot(axis[f][j], q_j)
    (offset[f][-1] := 0).  Link j is a capsule from the origin of frame_j to
    offset[f][j] (in frame_j coordinates) with radius radius[f][j].
    Surface point m of finger f lives on link surf_link[f][m], with position
    surf_p and outward normal surf_n expressed in that link's frame.
    """
    name: str
    base: np.ndarray       # [F,12] float32, row-major 3x4 (R | t), palm frame
    axis: np.ndarray       # [F,J,3] float32 unit joint axes
    offset: np.ndarray     # [F,J,3] float32 link vectors
    lo: np.ndarray         # [F,J] float32 joint lower limits (rad)
    hi: np.ndarray         # [F,J] float32 joint upper limits (rad)
    radius: np.ndarray     # [F,J] float32 capsule radii (0 for zero-length links)
    surf_p: np.ndarray     # [F,M,3] float32
    surf_n: np.ndarray     # [F,M,3] float32
    surf_link: np.ndarray  # [F,M] int32
    grasp_centre: np.ndarray  # [3] float64: mean of finger bases (placement anchor)
    palm_lo: np.ndarray = None  # [3] float32: the palm body, a box of the palm frame whose top face is z = 0
    palm_hi: np.ndarray = None  # [3] float32

    @property
    def F(self) -> int:
        return int(self.base.shape[0])

    @property
    def J(self) -> int:
        return int(self.axis.shape[1])

    @property
    def M(self) -> int:
        return int(self.surf_p.shape[1])


def _perp_basis(u: np.ndarray):
    """Two unit vectors completing u to a right-handed frame (deterministic)."""
    u = u / np.linalg.norm(u)
    a = np.array([1.0, 0.0, 0.0]) if abs(u[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(u, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u, e1)
    return e1, e2


def _hemisphere_dirs(u: np.ndarray, n: int) -> np.ndarray:
    """n Fibonacci directions on the hemisphere around unit vector u."""
    e1, e2 = _perp_basis(u)
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (i + 0.5) / n             # cos(angle to u) in (0, 1]
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    return (z[:, None] * u[None, :] + (r * np.cos(phi))[:, None] * e1[None, :]
            + (r * np.sin(phi))[:, None] * e2[None, :])


def _capsule_surface(offsets: np.ndarray, radii: np.ndarray,
                     n_station: int = 4, n_ring: int = 8, n_tip: int = 16):
    """Deterministic surface points of one finger's capsule links.

    Each non-zero link gets n_station axial stations x n_ring radial points
    (outward radial normals); the distal non-zero link also gets n_tip points
    on its tip hemisphere.  Returns (p [M,3], n [M,3], link [M]) in link frames.
    """
    P, N, L = [], [], []
    nz = [j for j in range(len(offsets)) if np.linalg.norm(offsets[j]) > 0]
    for j in nz:
        Lv = offsets[j].astype(np.float64)
        ln = np.linalg.norm(Lv)
        u = Lv / ln
        e1, e2 = _perp_basis(u)
        r = float(radii[j])
        for s in range(n_station):
            a = (s + 0.5) / n_station * ln
            for k in range(n_ring):
                th = 2.0 * math.pi * k / n_ring
                d = math.cos(th) * e1 + math.sin(th) * e2
                P.append(a * u + r * d)
                N.append(d)
                L.append(j)
    jt = nz[-1]
    Lv = offsets[jt].astype(np.float64)
    u = Lv / np.linalg.norm(Lv)
    for d in _hemisphere_dirs(u, n_tip):
        P.append(Lv + float(radii[jt]) * d)
        N.append(d)
        L.append(jt)
    return (np.asarray(P, np.float64), np.asarray(N, np.float64), np.asarray(L, np.int32))


def _rot_z(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _pack_hand(name, bases_R, bases_t, axes, offsets, lo, hi, radii, palm_lo=None, palm_hi=None) -> Hand:
    F = len(bases_R)
    J = len(axes[0])
    base = np.zeros((F, 12), np.float64)
    for f in range(F):
        base[f, 0:3] = bases_R[f][0]
        base[f, 3] = bases_t[f][0]
        base[f, 4:7] = bases_R[f][1]
        base[f, 7] = bases_t[f][1]
        base[f, 8:11] = bases_R[f][2]
        base[f, 11] = bases_t[f][2]
    sp, sn, sl = [], [], []
    for f in range(F):
        p, n, l = _capsule_surface(np.asarray(offsets[f]), np.asarray(radii[f]))
        sp.append(p)
        sn.append(n)
        sl.append(l)
    M = len(sp[0])
    assert all(len(x) == M for x in sp)
    g = np.mean(np.asarray(bases_t, np.float64), axis=0)
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    return Hand(name=name, base=f32(base), axis=f32(axes), offset=f32(offsets),
                lo=f32(lo), hi=f32(hi), radius=f32(radii),
                surf_p=f32(sp), surf_n=f32(sn),
                surf_link=np.ascontiguousarray(np.asarray(sl, np.int32)),
                grasp_centre=g,
                palm_lo=None if palm_lo is None else np.asarray(palm_lo, np.float32),
                palm_hi=None if palm_hi is None else np.asarray(palm_hi, np.float32))


def hand_three_finger(base_radius: float = 0.06) -> Hand:
    """3 fingers x 3 flexion joints (links 0.04/0.03/0.025 m, radius 8 mm,
    limits [0, 1.6] rad).  Finger f's base sits on the palm (z = 0) at
    ``base_radius`` from the palm axis, azimuth 2*pi*f/3, pointing along the
    palm normal +z; all joints flex about the tangential axis so that the
    finger curls toward the palm axis.  With bases at 0.04 m the fingers can
    only touch the underside of a 0.04 m sphere placed 0.08-0.12 m above the
    palm (no force-closed tuple exists); 0.06 m lets them reach its sides."""
    F, J = 3, 3
    lens = [0.04, 0.03, 0.025]
    R, t, ax, off, lo, hi, rad = [], [], [], [], [], [], []
    for f in range(F):
        phi = 2.0 * math.pi * f / F
        R.append(_rot_z(phi))
        t.append(np.array([base_radius * math.cos(phi), base_radius * math.sin(phi), 0.0]))
        ax.append([[0.0, -1.0, 0.0]] * J)
        off.append([[0.0, 0.0, l] for l in lens])
        lo.append([0.0] * J)
        hi.append([1.6] * J)
        rad.append([0.008] * J)
    # palm: a 15 mm slab under the bases, reaching the finger bases' circle
    r = base_radius
    return _pack_hand("three_finger_9dof", R, t, ax, off, lo, hi, rad, palm_lo=[-r, -r, -0.015], palm_hi=[r, r, 0.0])


def hand_anthropomorphic(n_fingers: int) -> Hand:
    """(n_fingers-1) parallel fingers plus a thumb, 4 revolute joints each.

    Joint 0 abducts about the palm normal (limits [-0.35, 0.35] rad) and has a
    zero-length link; joints 1..3 flex (limits [0, 1.6] rad) with links
    0.054/0.038/0.044 m and capsule radius 9 mm.  Fingers lie along +y from
    bases on the palm edge (x spacing 0.045 m) and flex toward +z; the thumb's
    base is rotated 90 degrees about the palm normal and sits on the palm side.
    """
    F, J = n_fingers, 4
    lens = [0.0, 0.054, 0.038, 0.044]
    R, t, ax, off, lo, hi, rad = [], [], [], [], [], [], []
    nf = F - 1
    for i in range(nf):
        x = (i - (nf - 1) / 2.0) * 0.045
        R.append(np.eye(3))
        t.append(np.array([x, 0.045, 0.0]))
    R.append(_rot_z(math.pi / 2.0))
    t.append(np.array([(nf / 2.0) * 0.045 + 0.02, -0.035, 0.0]))
    for f in range(F):
        ax.append([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
        off.append([[0.0, l, 0.0] for l in lens])
        lo.append([-0.35, 0.0, 0.0, 0.0])
        hi.append([0.35, 1.6, 1.6, 1.6])
        rad.append([0.0, 0.009, 0.009, 0.009])
    # palm: a 20 mm slab from the thumb side (y = -0.05) to the finger bases (y = 0.045), 25 mm past the
    # outer fingers
    xr = ((nf - 1) / 2.0) * 0.045 + 0.025
    return _pack_hand(f"anthropomorphic_{F}f_{F * J}dof", R, t, ax, off, lo, hi, rad,
                      palm_lo=[-xr, -0.05, -0.02], palm_hi=[xr, 0.045, 0.0])


def joint_samples(hand: Hand, S: int, seed: int) -> np.ndarray:
    """i.i.d. uniform joint configurations inside the limits, float32 [F,J,S]
    (Sec. 4.3: the field is approximated by randomly sampled configurations)."""
    rng = np.random.default_rng(seed)
    u = rng.random((hand.F, hand.J, S))
    lo = hand.lo.astype(np.float64)[:, :, None]
    hi = hand.hi.astype(np.float64)[:, :, None]
    return np.ascontiguousarray((lo + u * (hi - lo)).astype(np.float32))


# ---------------------------------------------------------------------------
# objects: surface points + outward unit normals (object frame), Morton-sorted
# ---------------------------------------------------------------------------

@dataclass
class Obj:
    name: str
    p: np.ndarray          # [N,3] float32 surface points
    n: np.ndarray          # [N,3] float32 outward unit normals
    centroid: np.ndarray   # [3] float32: mean of the points (torque reference)
    rho: float             # float32 value: max distance of a point to the centroid

    @property
    def N(self) -> int:
        return int(self.p.shape[0])

    def soa(self) -> np.ndarray:
        """[6,N] float32: px, py, pz, nx, ny, nz rows."""
        return np.ascontiguousarray(np.concatenate([self.p.T, self.n.T], axis=0))


def _morton_order(p: np.ndarray) -> np.ndarray:
    lo = p.min(axis=0)
    ext = np.maximum(p.max(axis=0) - lo, 1e-12)
    q = np.clip(((p - lo) / ext * 1023.0).astype(np.int64), 0, 1023)

    def spread(v):
        v = v & 0x3FF
        v = (v | (v << 16)) & 0x030000FF
        v = (v | (v << 8)) & 0x0300F00F
        v = (v | (v << 4)) & 0x030C30C3
        v = (v | (v << 2)) & 0x09249249
        return v

    code = spread(q[:, 0]) | (spread(q[:, 1]) << 1) | (spread(q[:, 2]) << 2)
    return np.argsort(code, kind="stable")


def _finish(name: str, p64: np.ndarray, n64: np.ndarray) -> Obj:
    n64 = n64 / np.linalg.norm(n64, axis=1, keepdims=True)
    order = _morton_order(p64)
    p = np.ascontiguousarray(p64[order].astype(np.float32))
    n = np.ascontiguousarray(n64[order].astype(np.float32))
    c64 = p.astype(np.float64).mean(axis=0)
    c = c64.astype(np.float32)
    rho = float(np.float32(np.max(np.linalg.norm(p.astype(np.float64) - c.astype(np.float64), axis=1))))
    return Obj(name=name, p=p, n=n, centroid=c, rho=rho)


def sphere(N: int, r: float, seed: int) -> Obj:
    """Area-uniform points on a sphere of radius r (normalised Gaussians)."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((N, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return _finish(f"sphere_r{r}", r * u, u.copy())


def _sgnpow(x, e):
    return np.sign(x) * np.abs(x) ** e


def superquadric(N: int, seed: int) -> Obj:
    """Superquadric with axes ~U[0.03,0.08] m and exponents ~U[0.3,1.5].

    Area-uniform by oversampling the (eta, omega) parameterisation 16x and
    resampling proportionally to |dx/deta x dx/domega| (finite differences);
    normals from the dual-superquadric closed form (Barr 1981)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.03, 0.08, 3)
    e1, e2 = rng.uniform(0.3, 1.5, 2)
    K = 16 * N
    eta = rng.uniform(-math.pi / 2, math.pi / 2, K)
    om = rng.uniform(-math.pi, math.pi, K)

    def X(et, o):
        ce, se = _sgnpow(np.cos(et), e1), _sgnpow(np.sin(et), e1)
        return np.stack([a[0] * ce * _sgnpow(np.cos(o), e2),
                         a[1] * ce * _sgnpow(np.sin(o), e2),
                         a[2] * se], axis=1)

    hstep = 1e-5
    de = (X(eta + hstep, om) - X(eta - hstep, om)) / (2 * hstep)
    do = (X(eta, om + hstep) - X(eta, om - hstep)) / (2 * hstep)
    w = np.linalg.norm(np.cross(de, do), axis=1)
    w = np.nan_to_num(w, nan=0.0, posinf=0.0)
    w /= w.sum()
    idx = rng.choice(K, size=N, replace=True, p=w)
    et, o = eta[idx], om[idx]
    p = X(et, o)
    ce2, se2 = _sgnpow(np.cos(et), 2 - e1), _sgnpow(np.sin(et), 2 - e1)
    n = np.stack([ce2 * _sgnpow(np.cos(o), 2 - e2) / a[0],
                  ce2 * _sgnpow(np.sin(o), 2 - e2) / a[1],
                  se2 / a[2]], axis=1)
    bad = ~np.isfinite(n).all(axis=1) | (np.linalg.norm(n, axis=1) < 1e-12)
    n[bad] = p[bad]  # degenerate parameter corners: fall back to the radial direction
    return _finish(f"superquadric_s{seed}", p, n)


def _rand_rot(rng, max_angle: float) -> np.ndarray:
    ax = rng.standard_normal(3)
    ax /= np.linalg.norm(ax)
    ang = rng.uniform(-max_angle, max_angle)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


def tool_composite(N: int, seed: int) -> Obj:
    """Irregular tool: cylinder handle (r=0.012, length 0.15) along x, a box
    head 0.06x0.03x0.02 at one end and a torus (R=0.03, r=0.006) at the other,
    head and torus at seeded rigid poses.  Area-weighted sampling per primitive;
    points inside another primitive are dropped; resampled to exactly N."""
    rng = np.random.default_rng(seed)
    # primitive poses (object frame)
    Rh = _rand_rot(rng, 0.3)
    th = np.array([0.075 + 0.012, 0.0, 0.0]) + rng.uniform(-0.004, 0.004, 3)
    hb = np.array([0.02, 0.06, 0.03]) / 2.0  # head half-extents (x thin, y long)
    Rt = _rand_rot(rng, 0.4)
    tt = np.array([-0.075 - 0.03, 0.0, 0.0]) + rng.uniform(-0.004, 0.004, 3)
    Rr, rr = 0.03, 0.006
    rc, L = 0.012, 0.15

    def in_cyl(x):
        return (np.abs(x[:, 0]) <= L / 2) & (x[:, 1] ** 2 + x[:, 2] ** 2 <= rc * rc)

    def in_box(x):
        y = (x - th) @ Rh
        return np.all(np.abs(y) <= hb, axis=1)

    def in_torus(x):
        y = (x - tt) @ Rt
        q = np.sqrt(y[:, 0] ** 2 + y[:, 1] ** 2) - Rr
        return q * q + y[:, 2] ** 2 <= rr * rr

    K = 4 * N
    # areas
    A_cyl_side = 2 * math.pi * rc * L
    A_cap = math.pi * rc * rc
    A_box = 8 * (hb[0] * hb[1] + hb[1] * hb[2] + hb[0] * hb[2])
    A_tor = 4 * math.pi ** 2 * Rr * rr
    areas = np.array([A_cyl_side, 2 * A_cap, A_box, A_tor])
    counts = np.maximum(1, np.round(K * areas / areas.sum()).astype(int))
    P, Nn, src = [], [], []
    # cylinder side
    c = counts[0]
    x = rng.uniform(-L / 2, L / 2, c)
    a = rng.uniform(0, 2 * math.pi, c)
    P.append(np.stack([x, rc * np.cos(a), rc * np.sin(a)], 1))
    Nn.append(np.stack([np.zeros(c), np.cos(a), np.sin(a)], 1))
    src.append(np.zeros(c, int))
    # caps
    c = counts[1]
    rr2 = rc * np.sqrt(rng.random(c))
    a = rng.uniform(0, 2 * math.pi, c)
    side = np.where(rng.random(c) < 0.5, -1.0, 1.0)
    P.append(np.stack([side * L / 2, rr2 * np.cos(a), rr2 * np.sin(a)], 1))
    Nn.append(np.stack([side, np.zeros(c), np.zeros(c)], 1))
    src.append(np.zeros(c, int))
    # box faces (area-weighted face choice)
    c = counts[2]
    fa = np.array([hb[1] * hb[2], hb[1] * hb[2], hb[0] * hb[2], hb[0] * hb[2], hb[0] * hb[1], hb[0] * hb[1]])
    face = rng.choice(6, size=c, p=fa / fa.sum())
    y = rng.uniform(-1, 1, (c, 3)) * hb
    nrm = np.zeros((c, 3))
    for fi in range(6):
        m = face == fi
        axi, sg = fi // 2, (1.0 if fi % 2 == 0 else -1.0)
        y[m, axi] = sg * hb[axi]
        nrm[m, axi] = sg
    P.append(y @ Rh.T + th)
    Nn.append(nrm @ Rh.T)
    src.append(np.ones(c, int))
    # torus (area element proportional to R + r cos v)
    c = counts[3]
    u = rng.uniform(0, 2 * math.pi, 4 * c)
    v = rng.uniform(0, 2 * math.pi, 4 * c)
    keep = rng.random(4 * c) < (Rr + rr * np.cos(v)) / (Rr + rr)
    u, v = u[keep][:c], v[keep][:c]
    y = np.stack([(Rr + rr * np.cos(v)) * np.cos(u), (Rr + rr * np.cos(v)) * np.sin(u), rr * np.sin(v)], 1)
    nrm = np.stack([np.cos(v) * np.cos(u), np.cos(v) * np.sin(u), np.sin(v)], 1)
    P.append(y @ Rt.T + tt)
    Nn.append(nrm @ Rt.T)
    src.append(np.full(len(u), 2))
    P, Nn, src = np.concatenate(P), np.concatenate(Nn), np.concatenate(src)
    # drop points strictly inside another primitive
    eps = 1e-9
    inside = np.zeros(len(P), bool)
    sh = P - Nn * eps  # nudge inward off the own surface
    sh_out = P + Nn * eps
    inside |= (src != 0) & in_cyl(sh_out)
    inside |= (src != 1) & in_box(sh_out)
    inside |= (src != 2) & in_torus(sh_out)
    del sh
    P, Nn = P[~inside], Nn[~inside]
    sel = rng.choice(len(P), size=N, replace=len(P) < N)
    return _finish(f"tool_composite_s{seed}", P[sel], Nn[sel])


# ---------------------------------------------------------------------------
# palm poses: uniform SO(3) (Shoemake 1992) x offset along the palm normal
# ---------------------------------------------------------------------------

def palm_poses(P: int, seed: int, grasp_centre: np.ndarray, obj_centroid: np.ndarray,
               d_lo: float = 0.08, d_hi: float = 0.12) -> np.ndarray:
    """[P,12] float32 object->palm rigid transforms, row-major 3x4 (R | t).

    Canonical placement (Sec. 5.2): the object centroid goes to
    grasp_centre + d * z_palm, d ~ U[d_lo, d_hi], with a uniformly random
    rotation about the centroid."""
    rng = np.random.default_rng(seed)
    u1, u2, u3 = rng.random(P), rng.random(P), rng.random(P)
    a = np.sqrt(1 - u1)
    b = np.sqrt(u1)
    qx, qy = a * np.sin(2 * math.pi * u2), a * np.cos(2 * math.pi * u2)
    qz, qw = b * np.sin(2 * math.pi * u3), b * np.cos(2 * math.pi * u3)
    R = np.empty((P, 3, 3))
    R[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz)
    R[:, 0, 1] = 2 * (qx * qy - qz * qw)
    R[:, 0, 2] = 2 * (qx * qz + qy * qw)
    R[:, 1, 0] = 2 * (qx * qy + qz * qw)
    R[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz)
    R[:, 1, 2] = 2 * (qy * qz - qx * qw)
    R[:, 2, 0] = 2 * (qx * qz - qy * qw)
    R[:, 2, 1] = 2 * (qy * qz + qx * qw)
    R[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    d = rng.uniform(d_lo, d_hi, P)
    target = np.asarray(grasp_centre, np.float64)[None, :] + d[:, None] * np.array([0.0, 0.0, 1.0])[None, :]
    c = np.asarray(obj_centroid, np.float64)
    t = target - np.einsum("pij,j->pi", R, c)
    out = np.concatenate([R, t[:, :, None]], axis=2).reshape(P, 12)
    return np.ascontiguousarray(out.astype(np.float32))


# ---------------------------------------------------------------------------
# named workloads (the paper's scenarios, synthetic stand-ins)
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    hand: Hand
    obj: Obj
    q: np.ndarray          # [F,J,S] float32 joint samples
    h: float               # voxel edge (m)
    inv_h: np.float32      # FP32 inverse voxel edge: cells are floor(x * inv_h)
    bins: np.ndarray       # [B,3] float32 normal-bin directions
    poses: np.ndarray      # [P,12] float32
    T: int                 # tuples per pose
    k: int                 # contacts per tuple
    mu: float              # friction coefficient
    K: int                 # friction-pyramid edges
    eps: float             # closure threshold on the margin
    seed: int              # tuple-sampling key
    meta: dict = field(default_factory=dict)

    @property
    def S(self) -> int:
        return int(self.q.shape[2])

    @property
    def B(self) -> int:
        return int(self.bins.shape[0])

    @property
    def P(self) -> int:
        return int(self.poses.shape[0])


WORKLOADS = {
    # tiny: 3-finger 9-DOF hand, sphere
    "tiny_sphere": dict(hand="three", obj="sphere", N=2048, S=4096, h=0.005, B=8,
                        P=256, T=16, mu=0.5, K=8, k=3),
    # 4-finger 16-DOF hand, superquadric
    "hand16_superquadric": dict(hand="anthro4", obj="superquadric", N=16384, S=65536,
                                h=0.0025, B=16, P=8192, T=64, mu=0.5, K=8, k=3),
    # 5-finger 20-DOF hand, irregular tool
    "hand20_tool": dict(hand="anthro5", obj="tool", N=65536, S=131072, h=0.002, B=32,
                        P=32768, T=128, mu=0.4, K=8, k=3),
}


def _make_hand(kind: str) -> Hand:
    if kind == "three":
        return hand_three_finger()
    if kind == "anthro4":
        return hand_anthropomorphic(4)
    if kind == "anthro5":
        return hand_anthropomorphic(5)
    raise ValueError(kind)


def _make_obj(kind: str, N: int, seed: int) -> Obj:
    if kind == "sphere":
        return sphere(N, 0.04, seed)
    if kind == "superquadric":
        return superquadric(N, seed)
    if kind == "tool":
        return tool_composite(N, seed)
    raise ValueError(kind)


def batch_objects(n: int, seed: int = 0, n_range=(2048, 131072), p_range=(4096, 32768),
                  scale: float = 1.0):
    """The many-object batch: n objects, half superquadrics and half tool
    composites, point counts and pose counts log-uniform in the given ranges
    (times ``scale``), each with a hand drawn uniformly from the three hands.
    Returns a list of dicts (kind, hand key, N, P, obj seed, pose seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for o in range(n):
        lo, hi = np.log(n_range[0] * scale), np.log(n_range[1] * scale)
        N = int(max(32, round(np.exp(rng.uniform(lo, hi)))))
        P = int(max(8, round(np.exp(rng.uniform(np.log(p_range[0] * scale), np.log(p_range[1] * scale))))))
        hand = ["tiny_sphere", "hand16_superquadric", "hand20_tool"][int(rng.integers(3))]
        out.append(dict(kind="superquadric" if o % 2 == 0 else "tool", hand=hand, N=N, P=P,
                        obj_seed=1000 + o, pose_seed=seed * 7919 + o))
    return out


def batch_object_inputs(spec: dict, hand: Hand):
    """(Obj, poses) of one batch object."""
    obj = superquadric(spec["N"], spec["obj_seed"]) if spec["kind"] == "superquadric" else \
        tool_composite(spec["N"], spec["obj_seed"])
    return obj, palm_poses(spec["P"], spec["pose_seed"], hand.grasp_centre, obj.centroid)


def workload(name: str, *, P: int | None = None, N: int | None = None, S: int | None = None,
             T: int | None = None, seed: int = 0, obj_seed: int = 1000, eps: float = 1e-2) -> Workload:
    """Build a named workload; P/N/S/T override the sizes (for small parity cases)."""
    w = dict(WORKLOADS[name])
    if P is not None:
        w["P"] = P
    if N is not None:
        w["N"] = N
    if S is not None:
        w["S"] = S
    if T is not None:
        w["T"] = T
    hand = _make_hand(w["hand"])
    obj = _make_obj(w["obj"], w["N"], obj_seed)
    q = joint_samples(hand, w["S"], seed + 1)
    poses = palm_poses(w["P"], seed + 2, hand.grasp_centre, obj.centroid)
    inv_h = np.float32(1.0 / w["h"])
    return Workload(name=name, hand=hand, obj=obj, q=q, h=w["h"], inv_h=inv_h,
                    bins=fibonacci_dirs(w["B"]), poses=poses, T=w["T"], k=w["k"],
                    mu=w["mu"], K=w["K"], eps=eps, seed=seed,
                    meta=dict(w))
