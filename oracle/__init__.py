"""CPU oracle for the Contact-Field grasp path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct reference implementation that the GPU library is
checked against: C in ``cf_oracle.c`` for kinematics, field codes, masks and
sampling (FP64 geometry, OpenMP over independent poses), numpy for the wrench
construction, and a library LP solver (scipy's HiGHS) for the closure LPs, which
are written out exactly as defined.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the GPU library and never imports it.

Functions (paper passages they follow are cited in ``cf_oracle.c``):
  philox4x32_10       counter-based generator (Salmon et al., SC'11)
  fk_links            FP64 forward kinematics of one finger (Sec. 3.1)
  contact_vectors     FK((p,n); i, q) of all surface points of one finger sample
  Field               the sampled hand contact field as a set of codes
                      (Sec. 4.3, Alg. 1; Def. Contact Field (Hand))
  Field.query         contact domains as bitmasks (Sec. 4.2, Sec. 4.3 query)
  PatchFields         fine-grained field: one field per (finger, link) patch,
                      and the merge of a finger's patch domains (Sec. 4.4, 5.3)
  query_masks_brute   literal existential check, tiny inputs only
  sample_tuples       random k-tuples from k distinct finger domains (Sec. 5.3)
  closure_lp          linearised GSWO margin of one tuple (Eq. GSWO): k LPs
  score_tuples        margins / accept flags of many tuples (process pool)
  rep_codes           reverse-lookup representatives of a finger's codes (Sec. 5.5)
  point_codes         FP64 code of an object point under a pose (the query's decision)
  kinematics.*        FP64 numpy FK / Jacobian / DLS IK / SDF grid / realization
                      checks (Sec. 5.5, Sec. 5.6)

Precision: geometry and every integer decision (voxel cell, normal bin, and
from them field codes, masks, representatives and contact codes) are FP64.
Beside a decision the oracle can flag it as ambiguous when a perturbation of
at most tau = 1e-5 m of any coordinate involved, or 1e-6 in cosine on a bin
tie, could change it; those are the only entries where a correct FP32
implementation may decide otherwise.  The same codes decided in FP32
(``codes(f, "fp32")``, ``query(..., mask32=True)``) are diagnostics only.

Parity status: every function is pinned by tests under ``tests/`` against
closed forms, an independent library routine (triton's Philox in
CPU-interpreter mode), brute force (vertex enumeration of small LPs, literal
existential mask check) or invariants, except the items
listed as "parity unpinned" in the design notes (the value of the acceptance
threshold eps and the synthetic hand surface-point set, which the paper does not
fix).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from ctypes import POINTER, c_double, c_float, c_int, c_int32, c_int64, c_uint8, c_uint32, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cf_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

__all__ = ["build", "lib", "philox4x32_10", "fk_links", "contact_vectors", "Field", "PatchFields",
           "query_masks_brute", "sample_tuples", "closure_lp", "score_tuples", "num_threads", "pack_code",
           "rep_codes", "point_codes", "dilation_masks"]


def build(force: bool = False) -> str:
    """Compile cf_oracle.c into liborc.so (plain gcc, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        fp = POINTER(c_float)
        dp = POINTER(c_double)
        u32p = POINTER(c_uint32)
        i32p = POINTER(c_int32)
        u8p = POINTER(c_uint8)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_fk_links.argtypes = [c_int, fp, fp, fp, dp, dp, dp]
        L.orc_contact_vectors.argtypes = [c_int, c_int, fp, fp, fp, fp, fp, i32p, dp, fp, fp, dp, dp]
        L.orc_field_create.restype = c_void_p
        L.orc_field_create.argtypes = [c_int, c_int, c_int, fp, fp, fp, fp, fp, i32p, fp, c_int, c_float,
                                       c_int, fp, c_int, c_double, c_double]
        L.orc_field_free.argtypes = [c_void_p]
        L.orc_field_sizes.argtypes = [c_void_p, POINTER(c_int64)]
        L.orc_field_code_set.restype = c_int64
        L.orc_field_code_set.argtypes = [c_void_p, c_int, c_int, POINTER(c_uint64), c_int64]
        L.orc_query_masks.argtypes = [c_void_p, c_int, fp, c_int, fp, u32p, u32p, u8p, u32p]
        L.orc_query_masks_brute.argtypes = [c_int, c_int, c_int, fp, fp, fp, fp, fp, i32p, fp, c_int, c_float,
                                            c_int, fp, c_int, fp, c_int, fp, u32p, u32p]
        L.orc_field_set_dilation.argtypes = [c_void_p, u32p]
        L.orc_sample_tuples.argtypes = [c_int, c_int, c_int, u32p, u32p, c_int, c_int, c_uint64, i32p, u8p]
        L.orc_num_threads.restype = c_int
        L.orc_set_threads.argtypes = [c_int]
        L.orc_rep_codes.restype = c_int64
        L.orc_rep_codes.argtypes = [c_int, c_int, c_int, fp, fp, fp, fp, fp, i32p, fp, c_int, c_float, c_int, fp,
                                    c_int, c_double, c_double, POINTER(c_uint64), u32p, u8p, c_int64]
        L.orc_point_codes.argtypes = [c_int, fp, fp, c_int, i32p, i32p, c_float, c_int, fp, c_double, c_double,
                                      POINTER(c_int64), u8p]
        _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(POINTER(ct))


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c, c_uint32), _p(k, c_uint32), _p(out, c_uint32))
    return out


def fk_links(J: int, base12, axis, offset, q):
    """Link frames of one finger: (R [J,3,3], t [J,3]) in FP64."""
    b, a, o = _c(base12, np.float32), _c(axis, np.float32), _c(offset, np.float32)
    qq = _c(q, np.float64)
    R = np.zeros((J, 9))
    t = np.zeros((J, 3))
    lib().orc_fk_links(J, _p(b, c_float), _p(a, c_float), _p(o, c_float), _p(qq, c_double),
                       _p(R, c_double), _p(t, c_double))
    return R.reshape(J, 3, 3), t


def contact_vectors(hand, f: int, q):
    """Contact vectors of all M surface points of finger f at configuration q:
    (p32, n32, p64, n64) with shapes [M,3]."""
    J, M = hand.J, hand.M
    qq = _c(q, np.float64)
    p32 = np.zeros((M, 3), np.float32)
    n32 = np.zeros((M, 3), np.float32)
    p64 = np.zeros((M, 3))
    n64 = np.zeros((M, 3))
    b = _c(hand.base[f], np.float32)
    a = _c(hand.axis[f], np.float32)
    o = _c(hand.offset[f], np.float32)
    sp = _c(hand.surf_p[f], np.float32)
    sn = _c(hand.surf_n[f], np.float32)
    sl = _c(hand.surf_link[f], np.int32)
    lib().orc_contact_vectors(J, M, _p(b, c_float), _p(a, c_float), _p(o, c_float), _p(sp, c_float),
                              _p(sn, c_float), _p(sl, c_int32), _p(qq, c_double), _p(p32, c_float),
                              _p(n32, c_float), _p(p64, c_double), _p(n64, c_double))
    return p32, n32, p64, n64


def _hand_args(hand):
    arrs = [_c(hand.base, np.float32), _c(hand.axis, np.float32), _c(hand.offset, np.float32),
            _c(hand.surf_p, np.float32), _c(hand.surf_n, np.float32), _c(hand.surf_link, np.int32)]
    ptrs = [_p(arrs[0], c_float), _p(arrs[1], c_float), _p(arrs[2], c_float), _p(arrs[3], c_float),
            _p(arrs[4], c_float), _p(arrs[5], c_int32)]
    return arrs, ptrs


class Field:
    """The sampled contact field of a hand as per-finger sets of
    (cell, bin) codes.  ``band=True`` also keeps the FP64 / tolerance-band code
    sets used to flag ambiguous entries (tau metres, bin_tol in cosine)."""

    def __init__(self, hand, q: np.ndarray, inv_h, bins: np.ndarray, band: bool = False,
                 tau: float = 1e-5, bin_tol: float = 1e-6, dilate_deg=None):
        self.F, self.J, self.M = hand.F, hand.J, hand.M
        self.B = int(bins.shape[0])
        self.inv_h = np.float32(inv_h)
        keep, ptrs = _hand_args(hand)
        qq = _c(q, np.float32)
        self._bins = _c(bins, np.float32)
        S = int(qq.shape[2])
        self.band = bool(band)
        self._h = lib().orc_field_create(self.F, self.J, self.M, *ptrs, _p(qq, c_float), S, c_float(self.inv_h),
                                         self.B, _p(self._bins, c_float), int(band), tau, bin_tol)
        del keep
        self.dilation = dilation_masks(self._bins, dilate_deg) if dilate_deg is not None else None
        if self.dilation is not None:
            lib().orc_field_set_dilation(self._h, _p(self.dilation, c_uint32))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_field_free(h)
            self._h = None

    def n_codes(self) -> np.ndarray:
        out = np.zeros(self.F, np.int64)
        lib().orc_field_sizes(self._h, out.ctypes.data_as(POINTER(c_int64)))
        return out

    def codes(self, f: int, which: str = "fp64") -> np.ndarray:
        """Sorted distinct (kx, ky, kz, bin) codes of finger f, int64 [n,4].
        which: "fp64" (the oracle's decisions, which the acceptance tests use),
        "fp32" (the same codes decided in FP32: a diagnostic), "possible" (codes
        some sample takes somewhere in the tolerance band), "sure" (codes of
        samples whose code is the same everywhere in the band); the last three
        need band=True."""
        sel = {"fp32": 0, "fp64": 1, "possible": 2, "sure": 3}[which]
        n = int(lib().orc_field_code_set(self._h, f, sel, None, 0))
        if n < 0:
            raise ValueError(f"code set {which!r} needs Field(..., band=True)")
        raw = np.zeros(n, np.uint64)
        lib().orc_field_code_set(self._h, f, sel, raw.ctypes.data_as(POINTER(c_uint64)), n)
        off = 32768
        kx = ((raw >> np.uint64(40)) & np.uint64(0xFFFF)).astype(np.int64) - off
        ky = ((raw >> np.uint64(24)) & np.uint64(0xFFFF)).astype(np.int64) - off
        kz = ((raw >> np.uint64(8)) & np.uint64(0xFFFF)).astype(np.int64) - off
        b = (raw & np.uint64(0xFF)).astype(np.int64)
        return np.stack([kx, ky, kz, b], axis=1)

    def query(self, soa: np.ndarray, poses: np.ndarray, amb: bool = False, mask32: bool = False):
        """Domain masks [P,F,W] uint32 and counts [P,F] uint32, decided in FP64
        (plus optional ambiguity flags [P,F,N] uint8, which need band=True, and
        the FP32-decision masks [P,F,W] as a diagnostic)."""
        soa = _c(soa, np.float32)
        poses = _c(poses, np.float32).reshape(-1, 12)
        N = int(soa.shape[1])
        P = int(poses.shape[0])
        W = (N + 31) // 32
        masks = np.zeros((P, self.F, W), np.uint32)
        counts = np.zeros((P, self.F), np.uint32)
        a = np.zeros((P, self.F, N), np.uint8) if amb else None
        m32 = np.zeros((P, self.F, W), np.uint32) if mask32 else None
        if amb and not self.band:
            raise ValueError("ambiguity flags need Field(..., band=True)")
        lib().orc_query_masks(self._h, N, _p(soa, c_float), P, _p(poses, c_float), _p(masks, c_uint32),
                              _p(counts, c_uint32), _p(a, c_uint8) if a is not None else None,
                              _p(m32, c_uint32) if m32 is not None else None)
        out = [masks, counts]
        if amb:
            out.append(a)
        if mask32:
            out.append(m32)
        return tuple(out)


class _SubHand:
    """One finger of a hand restricted to the surface points of one link."""

    def __init__(self, hand, f: int, link: int):
        sel = np.asarray(hand.surf_link[f]) == link
        self.F, self.J, self.M = 1, hand.J, int(sel.sum())
        self.base = np.asarray(hand.base)[f:f + 1]
        self.axis = np.asarray(hand.axis)[f:f + 1]
        self.offset = np.asarray(hand.offset)[f:f + 1]
        self.surf_p = np.asarray(hand.surf_p)[f:f + 1, sel]
        self.surf_n = np.asarray(hand.surf_n)[f:f + 1, sel]
        self.surf_link = np.asarray(hand.surf_link)[f:f + 1, sel]


class PatchFields:
    """The fine-grained contact field of Sec. 4.4: the hand surface broken into
    patches, one field per patch, queried separately.  A patch is the surface
    points of one link of one finger; patches are ordered by finger, then link
    (ascending), skipping links without surface points.  Sec. 5.3 merges the
    domains of a dependency group (a finger): ``merge``."""

    def __init__(self, hand, q, inv_h, bins, band: bool = False, **kw):
        q = np.asarray(q, np.float32)
        self.F = hand.F
        self.slots = []  # (finger, link)
        self.fields = []
        for f in range(hand.F):
            for link in np.unique(np.asarray(hand.surf_link[f])).tolist():
                self.slots.append((f, int(link)))
                self.fields.append(Field(_SubHand(hand, f, link), q[f:f + 1], inv_h, bins, band=band, **kw))

    def codes(self, s: int, which: str = "fp64") -> np.ndarray:
        """Codes of slot s (as Field.codes of one finger)."""
        return self.fields[s].codes(0, which)

    def query(self, soa, poses, amb: bool = False):
        """Per-patch domains [P, n_slots, W] and counts [P, n_slots] (plus band flags [P, n_slots, N])."""
        outs = [fd.query(soa, poses, amb=amb) for fd in self.fields]
        masks = np.concatenate([o[0] for o in outs], axis=1)
        counts = np.concatenate([o[1] for o in outs], axis=1)
        if amb:
            return masks, counts, np.concatenate([o[2] for o in outs], axis=1)
        return masks, counts

    def merge(self, masks):
        """Sec. 5.3: OR of each finger's patch rows -> [P, F, W] and the counts [P, F]."""
        P, _, W = masks.shape
        out = np.zeros((P, self.F, W), np.uint32)
        for s, (f, _) in enumerate(self.slots):
            out[:, f] |= masks[:, s]
        counts = np.unpackbits(out.view(np.uint8), axis=2).sum(axis=2).astype(np.uint32)
        return out, counts


def dilation_masks(bins: np.ndarray, dilate_deg: float) -> np.ndarray:
    """Theta-dilated bins (the leaf test -x^T n >= theta_hit of Sec. 4.3): bit b'
    of entry b is set when d_b . d_b' >= cos(theta), theta = dilate_deg degrees
    (FP64 dot of the FP32 directions, x + y + z in that order); bit b always;
    theta = 0 keeps the same bin only."""
    d = np.asarray(bins, np.float32).astype(np.float64)
    B = d.shape[0]
    deg = float(np.float32(dilate_deg))
    c = math.cos(deg * (math.pi / 180.0))
    out = np.zeros(B, np.uint32)
    for b in range(B):
        m = 1 << b
        for b2 in range(B):
            dot = float(d[b, 0]) * float(d[b2, 0]) + float(d[b, 1]) * float(d[b2, 1]) + float(d[b, 2]) * float(d[b2, 2])
            if deg > 0.0 and dot >= c:
                m |= 1 << b2
        out[b] = m
    return out


def query_masks_brute(hand, q, inv_h, bins, soa, poses, dilate_deg=None) -> np.ndarray:
    keep, ptrs = _hand_args(hand)
    qq = _c(q, np.float32)
    bb = _c(bins, np.float32)
    soa = _c(soa, np.float32)
    poses = _c(poses, np.float32).reshape(-1, 12)
    N, P = int(soa.shape[1]), int(poses.shape[0])
    W = (N + 31) // 32
    masks = np.zeros((P, hand.F, W), np.uint32)
    dil = dilation_masks(bb, dilate_deg) if dilate_deg is not None else None
    lib().orc_query_masks_brute(hand.F, hand.J, hand.M, *ptrs, _p(qq, c_float), int(qq.shape[2]),
                                c_float(np.float32(inv_h)), int(bb.shape[0]), _p(bb, c_float), N,
                                _p(soa, c_float), P, _p(poses, c_float),
                                _p(dil, c_uint32) if dil is not None else None, _p(masks, c_uint32))
    del keep
    return masks


KEY_OFFSET = 32768


def pack_code(f, kx, ky, kz, b) -> int:
    """Packed (finger, cell, bin) key of the oracle's code sets."""
    o = KEY_OFFSET
    return (int(f) << 56) | ((int(kx) + o) << 40) | ((int(ky) + o) << 24) | ((int(kz) + o) << 8) | int(b)


def rep_codes(hand, q, inv_h, bins, f: int, with_sure: bool = False, tau: float = 1e-5, bin_tol: float = 1e-6):
    """Reverse lookup table of finger f (Sec. 5.5): packed FP64 code -> smallest
    s * M + m over the field samples producing it (m in the hand's order).
    with_sure: also the set of codes whose representative no perturbation
    within the band (tau metres, bin_tol in cosine) can change."""
    keep, ptrs = _hand_args(hand)
    qq = _c(q, np.float32)
    bb = _c(bins, np.float32)
    S = int(qq.shape[2])
    cap = S * hand.M
    keys = np.zeros(max(cap, 1), np.uint64)
    vals = np.zeros(max(cap, 1), np.uint32)
    sure = np.zeros(max(cap, 1), np.uint8) if with_sure else None
    n = lib().orc_rep_codes(hand.F, hand.J, hand.M, *ptrs, _p(qq, c_float), S, c_float(np.float32(inv_h)),
                            int(bb.shape[0]), _p(bb, c_float), int(f), float(tau), float(bin_tol),
                            keys.ctypes.data_as(POINTER(c_uint64)), _p(vals, c_uint32),
                            _p(sure, c_uint8) if sure is not None else None, cap)
    del keep
    rep = dict(zip(keys[:n].tolist(), vals[:n].tolist()))
    if not with_sure:
        return rep
    return rep, set(keys[:n][sure[:n].astype(bool)].tolist())


def point_codes(soa, poses, pose_idx, pt_idx, inv_h, bins, with_amb: bool = False, tau: float = 1e-5,
                bin_tol: float = 1e-6):
    """FP64 (kx, ky, kz, bin) of the contact-surface vector of points pt_idx
    under poses pose_idx, as the domain query decides it: int64 [n, 4]
    (with_amb: also uint8 [n] flags of codes that a perturbation within the
    band could change)."""
    soa = _c(soa, np.float32)
    poses = _c(poses, np.float32).reshape(-1, 12)
    pi = _c(pose_idx, np.int32).ravel()
    xi = _c(pt_idx, np.int32).ravel()
    bb = _c(bins, np.float32)
    out = np.zeros((pi.size, 4), np.int64)
    amb = np.zeros(pi.size, np.uint8)
    lib().orc_point_codes(int(soa.shape[1]), _p(soa, c_float), _p(poses, c_float), int(pi.size), _p(pi, c_int32),
                          _p(xi, c_int32), c_float(np.float32(inv_h)), int(bb.shape[0]), _p(bb, c_float),
                          float(tau), float(bin_tol), out.ctypes.data_as(POINTER(c_int64)), _p(amb, c_uint8))
    return (out, amb) if with_amb else out


def sample_tuples(masks: np.ndarray, counts: np.ndarray, N: int, T: int, k: int, seed: int):
    masks = _c(masks, np.uint32)
    counts = _c(counts, np.uint32)
    P, F = int(counts.shape[0]), int(counts.shape[1])
    tuples = np.zeros((P, T, k), np.int32)
    fingers = np.zeros((P, T, k), np.uint8)
    lib().orc_sample_tuples(P, F, N, _p(masks, c_uint32), _p(counts, c_uint32), T, k, c_uint64(seed),
                            _p(tuples, c_int32), _p(fingers, c_uint8))
    return tuples, fingers


# ---------------------------------------------------------------------------
# closure margin (Eq. GSWO, Sec. 3.2, linearised)
# ---------------------------------------------------------------------------

def _onb_duff(nu):
    """Tangent basis (x, y) of unit vector nu: Duff et al., "Building an
    Orthonormal Basis, Revisited" (JCGT 2017)."""
    s = math.copysign(1.0, nu[2])
    a = -1.0 / (s + nu[2])
    b = nu[0] * nu[1] * a
    x = np.array([1.0 + s * nu[0] * nu[0] * a, s * b, -s * nu[0]])
    y = np.array([b, s + nu[1] * nu[1] * a, -nu[1]])
    return x, y


def wrench_matrix(p, n, mu: float, K: int, c, rho: float) -> np.ndarray:
    """6 x kK matrix of pyramid-edge wrenches, column i*K + m:
    w_im = [e_im ; (p_i - c) x e_im / rho], e_im = nu_i + mu (cos th_m x_i +
    sin th_m y_i), th_m = 2 pi m / K, nu_i = -n_i (force into the object)."""
    p = np.asarray(p, np.float64).reshape(-1, 3)
    n = np.asarray(n, np.float64).reshape(-1, 3)
    c = np.asarray(c, np.float64)
    cols = []
    for i in range(p.shape[0]):
        nu = -n[i]
        x, y = _onb_duff(nu)
        r = p[i] - c
        for m in range(K):
            th = 2.0 * math.pi * m / K
            e = nu + mu * (math.cos(th) * x + math.sin(th) * y)
            cols.append(np.concatenate([e, np.cross(r, e) / rho]))
    return np.array(cols).T


def lp_subproblem(W: np.ndarray, K: int, j: int):
    """LP_j: minimise t over (c >= 0, t) subject to -t <= (W c)_r <= t for the
    six wrench rows and sum_m c_jm = 1.  Returns (t*, solver iterations)."""
    from scipy.optimize import linprog
    nc = W.shape[1]
    cost = np.zeros(nc + 1)
    cost[-1] = 1.0
    A = np.zeros((12, nc + 1))
    A[:6, :nc] = W
    A[6:, :nc] = -W
    A[:, nc] = -1.0
    Aeq = np.zeros((1, nc + 1))
    Aeq[0, j * K:(j + 1) * K] = 1.0
    res = linprog(cost, A_ub=A, b_ub=np.zeros(12), A_eq=Aeq, b_eq=[1.0], bounds=[(0, None)] * (nc + 1),
                  method="highs")
    if res.status != 0:
        return float("nan"), -1
    return float(res.fun), int(res.nit)


def closure_lp(p, n, mu: float, K: int, c, rho: float):
    """Margin t* = min_j LP_j of one tuple; returns (t*, t_per_j [k], iterations [k]).
    A failed subproblem makes t* NaN."""
    W = wrench_matrix(p, n, mu, K, c, rho)
    k = W.shape[1] // K
    tj = np.zeros(k)
    it = np.zeros(k, np.int32)
    for j in range(k):
        tj[j], it[j] = lp_subproblem(W, K, j)
    t = float("nan") if np.isnan(tj).any() else float(tj.min())
    return t, tj, it


def _score_chunk(args):
    soa, tuples, mu, K, c, rho, eps = args
    N = soa.shape[1]
    out_m = np.empty(len(tuples))
    out_it = np.zeros(len(tuples), np.int32)
    for u, ids in enumerate(tuples):
        if np.any(ids < 0) or np.any(ids >= N):
            out_m[u] = np.inf
            continue
        p = soa[0:3, ids].T.astype(np.float64)
        nn = soa[3:6, ids].T.astype(np.float64)
        t, _, it = closure_lp(p, nn, mu, K, c, rho)
        out_m[u] = t
        out_it[u] = int(it.sum())
    return out_m, out_it


_pool = None


def _get_pool():
    """Process pool started with 'spawn' (safe after CUDA initialisation)."""
    global _pool
    if _pool is None:
        import concurrent.futures
        import multiprocessing as mp
        _pool = concurrent.futures.ProcessPoolExecutor(max_workers=max(1, os.cpu_count() or 1),
                                                       mp_context=mp.get_context("spawn"))
    return _pool


def score_tuples(soa: np.ndarray, tuples: np.ndarray, mu: float, K: int, c, rho: float, eps: float,
                 workers: bool = True):
    """margins (float64, +inf for invalid tuples), accept (uint8: margin <= eps),
    solver iterations (int32) per tuple.  mu, c, rho, eps are taken at the FP32
    values the GPU receives."""
    soa = _c(soa, np.float32)
    tuples = _c(tuples, np.int32)
    k = int(tuples.shape[-1])
    flat = tuples.reshape(-1, k)
    mu64 = float(np.float32(mu))
    c64 = np.asarray(c, np.float32).astype(np.float64)
    rho64 = float(np.float32(rho))
    eps32 = float(np.float32(eps))
    n = flat.shape[0]
    if workers and n > 64:
        chunks = np.array_split(np.arange(n), max(1, min(n // 64, 4 * (os.cpu_count() or 1))))
        futs = [_get_pool().submit(_score_chunk, (soa, flat[ch], mu64, K, c64, rho64, eps32)) for ch in chunks]
        res = [f.result() for f in futs]
        margin = np.concatenate([r[0] for r in res])
        iters = np.concatenate([r[1] for r in res])
    else:
        margin, iters = _score_chunk((soa, flat, mu64, K, c64, rho64, eps32))
    accept = (margin <= eps32).astype(np.uint8)
    shp = tuples.shape[:-1]
    return margin.reshape(shp), accept.reshape(shp), iters.reshape(shp)
