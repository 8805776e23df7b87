"""Python binding of libcf, the B300 Contact-Field grasp hot path.

Argument marshalling only: every step runs in the CUDA kernels of ``libcf.so``
(see ``include/cf.h``).  PyTorch supplies device memory and the current CUDA
stream.  There is no CPU fallback: importing this package fails if the library
has not been built (``python paper_2511_07418_b300/build_lib.py``).

Entry points mirror the C ABI:
  build(hand, inv_h, bin_dirs, q)            -> Field          (cf_build)
  query_domains(field, soa, poses, ...)      -> masks, counts  (cf_query_domains)
  score_tuples(soa, n_fingers, masks, counts, params, ...)     (cf_score_tuples)
  Plan(n_fingers, n_max, p_max, params).run_host(field, ...)   (cf_plan_*)
  ik_dls(field, soa, poses, T, k, tuples, fingers, accept, params)  (cf_ik_dls)
  Sdf(soa, lo, h, dims); realize(field, sdf, poses, T, q, used, ...)  (cf_sdf_build, cf_realize)
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, byref, c_char_p, c_double, c_float, c_int, c_int32, c_int64, c_uint8, \
    c_uint32, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcf.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2511_07418_b300/build_lib.py` "
                      "(the CUDA library is required; there is no CPU path)")

_lib = ctypes.CDLL(LIB_PATH)

CF_MAX_FINGERS = 8
CF_MAX_SLOTS = 16
CF_MAX_BINS = 32
CF_OK = 0
CF_EINVAL = 1
CF_ENOMEM = 2
CF_ECUDA = 3
CF_ETIMEOUT = 4
CF_EBUSY = 5
CF_DEV_LP_PIVOT_CAP = 0x1
CF_DEV_LP_UNBOUNDED = 0x2
CF_DEV_REP_FULL = 0x4
CF_DEV_REP_MISS = 0x8


class CfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libcf error {code}: {msg}")
        self.code = code


class HandDesc(Structure):
    _fields_ = [("n_fingers", c_int32), ("n_joints", c_int32), ("n_surf", c_int32),
                ("base", POINTER(c_float)), ("axis", POINTER(c_float)), ("offset", POINTER(c_float)),
                ("surf_p", POINTER(c_float)), ("surf_n", POINTER(c_float)), ("surf_link", POINTER(c_int32)),
                ("lo", POINTER(c_float)), ("hi", POINTER(c_float)), ("radius", POINTER(c_float))]


class FieldParams(Structure):
    _fields_ = [("inv_h", c_float), ("n_bins", c_int32), ("bin_dirs", POINTER(c_float)), ("want_rep", c_int32),
                ("dilate_deg", c_float), ("patches", c_int32)]


class IkParams(Structure):
    _fields_ = [("beta", c_float), ("lambda_", c_float), ("n_phase1", c_int32), ("n_rounds", c_int32),
                ("n_phase2", c_int32), ("tol_pos", c_float), ("tol_cos", c_float)]


class OptParams(Structure):
    _fields_ = [("n_outer", c_int32), ("n_inner", c_int32), ("sigma", c_float), ("zero_tol", c_float),
                ("min_gain", c_float), ("warm_start", c_int32)]


class Tuning(Structure):
    _fields_ = [("query_poses_per_block", c_int32), ("score_refill", c_int32),
                ("score_blocks_per_sm", c_int32)]


class PlaceParams(Structure):
    _fields_ = [("exhaustive", c_int32), ("centroid", c_float * 3), ("g", c_float * 3), ("up", c_float * 3),
                ("d_lo", c_float), ("d_hi", c_float), ("seed", c_uint64), ("pose_base", c_uint32)]


class RealizeParams(Structure):
    _fields_ = [("pen_margin", c_float), ("axis_step", c_float), ("seed", c_uint64)]


class PalmDesc(Structure):
    _fields_ = [("lo", c_float * 3), ("hi", c_float * 3)]


class FieldInfo(Structure):
    _fields_ = [("n_fingers", c_int32), ("n_joints", c_int32), ("n_surf", c_int32), ("n_bins", c_int32),
                ("n_samples", c_int32), ("inv_h", c_float),
                ("box_lo", c_int32 * 3), ("box_dims", c_int32 * 3), ("bits_per_finger", c_int32),
                ("fingers_per_word", c_int32), ("record_words", c_int32),
                ("finger_lo", (c_int32 * 3) * CF_MAX_FINGERS), ("finger_dims", (c_int32 * 3) * CF_MAX_FINGERS),
                ("table_words", c_int64), ("device_bytes", c_int64), ("build_ms", c_float), ("dilate_deg", c_float),
                ("dilation", c_uint32 * CF_MAX_BINS), ("n_slots", c_int32), ("slot_finger", c_int32 * CF_MAX_SLOTS),
                ("slot_link", c_int32 * CF_MAX_SLOTS)]


class Points(Structure):
    _fields_ = [("px", c_void_p), ("py", c_void_p), ("pz", c_void_p), ("nx", c_void_p), ("ny", c_void_p),
                ("nz", c_void_p), ("n", c_int32)]


class ScoreParams(Structure):
    _fields_ = [("n_tuples", c_int32), ("k", c_int32), ("n_edges", c_int32), ("mu", c_float), ("eps", c_float),
                ("centroid", c_float * 3), ("rho", c_float), ("seed", c_uint64), ("tuples_given", c_int32)]


class BatchItem(Structure):
    _fields_ = [("field", c_void_p), ("obj", Points), ("d_poses", c_void_p), ("n_poses", c_int32),
                ("prm", ScoreParams), ("d_masks", c_void_p), ("d_counts", c_void_p), ("d_tuples", c_void_p),
                ("d_fingers", c_void_p), ("d_margin", c_void_p), ("d_accept", c_void_p)]


class EngineParams(Structure):
    _fields_ = [("fields", POINTER(c_void_p)), ("n_fields", c_int32), ("hbm_budget_bytes", c_int64),
                ("max_active", c_int32), ("pose_chunk", c_int32), ("pose_cap", c_int32),
                ("pose_chunk_max", c_int32), ("chunk_pairs_max", c_int64), ("reserve_bytes", c_int64)]


class Request(Structure):
    _fields_ = [("field", c_int32), ("h_soa", c_void_p), ("n", c_int32), ("h_poses", c_void_p), ("n_poses", c_int32),
                ("prm", ScoreParams), ("n_grasps", c_int32), ("tag", c_uint64)]


class Result(Structure):
    _fields_ = [("id", c_uint64), ("tag", c_uint64), ("status", c_int32), ("partial", c_int32), ("k", c_int32),
                ("n_accepted", c_int32), ("n_poses_used", c_int32), ("t_submit", c_double), ("t_admit", c_double),
                ("t_done", c_double), ("pose", POINTER(c_int32)), ("tuples", POINTER(c_int32)),
                ("margin", POINTER(c_float)), ("n_rounds", c_int32), ("t_first_round", c_double)]


class EngineStats(Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("rounds", c_int64), ("launches", c_int64),
                ("queued", c_int32), ("active", c_int32), ("bytes_in_use", c_int64), ("peak_bytes_in_use", c_int64),
                ("peak_active", c_int32), ("admit_s", c_double), ("round_host_s", c_double),
                ("round_wait_s", c_double)]


def _sig(name, args, res=c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_cf_build = _sig("cf_build", [POINTER(HandDesc), POINTER(FieldParams), c_void_p, c_int32, c_void_p, POINTER(c_void_p)])
_cf_field_get_info = _sig("cf_field_get_info", [c_void_p, POINTER(FieldInfo)])
_cf_field_copy_table = _sig("cf_field_copy_table", [c_void_p, POINTER(c_uint32), c_int64])
_cf_field_destroy = _sig("cf_field_destroy", [c_void_p])
_cf_field_save = _sig("cf_field_save", [c_void_p, c_char_p])
_cf_field_load = _sig("cf_field_load", [c_char_p, POINTER(c_void_p)])
_cf_query = _sig("cf_query_domains", [c_void_p, POINTER(Points), c_void_p, c_int32, c_void_p, c_void_p, c_void_p])
_cf_score = _sig("cf_score_tuples", [POINTER(Points), c_int32, c_void_p, c_void_p, c_int32, POINTER(ScoreParams),
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p])
_cf_sample = _sig("cf_sample_tuples", [POINTER(Points), c_int32, c_void_p, c_void_p, c_int32, POINTER(ScoreParams),
                                       c_void_p, c_void_p, c_void_p])
_cf_score_noalloc = _sig("cf_score_tuples_noalloc", [POINTER(Points), c_int32, c_void_p, c_void_p, c_int32,
                                                     POINTER(ScoreParams), c_void_p, c_void_p, c_void_p, c_void_p,
                                                     c_void_p])
_cf_batch_create = _sig("cf_batch_create", [POINTER(BatchItem), c_int32, POINTER(c_void_p)])
_cf_batch_run = _sig("cf_batch_run", [c_void_p, c_void_p])
_cf_batch_launches = _sig("cf_batch_launches", [c_void_p, POINTER(c_int32), POINTER(c_int32)])
_cf_batch_destroy = _sig("cf_batch_destroy", [c_void_p])
_cf_engine_create = _sig("cf_engine_create", [POINTER(EngineParams), POINTER(c_void_p)])
_cf_engine_submit = _sig("cf_engine_submit", [c_void_p, POINTER(Request), POINTER(c_uint64)])
_cf_engine_poll = _sig("cf_engine_poll", [c_void_p, POINTER(Result), c_int32, POINTER(c_int32)])
_cf_engine_result_free = _sig("cf_engine_result_free", [POINTER(Result)])
_cf_engine_get_stats = _sig("cf_engine_get_stats", [c_void_p, POINTER(EngineStats)])
_cf_engine_drain = _sig("cf_engine_drain", [c_void_p, c_int32])
_cf_engine_destroy = _sig("cf_engine_destroy", [c_void_p])
_cf_plan_create = _sig("cf_plan_create", [c_int32, c_int32, c_int32, POINTER(ScoreParams), POINTER(c_void_p)])
_cf_plan_run_host = _sig("cf_plan_run_host", [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_int32,
                                              POINTER(ScoreParams), c_void_p, c_void_p, c_void_p, POINTER(c_int64),
                                              c_void_p])
_cf_plan_run_host_accepted = _sig("cf_plan_run_host_accepted", [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_int32,
                                                                POINTER(ScoreParams), c_void_p, c_int64,
                                                                POINTER(c_int64), c_void_p])
_cf_plan_destroy = _sig("cf_plan_destroy", [c_void_p])
_cf_field_rep_slots = _sig("cf_field_rep_slots", [c_void_p, POINTER(c_int64)])
_cf_field_copy_rep = _sig("cf_field_copy_rep", [c_void_p, POINTER(c_uint64), POINTER(c_uint32), c_int64])
_cf_ik_dls = _sig("cf_ik_dls", [c_void_p, POINTER(Points), c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p,
                                c_void_p, POINTER(IkParams), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_void_p])
_cf_sdf_build = _sig("cf_sdf_build", [POINTER(Points), POINTER(c_float), c_float, POINTER(c_int32), c_void_p,
                                      POINTER(c_void_p)])
_cf_sdf_copy = _sig("cf_sdf_copy", [c_void_p, POINTER(c_float), c_int64])
_cf_sdf_destroy = _sig("cf_sdf_destroy", [c_void_p])
_cf_realize = _sig("cf_realize", [c_void_p, c_void_p, c_void_p, c_int32, c_int32, POINTER(RealizeParams), c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_void_p, c_void_p])
_cf_fp32_peak = _sig("cf_fp32_peak", [POINTER(c_double)])
_cf_place = _sig("cf_place", [c_void_p, POINTER(Points), c_int32, POINTER(PlaceParams), c_void_p, c_void_p])
_cf_concave = _sig("cf_concave_filter", [POINTER(Points), c_void_p, c_float, c_float, c_void_p, c_void_p, c_void_p,
                                         c_void_p])
_cf_get_tuning = _sig("cf_get_tuning", [POINTER(Tuning)])
_cf_set_tuning = _sig("cf_set_tuning", [POINTER(Tuning)])
_cf_autotune = _sig("cf_autotune", [POINTER(BatchItem), c_int32, c_int32, POINTER(Tuning), POINTER(c_double)])
_cf_gswo = _sig("cf_score_gswo", [POINTER(Points), c_int32, POINTER(ScoreParams), c_int32, c_float, c_void_p, c_void_p,
                                  c_void_p, c_void_p])
_cf_optimize = _sig("cf_optimize_tuples", [POINTER(Points), c_int32, c_void_p, c_int32, POINTER(ScoreParams),
                                           POINTER(OptParams), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p])
_cf_last_error = _sig("cf_last_error", [], c_char_p)
_cf_device_status = _sig("cf_device_status", [POINTER(c_uint32)])
_cf_device_counters = _sig("cf_device_counters", [POINTER(c_uint64), c_int])
_cf_pool_usage = _sig("cf_pool_usage", [POINTER(c_uint64), c_int])
_cf_sdf_box = _sig("cf_sdf_box", [POINTER(c_float), c_int32, c_float, c_float, POINTER(c_float), POINTER(c_int32)])
_cf_merge = _sig("cf_merge_domains", [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p])
_cf_place_static = _sig("cf_place_static", [POINTER(PalmDesc), POINTER(Points), c_int32, c_uint64, c_uint32, c_float,
                                            c_void_p, c_void_p, c_void_p, c_void_p])
_cf_append = _sig("cf_append_contact", [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p])

EXPORTED = ["cf_build", "cf_field_get_info", "cf_field_copy_table", "cf_field_destroy", "cf_field_save",
            "cf_field_load", "cf_query_domains", "cf_score_tuples", "cf_plan_create", "cf_plan_run_host",
            "cf_plan_run_host_accepted", "cf_plan_destroy", "cf_last_error", "cf_device_status", "cf_device_counters", "cf_pool_usage", "cf_sdf_box", "cf_merge_domains", "cf_place_static", "cf_append_contact", "cf_score_tuples_noalloc",
            "cf_sample_tuples", "cf_batch_create", "cf_batch_run", "cf_batch_launches", "cf_batch_destroy",
            "cf_engine_create", "cf_engine_submit", "cf_engine_poll", "cf_engine_result_free", "cf_engine_get_stats",
            "cf_engine_drain", "cf_engine_destroy", "cf_field_rep_slots", "cf_field_copy_rep", "cf_ik_dls",
            "cf_sdf_build", "cf_sdf_copy", "cf_sdf_destroy", "cf_realize", "cf_fp32_peak", "cf_optimize_tuples", "cf_score_gswo",
            "cf_get_tuning", "cf_set_tuning", "cf_autotune", "cf_place", "cf_concave_filter"]


def _check(rc: int):
    if rc != CF_OK:
        raise CfError(rc, _cf_last_error().decode(errors="replace"))


def _np(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _fp(a):
    return a.ctypes.data_as(POINTER(c_float))


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return c_void_p(t.data_ptr())


def points_struct(soa):
    """cf_points view of a contiguous [6, N] float32 CUDA tensor (px..nz rows)."""
    import torch
    _dev(soa, torch.float32, "soa")
    if soa.dim() != 2 or soa.shape[0] != 6:
        raise ValueError("soa must be [6, N]")
    n = int(soa.shape[1])
    base = soa.data_ptr()
    step = 4 * n
    return Points(*[c_void_p(base + r * step) for r in range(6)], n)


def _check_score_shapes(soa, n_fingers, masks, counts, prm, P, tuples=None, fingers=None, margin=None, accept=None):
    """Shapes and devices of the scoring calls' tensors, checked before any
    launch: the C side receives bare pointers and cannot see an undersized
    buffer, which the kernels would overrun."""
    T, k = int(prm.n_tuples), int(prm.k)
    if soa.dim() != 2 or soa.shape[0] != 6:
        raise ValueError("soa must be [6, N]")
    N = int(soa.shape[1])
    W = (N + 31) // 32
    want = {"tuples": (P, T, k), "fingers": (P, T, k), "margin": (P, T), "accept": (P, T)}
    if not prm.tuples_given:
        F = int(n_fingers)
        want["counts"] = (P, F)
        want["masks"] = (P, F, W)
    given = {"tuples": tuples, "fingers": fingers, "margin": margin, "accept": accept, "counts": counts,
             "masks": masks}
    for name, shape in want.items():
        t = given[name]
        if t is None:
            if name in ("counts", "masks"):
                raise ValueError(f"{name} is required when tuples are sampled")
            continue
        if tuple(t.shape) != shape:
            raise ValueError(f"{name} must be {list(shape)}, got {list(t.shape)}")
        if t.device != soa.device:
            raise ValueError(f"{name} is on {t.device}, soa on {soa.device}")


class Field:
    """Library-owned contact field (cf_field)."""

    def __init__(self, handle: int, n_fingers: int | None = None, n_joints: int | None = None,
                 n_slots: int | None = None):
        self._h = c_void_p(handle)
        self._shape = (n_fingers, n_joints) if n_fingers is not None and n_joints is not None else None
        self._slots = n_slots

    @property
    def handle(self):
        return self._h

    def _fj(self):
        """(fingers, joints) without waiting for the build: known from the hand when the field was built
        here (info() waits for the build to finish, to report its time)."""
        if self._shape is None:
            inf = self.info()
            self._shape = (int(inf.n_fingers), int(inf.n_joints))
        return self._shape

    @property
    def n_fingers(self) -> int:
        return self._fj()[0]

    @property
    def n_joints(self) -> int:
        return self._fj()[1]

    @property
    def n_slots(self) -> int:
        """Table slots = rows per pose of the query: the fingers, or the patches of a patch field."""
        if self._slots is None:
            self._slots = int(self.info().n_slots)
        return self._slots

    def info(self) -> FieldInfo:
        inf = FieldInfo()
        _check(_cf_field_get_info(self._h, byref(inf)))
        return inf

    def table(self) -> np.ndarray:
        inf = self.info()
        out = np.zeros(int(inf.table_words), np.uint32)
        _check(_cf_field_copy_table(self._h, out.ctypes.data_as(POINTER(c_uint32)), out.size))
        return out

    def rep(self):
        """Representative table (want_rep): (keys uint64 [slots], vals uint32 [slots]); empty slots have key ~0."""
        n = c_int64()
        _check(_cf_field_rep_slots(self._h, byref(n)))
        keys = np.zeros(int(n.value), np.uint64)
        vals = np.zeros(int(n.value), np.uint32)
        if n.value:
            _check(_cf_field_copy_rep(self._h, keys.ctypes.data_as(POINTER(c_uint64)),
                                      vals.ctypes.data_as(POINTER(c_uint32)), keys.size))
        return keys, vals

    def save(self, path: str):
        _check(_cf_field_save(self._h, path.encode()))

    @staticmethod
    def load(path: str) -> "Field":
        h = c_void_p()
        _check(_cf_field_load(path.encode(), byref(h)))
        return Field(h.value)

    def close(self):
        if self._h:
            _cf_field_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build(hand, inv_h, bin_dirs, q, stream=None, want_rep: bool = False, dilate_deg: float = 0.0,
          patches: bool = False) -> Field:
    """cf_build: hand is any object with base/axis/offset/surf_p/surf_n/surf_link
    arrays (host) and optionally lo/hi/radius, q a [F, J, S] float32 CUDA tensor
    of joint samples.  want_rep keeps the reverse-lookup table (needs limits).
    patches: one table slot per (finger, link with surface points)."""
    import torch
    keep = [_np(hand.base, np.float32), _np(hand.axis, np.float32), _np(hand.offset, np.float32),
            _np(hand.surf_p, np.float32), _np(hand.surf_n, np.float32), _np(hand.surf_link, np.int32)]
    F, J, M = int(keep[0].shape[0]), int(keep[1].shape[1]), int(keep[3].shape[1])
    lim = None
    if getattr(hand, "lo", None) is not None:
        lim = [_np(hand.lo, np.float32), _np(hand.hi, np.float32), _np(hand.radius, np.float32)]
        for a in lim:
            if a.shape != (F, J):
                raise ValueError(f"lo / hi / radius must be [F={F}, J={J}]")
    hd = HandDesc(F, J, M, _fp(keep[0]), _fp(keep[1]), _fp(keep[2]), _fp(keep[3]), _fp(keep[4]),
                  keep[5].ctypes.data_as(POINTER(c_int32)),
                  *([_fp(a) for a in lim] if lim else [None, None, None]))
    dirs = _np(bin_dirs, np.float32)
    prm = FieldParams(float(np.float32(inv_h)), int(dirs.shape[0]), _fp(dirs), 1 if want_rep else 0,
                      float(dilate_deg), 1 if patches else 0)
    qp = _dev(q, torch.float32, "q")
    if q.dim() != 3 or tuple(q.shape[:2]) != (F, J):
        raise ValueError(f"q must be [F={F}, J={J}, S]")
    h = c_void_p()
    _check(_cf_build(byref(hd), byref(prm), qp, int(q.shape[2]), _stream(stream), byref(h)))
    n_slots = sum(len(np.unique(keep[5][f])) for f in range(F)) if patches else F
    return Field(h.value, F, J, n_slots)


def query_domains(field: Field, soa, poses, masks=None, counts=None, want_masks: bool = True, stream=None):
    """cf_query_domains -> (masks [P, S, W] int32 view of uint32 words or None, counts [P, S] int32),
    S = field.n_slots (the fingers, or the patches of a patch field)."""
    import torch
    F = field.n_slots
    obj = points_struct(soa)
    P = int(poses.shape[0])
    _dev(poses, torch.float32, "poses")
    W = (obj.n + 31) // 32
    dev = soa.device
    if want_masks and masks is None:
        masks = torch.empty((P, F, W), dtype=torch.int32, device=dev)
    if counts is None:
        counts = torch.empty((P, F), dtype=torch.int32, device=dev)
    mp = _dev(masks, torch.int32, "masks") if masks is not None else None
    _check(_cf_query(field.handle, byref(obj), c_void_p(poses.data_ptr()), P, mp, _dev(counts, torch.int32, "counts"),
                     _stream(stream)))
    return masks, counts


def merge_domains(field: Field, slot_masks, n_words: int, masks=None, counts=None, stream=None):
    """cf_merge_domains: per-finger domains [P, F, W] and counts [P, F] from a
    query's slot rows [P, n_slots, W] (Sec. 5.3 dependency groups)."""
    import torch
    P = int(slot_masks.shape[0])
    F = field.n_fingers
    if tuple(slot_masks.shape) != (P, field.n_slots, n_words):
        raise ValueError(f"slot_masks must be [{P}, {field.n_slots}, {n_words}], got {list(slot_masks.shape)}")
    dev = slot_masks.device
    if masks is None:
        masks = torch.empty((P, F, n_words), dtype=torch.int32, device=dev)
    if counts is None:
        counts = torch.empty((P, F), dtype=torch.int32, device=dev)
    if tuple(masks.shape) != (P, F, n_words) or tuple(counts.shape) != (P, F):
        raise ValueError("masks / counts must be [P, F, W] / [P, F]")
    _check(_cf_merge(field.handle, _dev(slot_masks, torch.int32, "slot_masks"), P, int(n_words),
                     _dev(masks, torch.int32, "masks"), _dev(counts, torch.int32, "counts"), _stream(stream)))
    return masks, counts


def score_params(T, k, mu, K, eps, centroid, rho, seed, tuples_given=False) -> ScoreParams:
    c = (c_float * 3)(*[float(x) for x in np.asarray(centroid, np.float32)])
    return ScoreParams(int(T), int(k), int(K), float(mu), float(eps), c, float(np.float32(rho)), int(seed),
                       1 if tuples_given else 0)


def score_tuples(soa, n_fingers: int, masks, counts, prm: ScoreParams, tuples=None, fingers=None, stream=None,
                 margin=None, accept=None):
    """cf_score_tuples -> (tuples [P,T,k] int32, fingers [P,T,k] uint8, margin [P,T] f32, accept [P,T] uint8).
    With prm.tuples_given the given ``tuples`` tensor is scored (masks/counts may be None).
    Output tensors not given are allocated."""
    import torch
    obj = points_struct(soa)
    dev = soa.device
    if prm.tuples_given:
        if tuples is None:
            raise ValueError("tuples_given needs tuples")
        P = int(tuples.shape[0])
    else:
        P = int(counts.shape[0])
    T, k = int(prm.n_tuples), int(prm.k)
    _check_score_shapes(soa, n_fingers, masks, counts, prm, P, tuples, fingers, margin, accept)
    if tuples is None:
        tuples = torch.empty((P, T, k), dtype=torch.int32, device=dev)
    if fingers is None and not prm.tuples_given:
        fingers = torch.empty((P, T, k), dtype=torch.uint8, device=dev)
    if margin is None:
        margin = torch.empty((P, T), dtype=torch.float32, device=dev)
    if accept is None:
        accept = torch.empty((P, T), dtype=torch.uint8, device=dev)
    mp = _dev(masks, torch.int32, "masks") if masks is not None else None
    cp = _dev(counts, torch.int32, "counts") if counts is not None else None
    fp = _dev(fingers, torch.uint8, "fingers") if fingers is not None else None
    _check(_cf_score(byref(obj), int(n_fingers), mp, cp, P, byref(prm), _dev(tuples, torch.int32, "tuples"), fp,
                     _dev(margin, torch.float32, "margin"), _dev(accept, torch.uint8, "accept"), _stream(stream)))
    return tuples, fingers, margin, accept


def sample_tuples(soa, n_fingers: int, masks, counts, prm: ScoreParams, tuples=None, fingers=None, stream=None):
    """cf_sample_tuples -> (tuples [P,T,k] int32, fingers [P,T,k] uint8)."""
    import torch
    obj = points_struct(soa)
    P = int(counts.shape[0])
    T, k = int(prm.n_tuples), int(prm.k)
    _check_score_shapes(soa, n_fingers, masks, counts, prm, P, tuples, fingers)
    if tuples is None:
        tuples = torch.empty((P, T, k), dtype=torch.int32, device=soa.device)
    if fingers is None:
        fingers = torch.empty((P, T, k), dtype=torch.uint8, device=soa.device)
    _check(_cf_sample(byref(obj), int(n_fingers), _dev(masks, torch.int32, "masks"), _dev(counts, torch.int32, "counts"),
                      P, byref(prm), _dev(tuples, torch.int32, "tuples"), _dev(fingers, torch.uint8, "fingers"),
                      _stream(stream)))
    return tuples, fingers


def score_tuples_noalloc(soa, n_fingers: int, masks, counts, prm: ScoreParams, tuples, fingers, margin, accept,
                         stream=None):
    """cf_score_tuples_noalloc: like score_tuples, but every output tensor is
    supplied by the caller and libcf allocates no device memory during the call
    (any global scratch comes from a library-wide device array; calls that
    overlap on the GPU must be serialised by the caller)."""
    import torch
    P = int(tuples.shape[0])
    _check_score_shapes(soa, n_fingers, masks, counts, prm, P, tuples, fingers, margin, accept)
    obj = points_struct(soa)
    mp = _dev(masks, torch.int32, "masks") if masks is not None else None
    cp = _dev(counts, torch.int32, "counts") if counts is not None else None
    fp = _dev(fingers, torch.uint8, "fingers") if fingers is not None else None
    _check(_cf_score_noalloc(byref(obj), int(n_fingers), mp, cp, P, byref(prm), _dev(tuples, torch.int32, "tuples"),
                             fp, _dev(margin, torch.float32, "margin"), _dev(accept, torch.uint8, "accept"),
                             _stream(stream)))
    return tuples, fingers, margin, accept


def _batch_items(items):
    import torch
    arr = (BatchItem * len(items))()
    for j, it in enumerate(items):
        obj = points_struct(it["soa"])
        P = int(it["poses"].shape[0])
        arr[j] = BatchItem(it["field"].handle, obj, _dev(it["poses"], torch.float32, "poses"), P, it["prm"],
                           _dev(it["masks"], torch.int32, "masks"), _dev(it["counts"], torch.int32, "counts"),
                           _dev(it["tuples"], torch.int32, "tuples"), _dev(it["fingers"], torch.uint8, "fingers"),
                           _dev(it["margin"], torch.float32, "margin"), _dev(it["accept"], torch.uint8, "accept"))
    return arr


class Batch:
    """cf_batch: many object requests run as one launch per kernel variant,
    replayed as a CUDA graph.  ``items`` are dicts with keys field, soa, poses,
    prm, masks, counts, tuples, fingers, margin, accept (CUDA tensors as in
    query_domains / score_tuples)."""

    def __init__(self, items):
        arr = _batch_items(items)
        self._keep = list(items)
        h = c_void_p()
        _check(_cf_batch_create(arr, len(items), byref(h)))
        self._h = h

    def run(self, stream=None):
        _check(_cf_batch_run(self._h, _stream(stream)))

    def launches(self):
        n, g = c_int32(0), c_int32(0)
        _check(_cf_batch_launches(self._h, byref(n), byref(g)))
        return int(n.value), int(g.value)

    def close(self):
        if self._h:
            _cf_batch_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_item(field: Field, soa, poses, prm: ScoreParams):
    """Allocate the outputs of one batch item (torch, on soa's device)."""
    import torch
    F = field.n_fingers
    P = int(poses.shape[0])
    W = (int(soa.shape[1]) + 31) // 32
    T, k = int(prm.n_tuples), int(prm.k)
    dev = soa.device
    return dict(field=field, soa=soa, poses=poses, prm=prm,
                masks=torch.empty((P, F, W), dtype=torch.int32, device=dev),
                counts=torch.empty((P, F), dtype=torch.int32, device=dev),
                tuples=torch.empty((P, T, k), dtype=torch.int32, device=dev),
                fingers=torch.empty((P, T, k), dtype=torch.uint8, device=dev),
                margin=torch.empty((P, T), dtype=torch.float32, device=dev),
                accept=torch.empty((P, T), dtype=torch.uint8, device=dev))


class Engine:
    """cf_engine: the served form (continuous batching over arriving requests).
    Results come back as dicts with the accepted tuples copied to numpy."""

    def __init__(self, fields, hbm_budget_bytes=64 << 30, max_active=64, pose_chunk=256, pose_cap=65536,
                 pose_chunk_max=0, chunk_pairs_max=0, reserve_bytes=0):
        """pose_chunk_max > pose_chunk: adaptive chunks (cf_engine_params.pose_chunk_max, chunk_pairs_max);
        reserve_bytes: device memory the library's pool grows by at creation."""
        self.fields = list(fields)
        arr = (c_void_p * len(self.fields))(*[f.handle.value for f in self.fields])
        self._arr = arr
        p = EngineParams(arr, len(self.fields), int(hbm_budget_bytes), int(max_active), int(pose_chunk),
                         int(pose_cap), int(pose_chunk_max), int(chunk_pairs_max), int(reserve_bytes))
        h = c_void_p()
        _check(_cf_engine_create(byref(p), byref(h)))
        self._h = h

    def submit(self, field: int, h_soa: np.ndarray, h_poses: np.ndarray, prm: ScoreParams, n_grasps: int,
               tag: int = 0) -> int:
        soa = _np(h_soa, np.float32)
        poses = _np(h_poses, np.float32).reshape(-1, 12)
        q = Request(int(field), c_void_p(soa.ctypes.data), int(soa.shape[1]), c_void_p(poses.ctypes.data),
                    int(poses.shape[0]), prm, int(n_grasps), int(tag))
        rid = c_uint64(0)
        _check(_cf_engine_submit(self._h, byref(q), byref(rid)))
        return int(rid.value)

    def poll(self, max_results: int = 256):
        buf = (Result * max_results)()
        n = c_int32(0)
        _check(_cf_engine_poll(self._h, buf, max_results, byref(n)))
        out = []
        for i in range(n.value):
            r = buf[i]
            na, k = int(r.n_accepted), int(r.k)
            d = dict(id=int(r.id), tag=int(r.tag), status=int(r.status), partial=bool(r.partial),
                     n_accepted=na, n_poses_used=int(r.n_poses_used), t_submit=r.t_submit, t_admit=r.t_admit,
                     t_done=r.t_done, n_rounds=int(r.n_rounds), t_first_round=r.t_first_round,
                     pose=np.ctypeslib.as_array(r.pose, (na,)).copy() if na else np.zeros(0, np.int32),
                     tuples=np.ctypeslib.as_array(r.tuples, (na * k,)).reshape(na, k).copy() if na
                     else np.zeros((0, k), np.int32),
                     margin=np.ctypeslib.as_array(r.margin, (na,)).copy() if na else np.zeros(0, np.float32))
            _cf_engine_result_free(byref(buf[i]))
            out.append(d)
        return out

    def stats(self) -> dict:
        s = EngineStats()
        _check(_cf_engine_get_stats(self._h, byref(s)))
        return {f: getattr(s, f) for f, _ in EngineStats._fields_}

    def drain(self, timeout_ms: int = -1):
        _check(_cf_engine_drain(self._h, int(timeout_ms)))

    def close(self):
        if self._h:
            _cf_engine_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# cf_grasp: one accepted grasp (pose index, margin, the k point ids padded with -1 to CF_MAX_K)
GRASP_DTYPE = np.dtype([("pose", "<i4"), ("margin", "<f4"), ("point", "<i4", (4,))])


class Plan:
    """cf_plan: one object request driven from host buffers (H2D, query,
    sample + score, D2H inside the call)."""

    def __init__(self, n_fingers: int, n_max: int, p_max: int, prm: ScoreParams):
        self.prm = prm
        h = c_void_p()
        _check(_cf_plan_create(int(n_fingers), int(n_max), int(p_max), byref(prm), byref(h)))
        self._h = h

    def run_host(self, field: Field, h_soa: np.ndarray, h_poses: np.ndarray, h_tuples=None, h_margin=None,
                 h_accept=None, stream=None) -> int:
        """h_soa [6, N] float32, h_poses [P, 12] float32 (host, ideally pinned
        numpy views of torch pinned tensors); outputs are optional host arrays.
        Returns the number of accepted tuples."""
        n = int(h_soa.shape[1])
        P = int(h_poses.shape[0])
        nacc = c_int64(0)

        def ptr(a):
            return c_void_p(a.ctypes.data) if a is not None else None

        _check(_cf_plan_run_host(self._h, field.handle, ptr(h_soa), n, ptr(h_poses), P, byref(self.prm), ptr(h_tuples),
                                 ptr(h_margin), ptr(h_accept), byref(nacc), _stream(stream)))
        return int(nacc.value)

    def run_host_accepted(self, field: Field, h_soa: np.ndarray, h_poses: np.ndarray, h_grasps: np.ndarray,
                          stream=None) -> int:
        """cf_plan_run_host_accepted: the accepted tuples only, gathered on the device into
        h_grasps (a GRASP_DTYPE array, ideally pinned), in (pose, tuple) order.  Returns the
        number accepted (larger than len(h_grasps) when the array was too small)."""
        if h_grasps.dtype != GRASP_DTYPE or not h_grasps.flags["C_CONTIGUOUS"]:
            raise ValueError("h_grasps must be a contiguous GRASP_DTYPE array")
        nacc = c_int64(0)
        _check(_cf_plan_run_host_accepted(self._h, field.handle, c_void_p(h_soa.ctypes.data), int(h_soa.shape[1]),
                                          c_void_p(h_poses.ctypes.data), int(h_poses.shape[0]), byref(self.prm),
                                          c_void_p(h_grasps.ctypes.data) if len(h_grasps) else None, len(h_grasps),
                                          byref(nacc), _stream(stream)))
        return int(nacc.value)

    def close(self):
        if self._h:
            _cf_plan_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def score_gswo(soa, prm: ScoreParams, tuples, n_iter: int = 256, eps_g: float = 1e-4, stream=None):
    """cf_score_gswo over tuples [P,T,k] -> (value [P,T] f32, accept [P,T] u8)."""
    import torch
    obj = points_struct(soa)
    P, T = int(tuples.shape[0]), int(prm.n_tuples)
    value = torch.empty((P, T), dtype=torch.float32, device=soa.device)
    accept = torch.empty((P, T), dtype=torch.uint8, device=soa.device)
    _check(_cf_gswo(byref(obj), P, byref(prm), int(n_iter), float(eps_g), _dev(tuples, torch.int32, "tuples"),
                    _dev(value, torch.float32, "value"), _dev(accept, torch.uint8, "accept"), _stream(stream)))
    return value, accept


def opt_params(n_outer=2, n_inner=8, sigma=0.005, zero_tol=1e-6, min_gain=1e-2, warm_start=True) -> OptParams:
    return OptParams(int(n_outer), int(n_inner), float(sigma), float(zero_tol), float(min_gain),
                     1 if warm_start else 0)


def optimize_tuples(soa, n_fingers: int, masks, prm: ScoreParams, opt: OptParams, tuples, fingers, stream=None):
    """cf_optimize_tuples: improves ``tuples`` [P,T,k] in place; returns (margin [P,T] f32, accept [P,T] u8).
    ``prm`` must have tuples_given set."""
    import torch
    obj = points_struct(soa)
    P, T = int(tuples.shape[0]), int(prm.n_tuples)
    margin = torch.empty((P, T), dtype=torch.float32, device=soa.device)
    accept = torch.empty((P, T), dtype=torch.uint8, device=soa.device)
    _check(_cf_optimize(byref(obj), int(n_fingers), _dev(masks, torch.int32, "masks"), P, byref(prm), byref(opt),
                        _dev(tuples, torch.int32, "tuples"), _dev(fingers, torch.uint8, "fingers"),
                        _dev(margin, torch.float32, "margin"), _dev(accept, torch.uint8, "accept"), _stream(stream)))
    return margin, accept


def ik_params(beta=0.01, lam=1e-4, n_phase1=16, n_rounds=4, n_phase2=4, tol_pos=2e-3, tol_deg=20.0) -> IkParams:
    return IkParams(float(beta), float(lam), int(n_phase1), int(n_rounds), int(n_phase2), float(tol_pos),
                    float(np.float32(np.cos(np.radians(tol_deg)))))


def ik_dls(field: Field, soa, poses, T: int, k: int, tuples, fingers, accept, prm: IkParams, stream=None):
    """cf_ik_dls over n = tuples.numel() // k slots -> dict of q [n,F,J] f32, used [n,F,J] u8,
    contacts [6, n*k] f32 (object frame), rtuples [n,k] i32, resid [n,k,2] f32, ok [n] u8."""
    import torch
    F, J = field.n_fingers, field.n_joints
    obj = points_struct(soa)
    n = int(tuples.numel()) // int(k)
    dev = soa.device
    out = dict(q=torch.empty((n, F, J), dtype=torch.float32, device=dev),
               used=torch.empty((n, F, J), dtype=torch.uint8, device=dev),
               contacts=torch.empty((6, n * k), dtype=torch.float32, device=dev),
               rtuples=torch.empty((n, k), dtype=torch.int32, device=dev),
               resid=torch.empty((n, k, 2), dtype=torch.float32, device=dev),
               ok=torch.empty((n,), dtype=torch.uint8, device=dev))
    ap = _dev(accept, torch.uint8, "accept") if accept is not None else None
    _check(_cf_ik_dls(field.handle, byref(obj), _dev(poses, torch.float32, "poses"), n, int(T), int(k),
                      _dev(tuples, torch.int32, "tuples"), _dev(fingers, torch.uint8, "fingers"), ap, byref(prm),
                      _dev(out["q"], torch.float32, "q"), _dev(out["used"], torch.uint8, "used"),
                      _dev(out["contacts"], torch.float32, "contacts"), _dev(out["rtuples"], torch.int32, "rtuples"),
                      _dev(out["resid"], torch.float32, "resid"), _dev(out["ok"], torch.uint8, "ok"),
                      _stream(stream)))
    return out


def sdf_box(soa_host, h: float, margin: float):
    """cf_sdf_box: the grid box of cf_sdf_build for host points [6, N] -> (lo [3] f32, h, dims [3] int32)."""
    pts = _np(soa_host, np.float32)
    if pts.ndim != 2 or pts.shape[0] != 6:
        raise ValueError("soa_host must be [6, N]")
    lo = (c_float * 3)()
    dims = (c_int32 * 3)()
    _check(_cf_sdf_box(_fp(pts), int(pts.shape[1]), float(np.float32(h)), float(np.float32(margin)), lo, dims))
    return np.array(lo[:], np.float32), float(np.float32(h)), np.array(dims[:], np.int32)


class Sdf:
    """Library-owned object SDF grid (cf_sdf)."""

    def __init__(self, soa, lo, h: float, dims, stream=None):
        obj = points_struct(soa)
        lo_ = _np(lo, np.float32)
        dims_ = _np(dims, np.int32)
        if lo_.shape != (3,) or dims_.shape != (3,):
            raise ValueError("lo and dims must have 3 entries")
        self.lo, self.h, self.dims = lo_, float(np.float32(h)), dims_
        hh = c_void_p()
        _check(_cf_sdf_build(byref(obj), _fp(lo_), float(h), dims_.ctypes.data_as(POINTER(c_int32)),
                             _stream(stream), byref(hh)))
        self._h = hh

    @property
    def handle(self):
        return self._h

    def grid(self) -> np.ndarray:
        """[dims[2], dims[1], dims[0]] float32 (x fastest)."""
        n = int(np.prod(self.dims.astype(np.int64)))
        out = np.zeros(n, np.float32)
        _check(_cf_sdf_copy(self._h, _fp(out), n))
        return out.reshape(int(self.dims[2]), int(self.dims[1]), int(self.dims[0]))

    def close(self):
        if self._h:
            _cf_sdf_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def realize_params(pen_margin=2e-3, axis_step=1.25e-3, seed=0) -> RealizeParams:
    return RealizeParams(float(pen_margin), float(axis_step), int(seed))


def realize(field: Field, sdf: Sdf, poses, T: int, q, used, gate_a, gate_b, prm: RealizeParams, stream=None):
    """cf_realize: fills the free joints of q in place; returns flags [n] uint8 (0 = realised grasp)."""
    import torch
    n = int(q.shape[0])
    flags = torch.empty((n,), dtype=torch.uint8, device=q.device)
    ga = _dev(gate_a, torch.uint8, "gate_a") if gate_a is not None else None
    gb = _dev(gate_b, torch.uint8, "gate_b") if gate_b is not None else None
    _check(_cf_realize(field.handle, sdf.handle, _dev(poses, torch.float32, "poses"), n, int(T), byref(prm), ga, gb,
                       _dev(q, torch.float32, "q"), _dev(used, torch.uint8, "used"),
                       _dev(flags, torch.uint8, "flags"), _stream(stream)))
    return flags


def place_canonical(n_poses: int, centroid, g, up, d_lo=0.08, d_hi=0.12, seed=0, pose_base=0, device="cuda",
                    stream=None):
    """cf_place (canonical placement) -> poses [n_poses, 12] float32."""
    import torch
    f3 = lambda v: (c_float * 3)(*[float(x) for x in np.asarray(v, np.float32)])
    prm = PlaceParams(0, f3(centroid), f3(g), f3(up), float(d_lo), float(d_hi), int(seed), int(pose_base))
    poses = torch.empty((int(n_poses), 12), dtype=torch.float32, device=device)
    _check(_cf_place(None, None, int(n_poses), byref(prm), _dev(poses, torch.float32, "poses"), _stream(stream)))
    return poses


def place_exhaustive(field: Field, soa, n_poses: int, seed=0, pose_base=0, stream=None):
    """cf_place (exhaustive placement: a random field code aligned with a random object point)."""
    import torch
    z = (c_float * 3)(0.0, 0.0, 0.0)
    prm = PlaceParams(1, z, z, z, 0.0, 0.0, int(seed), int(pose_base))
    obj = points_struct(soa)
    poses = torch.empty((int(n_poses), 12), dtype=torch.float32, device=soa.device)
    _check(_cf_place(field.handle, byref(obj), int(n_poses), byref(prm), _dev(poses, torch.float32, "poses"),
                     _stream(stream)))
    return poses


def concave_filter(soa, sdf: "Sdf", side: float = 0.004, tau: float = 0.001, stream=None):
    """cf_concave_filter -> (keep [N] uint8, kept points [6, N] (first n_kept columns valid), n_kept int32 [1])."""
    import torch
    obj = points_struct(soa)
    N = int(soa.shape[1])
    keep = torch.empty((N,), dtype=torch.uint8, device=soa.device)
    out = torch.empty((6, N), dtype=torch.float32, device=soa.device)
    n = torch.zeros((1,), dtype=torch.int32, device=soa.device)
    _check(_cf_concave(byref(obj), sdf.handle, float(side), float(tau), _dev(keep, torch.uint8, "keep"),
                       _dev(out, torch.float32, "out"), _dev(n, torch.int32, "n"), _stream(stream)))
    return keep, out, n


def get_tuning() -> dict:
    t = Tuning()
    _check(_cf_get_tuning(byref(t)))
    return {f: getattr(t, f) for f, _ in Tuning._fields_}


def set_tuning(query_poses_per_block=4, score_refill=8, score_blocks_per_sm=0):
    _check(_cf_set_tuning(byref(Tuning(int(query_poses_per_block), int(score_refill),
                                       int(score_blocks_per_sm)))))


def autotune(items, reps: int = 3):
    """cf_autotune over batch items (dicts from batch_item): returns (tuning dict, (query ms, score ms))."""
    arr = _batch_items(items)
    t = Tuning()
    ms = (c_double * 2)()
    _check(_cf_autotune(arr, len(items), int(reps), byref(t), ms))
    return {f: getattr(t, f) for f, _ in Tuning._fields_}, (ms[0], ms[1])


def fp32_peak() -> float:
    """Measured FP32 FMA throughput of the current device, TFLOP/s (cf_fp32_peak)."""
    v = c_double()
    _check(_cf_fp32_peak(byref(v)))
    return float(v.value)


def device_status() -> int:
    v = c_uint32(0)
    _check(_cf_device_status(byref(v)))
    return int(v.value)


def device_counters(reset: bool = False):
    v = (c_uint64 * 4)()
    _check(_cf_device_counters(v, 1 if reset else 0))
    return {"lp_pivots": int(v[0]), "lps": int(v[1]), "tuples_scored": int(v[2]), "warm_starts": int(v[3])}


def pool_usage(reset_high: bool = False):
    """cf_pool_usage: bytes of the library's device pool in use, reserved, and
    the high-water mark of use since the last reset."""
    v = (c_uint64 * 3)()
    _check(_cf_pool_usage(v, 1 if reset_high else 0))
    return {"used": int(v[0]), "reserved": int(v[1]), "high": int(v[2])}


def place_static(palm_lo, palm_hi, soa, n_poses: int, seed: int, pose_base: int = 0, pen_margin: float = 2e-3,
                 stream=None):
    """cf_place_static -> (poses [P, 12] f32, static point [P] int32, valid [P] uint8): the object placed
    against the palm box's top face (Sec. 5.2 static links), with the penetration filter."""
    import torch
    obj = points_struct(soa)
    dev = soa.device
    P = int(n_poses)
    poses = torch.empty((P, 12), dtype=torch.float32, device=dev)
    pt = torch.empty((P,), dtype=torch.int32, device=dev)
    valid = torch.empty((P,), dtype=torch.uint8, device=dev)
    palm = PalmDesc((c_float * 3)(*[float(x) for x in np.asarray(palm_lo, np.float32)]),
                    (c_float * 3)(*[float(x) for x in np.asarray(palm_hi, np.float32)]))
    _check(_cf_place_static(byref(palm), byref(obj), P, c_uint64(int(seed)), int(pose_base), float(pen_margin),
                            c_void_p(poses.data_ptr()), c_void_p(pt.data_ptr()), c_void_p(valid.data_ptr()),
                            _stream(stream)))
    return poses, pt, valid


def append_contact(tuples, first, valid=None, stream=None):
    """cf_append_contact: [P, T, k] tuples -> [P, T, k + 1] with first[i] in front (invalid -> -1)."""
    import torch
    P, T, k = (int(x) for x in tuples.shape)
    if tuple(first.shape) != (P,) or (valid is not None and tuple(valid.shape) != (P,)):
        raise ValueError("first / valid must be [P]")
    out = torch.empty((P, T, k + 1), dtype=torch.int32, device=tuples.device)
    _check(_cf_append(_dev(tuples, torch.int32, "tuples"), P, T, k, _dev(first, torch.int32, "first"),
                      _dev(valid, torch.uint8, "valid") if valid is not None else None,
                      _dev(out, torch.int32, "out"), _stream(stream)))
    return out

