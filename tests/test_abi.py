"""Host-side checks of the C ABI (no GPU needed): libcf.so loads, exports
every function include/cf.h declares, and rejects bad arguments before any
CUDA work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cf.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(cf_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    import paper_2511_07418_b300 as cf
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(cf._lib, n), n
    assert sorted(cf.EXPORTED) == names


def test_arguments_are_rejected_on_the_host():
    import paper_2511_07418_b300 as cf
    lib = cf._lib
    out = ctypes.c_void_p()
    assert lib.cf_build(None, None, None, 0, None, ctypes.byref(out)) == 1  # CF_EINVAL
    assert "hand" in cf._cf_last_error().decode()
    hd = cf.HandDesc(0, 3, 10)
    assert cf._cf_build(ctypes.byref(hd), None, None, 0, None, ctypes.byref(out)) == 1
    assert "n_fingers" in cf._cf_last_error().decode()
    pts = cf.Points(None, None, None, None, None, None, 0)
    prm = cf.score_params(T=4, k=7, mu=0.5, K=8, eps=0.01, centroid=[0, 0, 0], rho=0.05, seed=0)
    assert cf._cf_score(ctypes.byref(pts), 3, None, None, 1, ctypes.byref(prm), None, None, None, None, None) == 1
    assert "k=7" in cf._cf_last_error().decode()
    prm = cf.score_params(T=4, k=3, mu=0.5, K=16, eps=0.01, centroid=[0, 0, 0], rho=0.05, seed=0)
    assert cf._cf_score(ctypes.byref(pts), 3, None, None, 1, ctypes.byref(prm), None, None, None, None, None) == 1
    assert "> 32" in cf._cf_last_error().decode()
    assert cf._cf_query(None, ctypes.byref(pts), None, 0, None, None, None) == 1


def test_oracle_and_library_share_no_source():
    """The oracle is test infrastructure: the CUDA sources never include or
    name it, and the oracle never includes the library's headers."""
    csrc = os.path.join(ROOT, "paper_2511_07418_b300", "csrc")
    for f in os.listdir(csrc):
        s = open(os.path.join(csrc, f)).read()
        assert "oracle" not in s.lower(), f
    s = open(os.path.join(ROOT, "oracle", "cf_oracle.c")).read()
    assert '#include "cf' not in s
    py = open(os.path.join(ROOT, "paper_2511_07418_b300", "__init__.py")).read()
    assert "import oracle" not in py and "from oracle" not in py


def test_every_entry_point_rejects_missing_arguments_on_the_host():
    """Null handles, null outputs and out-of-range launch shapes come back as
    CF_EINVAL (a missing field file as CF_EIO) with a message, before any CUDA
    work; destroying a NULL handle is a no-op that succeeds."""
    import paper_2511_07418_b300 as cf
    from ctypes import byref, c_int32, c_int64, c_uint64, c_void_p
    out, n = c_void_p(), c_int32()
    pts = cf.Points(None, None, None, None, None, None, 0)
    bad_k = cf.score_params(T=4, k=7, mu=0.5, K=8, eps=0.01, centroid=[0, 0, 0], rho=0.05, seed=0)
    calls = {
        "cf_field_get_info": lambda: cf._cf_field_get_info(None, byref(cf.FieldInfo())),
        "cf_field_copy_table": lambda: cf._cf_field_copy_table(None, None, 0),
        "cf_field_save": lambda: cf._cf_field_save(None, b"unused"),
        "cf_field_load": lambda: cf._cf_field_load(None, byref(out)),
        "cf_field_rep_slots": lambda: cf._cf_field_rep_slots(None, byref(c_int64())),
        "cf_sample_tuples": lambda: cf._cf_sample(byref(pts), 3, None, None, 1, byref(bad_k), None, None, None),
        "cf_score_tuples_noalloc": lambda: cf._cf_score_noalloc(byref(pts), 3, None, None, 1, byref(bad_k),
                                                                None, None, None, None, None),
        "cf_batch_create": lambda: cf._cf_batch_create(None, 0, byref(out)),
        "cf_batch_run": lambda: cf._cf_batch_run(None, None),
        "cf_engine_create": lambda: cf._cf_engine_create(None, byref(out)),
        "cf_engine_create(no fields)": lambda: cf._cf_engine_create(
            byref(cf.EngineParams(None, 0, 1 << 30, 4, 1024, 4096)), byref(out)),
        "cf_engine_submit": lambda: cf._cf_engine_submit(None, None, byref(c_uint64())),
        "cf_engine_poll": lambda: cf._cf_engine_poll(None, None, 0, byref(n)),
        "cf_plan_create": lambda: cf._cf_plan_create(0, 0, 0, None, byref(out)),
        "cf_plan_run_host": lambda: cf._cf_plan_run_host(None, None, None, 0, None, 0, None, None, None, None,
                                                         None, None),
        "cf_ik_dls": lambda: cf._cf_ik_dls(None, None, None, 0, 0, 0, *([None] * 11)),
        "cf_sdf_build": lambda: cf._cf_sdf_build(None, None, 0.0, None, None, byref(out)),
        "cf_sdf_copy": lambda: cf._cf_sdf_copy(None, None, 0),
        "cf_realize": lambda: cf._cf_realize(None, None, None, 0, 0, *([None] * 7)),
        "cf_place": lambda: cf._cf_place(None, None, 0, None, None, None),
        "cf_concave_filter": lambda: cf._cf_concave(None, None, 0.0, 0.0, None, None, None, None),
        "cf_set_tuning(NULL)": lambda: cf._cf_set_tuning(None),
        "cf_set_tuning(17 poses per block)": lambda: cf._cf_set_tuning(byref(cf.Tuning(17, 8, 0))),
        "cf_set_tuning(refill 5)": lambda: cf._cf_set_tuning(byref(cf.Tuning(4, 5, 0))),
        "cf_get_tuning": lambda: cf._cf_get_tuning(None),
        "cf_autotune": lambda: cf._cf_autotune(None, 0, 1, None, None),
        "cf_score_gswo": lambda: cf._cf_gswo(None, 0, None, 0, 0.0, None, None, None, None),
        "cf_optimize_tuples": lambda: cf._cf_optimize(None, 0, None, 0, None, None, None, None, None, None, None),
        "cf_fp32_peak": lambda: cf._cf_fp32_peak(None),
        "cf_device_status": lambda: cf._cf_device_status(None),
        "cf_device_counters": lambda: cf._cf_device_counters(None, 0),
    }
    for name, call in calls.items():
        assert call() == 1, name
        assert cf._cf_last_error(), name
    assert cf._cf_field_load(b"/nonexistent/field.cf", byref(out)) == 7  # CF_EIO
    assert "cannot open" in cf._cf_last_error().decode()
    for destroy in (cf._cf_field_destroy, cf._cf_batch_destroy, cf._cf_engine_destroy, cf._cf_plan_destroy,
                    cf._cf_sdf_destroy, cf._cf_engine_result_free):
        assert destroy(None) == 0


def test_binding_without_the_library_fails_loudly(tmp_path):
    """The package has no CPU path: a copy of the binding without libcf.so
    refuses to import."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "cfcopy"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_2511_07418_b300", "__init__.py"), pkg / "__init__.py")
    r = subprocess.run([sys.executable, "-c", "import cfcopy"], cwd=tmp_path, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "no CPU path" in r.stderr


def test_binding_rejects_host_tensors():
    """Device tensors only: host tensors, wrong dtypes and wrong shapes are
    refused before any library call."""
    import torch
    import paper_2511_07418_b300 as cf
    with pytest.raises(TypeError, match="CUDA tensor"):
        cf.points_struct(torch.zeros(6, 64))
    with pytest.raises(TypeError, match="CUDA tensor"):
        cf.points_struct(np.zeros((6, 64), np.float32))
    prm = cf.score_params(T=4, k=3, mu=0.5, K=8, eps=0.01, centroid=[0, 0, 0], rho=0.05, seed=0)
    with pytest.raises(TypeError, match="CUDA tensor"):
        cf.score_tuples(torch.zeros(6, 64), 3, torch.zeros(2, 3, 2, dtype=torch.int32),
                        torch.zeros(2, 3, dtype=torch.int32), prm)


def test_scoring_wrappers_reject_bad_shapes_before_any_launch():
    """Every scoring wrapper checks the shapes of the tensors it passes on (the
    C side sees bare pointers): tuples / fingers [P, T, k], margin / accept
    [P, T], counts [P, F] and masks [P, F, ceil(N/32)] when sampling.  The
    check runs first, so host tensors suffice to exercise it."""
    import torch
    import paper_2511_07418_b300 as cf
    P, T, k, F, N = 3, 4, 3, 4, 70
    W = (N + 31) // 32
    soa = torch.zeros(6, N)
    prm = cf.score_params(T=T, k=k, mu=0.5, K=8, eps=0.01, centroid=[0, 0, 0], rho=0.05, seed=0)
    good = dict(masks=torch.zeros(P, F, W, dtype=torch.int32), counts=torch.zeros(P, F, dtype=torch.int32),
                tuples=torch.zeros(P, T, k, dtype=torch.int32), fingers=torch.zeros(P, T, k, dtype=torch.uint8),
                margin=torch.zeros(P, T), accept=torch.zeros(P, T, dtype=torch.uint8))
    bad = {"masks": torch.zeros(P, F, W - 1, dtype=torch.int32), "counts": torch.zeros(P, F + 1, dtype=torch.int32),
           "tuples": torch.zeros(P, T, k - 1, dtype=torch.int32), "fingers": torch.zeros(P, T - 1, k, dtype=torch.uint8),
           "margin": torch.zeros(P, T + 1), "accept": torch.zeros(P - 1, T, dtype=torch.uint8)}
    for name, t in bad.items():
        args = dict(good)
        args[name] = t
        with pytest.raises(ValueError, match=name):
            cf.score_tuples_noalloc(soa, F, args["masks"], args["counts"], prm, args["tuples"], args["fingers"],
                                    args["margin"], args["accept"])
    with pytest.raises(ValueError, match="counts is required"):
        cf.score_tuples_noalloc(soa, F, None, None, prm, good["tuples"], good["fingers"], good["margin"],
                                good["accept"])
    # shapes right: the next check (device tensors only) speaks
    with pytest.raises(TypeError, match="CUDA tensor"):
        cf.score_tuples_noalloc(soa, F, **{k_: v for k_, v in good.items() if k_ not in ("masks", "counts")},
                                masks=good["masks"], counts=good["counts"], prm=prm)


def test_scoring_rejects_tuple_counts_beyond_32_bits():
    """n_poses * n_tuples >= 2^32 is refused with CF_EINVAL before any launch
    (the kernels count tuples in 32 bits); the pointers are never touched."""
    import paper_2511_07418_b300 as cf
    from ctypes import byref, c_void_p
    fake = [c_void_p(256 * (i + 1)) for i in range(6)]
    pts = cf.Points(*fake, 64)
    prm = cf.score_params(T=1 << 16, k=3, mu=0.5, K=8, eps=0.01, centroid=[0, 0, 0], rho=0.05, seed=0,
                          tuples_given=True)
    p = c_void_p(4096)
    for fn in (cf._cf_score, cf._cf_score_noalloc):
        rc = fn(byref(pts), 4, None, None, 1 << 16, byref(prm), p, None, p, p, None)
        assert rc == cf.CF_EINVAL
        assert "2^32" in cf._cf_last_error().decode()


def test_sdf_box_covers_the_points_with_the_margin():
    """cf_sdf_box (host only): lo = min - margin, dims nodes spaced h reach past max + margin;
    bad arguments are refused."""
    import paper_2511_07418_b300 as cf
    rng = np.random.default_rng(4)
    soa = np.ascontiguousarray(rng.normal(scale=0.05, size=(6, 1000)).astype(np.float32))
    lo, h, dims = cf.sdf_box(soa, 0.004, 0.02)
    p = soa[:3].astype(np.float64)
    assert np.allclose(lo, p.min(axis=1) - 0.02, atol=1e-7)
    top = lo.astype(np.float64) + (dims - 1) * np.float32(0.004)
    assert np.all(top >= p.max(axis=1) + 0.02 - 1e-7) and np.all(top - np.float32(0.004) < p.max(axis=1) + 0.02)
    with pytest.raises(cf.CfError):
        cf.sdf_box(soa, 0.0, 0.02)
    bad = soa.copy()
    bad[1, 7] = np.nan
    with pytest.raises(cf.CfError, match="not finite"):
        cf.sdf_box(bad, 0.004, 0.02)
