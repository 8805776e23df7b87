#!/usr/bin/env python3
"""Benchmark of the Contact-Field grasp hot path on B300.

One step = the whole hot path over one synthetic request: build the hand's
contact field from its joint samples (FK + binning), query the object's
contact domains over every palm pose, sample T contact tuples per pose and
score them with the linearised closure LP.  The metric is valid grasps/s:
closure-accepted tuples per second of step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs (torchrun, one rank per GPU) are independent replicas: each
rank synthesises its own request (seed = rank), no data crosses ranks; value =
accepted tuples of all ranks / max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "hand20_tool"
METRIC = "valid grasps/s"
UNIT = "grasps/s"
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) per launch of each kernel, from one ncu capture of
# the current kernels per workload (dram__bytes_read.sum + dram__bytes_write.sum);
# a workload or kernel without a capture of its current code reports None.
# hand20_tool: captures at 4,096 of its 32,768 poses, scaled by 8 (the traffic grows with the poses).
NCU_TRAFFIC = {"hand16_superquadric": {"k_query_domains": 2_243_328 + 11_180_800, "k_score_lanes": 6_737_408 + 14_336,
                                       "k_fk_bin": 41_115_392 + 737_536, "k_sample_tuples": 67_277_824 + 822_016},
               "hand20_tool": {"k_query_domains": 8 * (29_575_168 + 116_316_416), "k_score_lanes": 8 * 7_904_768,
                               "k_sample_tuples": 8 * (167_910_656 + 2_677_760)}}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--poses", type=int, default=0, help="override the workload's pose count (profiling captures)")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--cpu-poses", type=int, default=32, help="poses in the oracle's timed sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-objects", type=int, default=64, help="objects of the batched-form leg (0: skip)")
    ap.add_argument("--served-seconds", type=float, default=30.0, help="seconds per offered rate (0: skip)")
    ap.add_argument("--served-rates", default="10,100,1000")
    ap.add_argument("--served-slots", type=int, default=256, help="engine slots (requests on the GPU at once)")
    ap.add_argument("--served-chunk", type=int, default=256, help="poses per request per engine round")
    ap.add_argument("--served-chunk-max", type=int, default=2048,
                    help="the adaptive_chunks streams: after its first round a request takes up to this many "
                         "poses per round (<= --served-chunk: no such streams)")
    ap.add_argument("--served-reserve-gb", type=float, default=4.0,
                    help="device memory each engine reserves in the library's pool at creation (GiB)")
    ap.add_argument("--served-chunk-pairs", type=int, default=1 << 26,
                    help="adaptive chunks: at most this many point-pose pairs per request and round (0: no limit)")
    ap.add_argument("--realized-steps", type=int, default=20, help="steps of the IK + realization leg (0: skip)")
    ap.add_argument("--optimized-steps", type=int, default=5, help="steps of the Alg. 2 optimisation leg (0: skip)")
    ap.add_argument("--gswo-steps", type=int, default=10, help="steps of the Eq. GSWO scoring leg (0: skip)")
    ap.add_argument("--extra-workload", default="hand16_superquadric",
                    help="a second workload whose main step is reported under its own key ('' to skip)")
    ap.add_argument("--extra-steps", type=int, default=100)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="time the main step under the default launch shapes instead of the autotuner's")
    ap.add_argument("--parity-poses", type=int, default=4,
                    help="poses of the timed step checked against the FP64 oracle (0: skip)")
    return ap.parse_args()


def _config(w):
    return {"workload": w.name, "fingers": w.hand.F, "dof": w.hand.F * w.hand.J, "points": w.obj.N,
            "joint_samples": w.S, "voxel_m": w.h, "normal_bins": w.B, "poses": w.P, "tuples_per_pose": w.T,
            "k": w.k, "mu": w.mu, "pyramid_edges": w.K, "eps": w.eps,
            "step": "field build + domain query + tuple sampling + closure LP",
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write, untimed)",
            "parallelism": "replicas"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except OSError:  # no nvidia-smi on this host: no clock record
            self.proc = None
            os.unlink(self.path)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for r in csv.reader(io.StringIO(fh.read())):
                r = [x.strip() for x in r]
                if len(r) < 10:
                    continue
                if self.uuid and self.uuid not in r[1]:
                    continue
                rows.append(r)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[6 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(times_ms, accepted, device=None):
    """Replica results -> job totals: the slowest rank's times (max) and the
    accepted tuples of all ranks (sum).  No data crosses ranks during a step;
    this runs once, after the timed region."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x) for x in times_ms], dtype=torch.float64, device=device)
    a = torch.tensor([int(x) for x in accepted], dtype=torch.int64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(a, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()], [int(x) for x in a.tolist()]


# ---------------------------------------------------------------------------
# oracle leg (CPU baseline / reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(w, n_poses: int, single_core: bool = False, fd=None):
    """The oracle on a bounded sample: field build (once per hand) and the
    per-pose path on the first n_poses poses.  Returns the sample's timings.
    single_core: one OpenMP thread and no LP process pool."""
    import numpy as np

    import oracle
    n_threads = oracle.num_threads()
    if single_core:
        oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        if fd is None:
            fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
        t_build = time.perf_counter() - t0
        soa = w.obj.soa()
        poses = w.poses[:n_poses]
        t1 = time.perf_counter()
        masks, counts = fd.query(soa, poses)
        tup, _ = oracle.sample_tuples(masks, counts, w.obj.N, w.T, w.k, w.seed)
        mar, acc, its = oracle.score_tuples(soa, tup, w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps,
                                            workers=not single_core)
        t_pose = time.perf_counter() - t1
    finally:
        oracle.set_threads(n_threads)
    valid = np.isfinite(mar)
    return {"t_build": t_build, "t_pose": t_pose, "accepted": int(acc.sum()), "n_poses": n_poses,
            "cores": 1 if single_core else max(n_threads, os.cpu_count() or 1), "field": fd,
            "lp_iterations_per_tuple": float(its[valid].mean()) if valid.any() else None}


def parity_leg(w, masks, counts, tuples, margin, accept, n_poses: int = 4):
    """The timed step's outputs on its first n_poses poses against the FP64
    oracle: mask entries that differ (each must lie inside the 1e-5 m / 1e-6
    band) and entries inside the band, then tuples on the poses whose masks
    agree and their margins and accept decisions.  Counts only; the GPU tests
    assert the rule."""
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins, band=True)
    soa = w.obj.soa()
    om, oc, amb = fd.query(soa, w.poses[:n_poses], amb=True)
    N = w.obj.N
    gm = masks[:n_poses].cpu().numpy().view(np.uint32)
    unpack = lambda m: np.unpackbits(np.ascontiguousarray(m).view(np.uint8), bitorder="little").reshape(
        m.shape[0], m.shape[1], -1)[:, :, :N]
    diff = unpack(gm) != unpack(om)
    same = np.all(gm.reshape(n_poses, -1) == om.reshape(n_poses, -1), axis=1)
    ot, _ = oracle.sample_tuples(om, oc, N, w.T, w.k, w.seed)
    gt = tuples[:n_poses].cpu().numpy()
    omar, _, _ = oracle.score_tuples(soa, ot[same], w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps)
    gmar = margin[:n_poses].cpu().numpy()[same].astype(np.float64).ravel()
    gacc = accept[:n_poses].cpu().numpy()[same].astype(bool).ravel()
    omar = omar.ravel()
    fin = np.isfinite(omar)
    rel = np.abs(gmar[fin] - np.maximum(omar[fin], 0)) / np.maximum(omar[fin], w.eps)
    dec = gacc != (omar <= w.eps)
    return {"poses": n_poses, "mask_entries": int(diff.size), "mask_differ": int(diff.sum()),
            "mask_differ_outside_band": int(np.sum(diff & (amb == 0))), "mask_in_band": int(np.count_nonzero(amb)),
            "mask_in_band_frac": float(np.count_nonzero(amb) / diff.size),
            "poses_masks_equal": int(same.sum()), "tuples_equal": bool(np.array_equal(gt[same], ot[same])),
            "tuples_scored": int(omar.size), "decisions_differ": int(dec.sum()),
            "decisions_in_band": int(np.sum(np.abs(omar - w.eps) <= 1e-4)),
            "margin_max_rel_err": float(rel.max(initial=0.0)), "seconds": time.perf_counter() - t0,
            "rule": "GPU vs FP64 oracle: differences allowed only inside the band (1e-5 m, 1e-6 cosine; 1e-4 of "
                    "eps for decisions) and below 1e-4 of all entries; margins within 1e-4 relative"}


def cpu_baseline(w, n_poses: int):
    s = oracle_sample(w, n_poses)
    scale = w.P / s["n_poses"]
    step_s = s["t_build"] + scale * s["t_pose"]
    value = s["accepted"] * scale / step_s
    # one core: the per-pose path on 2 poses (the field build is timed on all cores above and scaled by
    # the core count, an optimistic bound for one core)
    s1 = oracle_sample(w, 2, single_core=True, fd=s["field"])
    scale1 = w.P / s1["n_poses"]
    step1 = s["t_build"] * s["cores"] + scale1 * s1["t_pose"]
    one_core = {"value": s1["accepted"] * scale1 / step1, "per_pose_s": s1["t_pose"] / s1["n_poses"],
                "sample": "per-pose path of the first 2 poses on one thread (no LP pool); the build at "
                          f"{s['cores']} x its all-core time"}
    return {"value": value, "unit": UNIT, "cores": s["cores"], "kind": "oracle", "one_core": one_core,
            "lp_iterations_per_tuple": s["lp_iterations_per_tuple"],
            "sample": f"oracle field build over all {w.S} joint samples x {w.hand.F} fingers "
                      f"({s['t_build']:.2f} s) + query/sample/score of the first {n_poses} of {w.P} poses "
                      f"({s['t_pose']:.2f} s); a full step projected as build + {scale:.0f} x sample; "
                      "C/OpenMP field and masks, closure LPs by HiGHS over a process pool"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    import synth
    w = synth.workload(args.workload)
    # poses per step: about 0.1-0.3 s of host work (4 at 16,384 points x 64 tuples, 1 at 65,536 x 128)
    n = max(1, min(4, int(4 * 16384 * 64 // (w.obj.N * w.T))))
    t0 = time.perf_counter()
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
    t_build = time.perf_counter() - t0
    soa = w.obj.soa()

    def step(i):
        lo = (i * n) % w.P
        poses = w.poses[lo:lo + n]
        t = time.perf_counter()
        masks, counts = fd.query(soa, poses)
        tup, _ = oracle.sample_tuples(masks, counts, w.obj.N, w.T, w.k, w.seed)
        _, acc, _ = oracle.score_tuples(soa, tup, w.mu, w.K, w.obj.centroid, w.obj.rho, w.eps)
        return time.perf_counter() - t, int(acc.sum())

    for i in range(args.warmup):
        step(i)
    tot, accd = 0.0, 0
    for i in range(args.steps):
        dt, a = step(args.warmup + i)
        tot += dt + t_build * n / w.P  # the field build, amortised over the full request's poses
        accd += a
    value = accd / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle",
                             "cores": max(oracle.num_threads(), os.cpu_count() or 1),
                             "sample": f"each step: {n} poses of the {w.P}-pose request (query, sample, score) + the "
                                       f"field build ({t_build:.2f} s) pro rata {n}/{w.P}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main_leg(cf, torch, dev, w, steps, warmup, flush, barrier, sampler=None):
    """The timed main step (field build + query + sampling + scoring) on
    workload w: W untimed warm-up steps, then K steps timed with CUDA events on
    the launch stream, L2 flushed between them (untimed)."""
    import numpy as np
    F = w.hand.F
    q = torch.from_numpy(w.q).to(dev)
    soa = torch.from_numpy(w.obj.soa()).to(dev)
    poses = torch.from_numpy(w.poses).to(dev)
    W = (w.obj.N + 31) // 32
    masks = torch.empty((w.P, F, W), dtype=torch.int32, device=dev)
    counts = torch.empty((w.P, F), dtype=torch.int32, device=dev)
    tuples = torch.empty((w.P, w.T, w.k), dtype=torch.int32, device=dev)
    fingers = torch.empty((w.P, w.T, w.k), dtype=torch.uint8, device=dev)
    prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed)
    prm_given = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed, tuples_given=True)
    acc_total = torch.zeros((), dtype=torch.int64, device=dev)
    margin = torch.empty((w.P, w.T), dtype=torch.float32, device=dev)
    accept = torch.empty((w.P, w.T), dtype=torch.uint8, device=dev)
    n_ev = 5

    def step(ev):
        ev[0].record()
        field = cf.build(w.hand, w.inv_h, w.bins, q)
        ev[1].record()
        cf.query_domains(field, soa, poses, masks, counts)
        ev[2].record()
        cf.sample_tuples(soa, F, masks, counts, prm, tuples, fingers)
        ev[3].record()
        cf.score_tuples(soa, F, None, None, prm_given, tuples, margin=margin, accept=accept)
        ev[4].record()
        acc_total.add_(accept.sum())
        return field

    for _ in range(max(3, warmup)):
        step([torch.cuda.Event(enable_timing=True) for _ in range(n_ev)])
    acc_total.zero_()
    barrier()
    cf.device_counters(reset=True)
    cf.device_status()
    if sampler is not None:
        sampler.start()
        time.sleep(0.3)
    evs = []
    t_wall = time.perf_counter()
    for i in range(steps):
        flush.fill_(float(i))  # evict L2 between steps (not timed)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
        step(ev)
        evs.append(ev)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop() if sampler is not None else None
    status = cf.device_status()
    counters = cf.device_counters()
    ms = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(n_ev - 1)] for e in evs])
    return dict(ms=ms, total_ms=float(ms.sum()), accepted=int(acc_total.item()), t_wall=t_wall, clocks=clocks,
                status=status, counters=counters, masks=masks, counts=counts, tuples=tuples, fingers=fingers,
                margin=margin, accept=accept, launches_per_step=5)


# FP32 work counts (FMA = 2 flop) of the graded kernels, per unit:
#  - query, per (pose, point): the full-scan definition, 18 (rotate p and n) + 3B (bin argmax over B
#    directions) + 3F (cell index per finger), and the kernel's own count, 18 + 3 + 6 (the cube map names
#    <= 4 candidate bins, 2 on average: 6 FMA), an upper bound since it bins only where the cell's record
#    is not empty;
#  - score, per tuple: the dense two-phase tableau definition, pivots x 13 x 39 + 360 (wrench set-up,
#    k K x 15), with the pivots of the oracle's LP solver on the bench's own tuples, and the kernel's own
#    count, its pivots x 7 x (kK + 6) + 360 (one dense pivot of its scaled 6-row LP).
QUERY_FMA_OWN = 18 + 3 + 6


def roofline(w, per, counters, steps, peak_fp32, n_sm, sm_mhz, nominal_fp32, oracle_pivots_per_tuple=None):
    F = w.hand.F
    pairs = w.P * w.obj.N
    q_flop = pairs * (18 + 3 * w.B + 3 * F) * 2
    q_flop_own = pairs * QUERY_FMA_OWN * 2
    tuples = counters["tuples_scored"] / steps
    setup = w.k * w.K * 15
    s_flop_own = (counters["lp_pivots"] / steps * 7 * (w.k * w.K + 6) + tuples * setup) * 2
    s_flop_tableau = None
    if oracle_pivots_per_tuple is not None:
        s_flop_tableau = tuples * (oracle_pivots_per_tuple * 13 * 39 + setup) * 2
    b_flop = F * w.S * w.hand.M * (18 + 3 + 3 * w.B) * 2
    traffic = NCU_TRAFFIC.get(w.name, {})
    tf = lambda flop, ms: flop / (ms * 1e-3) / 1e12
    kernels = {
        "k_fk_cell_bounds+k_fk_bin": {"ms": per[0], "tflops": tf(b_flop, per[0]),
                                      "traffic_k_fk_bin": traffic.get("k_fk_bin")},
        "k_query_domains": {"ms": per[1], "tflops": tf(q_flop, per[1]), "tflops_kernel_count": tf(q_flop_own, per[1]),
                            "fma_per_pair": 18 + 3 * w.B + 3 * F, "fma_per_pair_kernel_count": QUERY_FMA_OWN,
                            "traffic": traffic.get("k_query_domains")},
        "k_sample_tuples": {"ms": per[2], "traffic": traffic.get("k_sample_tuples")},
        "k_score_lanes": {"ms": per[3], "tflops": tf(s_flop_tableau, per[3]) if s_flop_tableau else None,
                          "tflops_kernel_count": tf(s_flop_own, per[3]),
                          "oracle_pivots_per_tuple": oracle_pivots_per_tuple,
                          "kernel_pivots_per_tuple": counters["lp_pivots"] / max(1, counters["tuples_scored"]),
                          "traffic": traffic.get("k_score_lanes")},
    }
    for v in kernels.values():
        for key in ("tflops", "tflops_kernel_count"):
            if v.get(key) is not None:
                v["frac" + key[6:]] = v[key] / peak_fp32
    dom = max(["k_query_domains", "k_score_lanes"], key=lambda k: kernels[k]["ms"])
    # the definition's count where it is known (the scorer's needs the oracle's pivots), else the kernel's own
    dk = "" if kernels[dom].get("tflops") is not None else "_kernel_count"
    return {"kernel": dom, "bound": "alu", "achieved": kernels[dom]["tflops" + dk], "peak": peak_fp32,
            "unit": "TFLOP/s", "frac": kernels[dom]["frac" + dk], "traffic": kernels[dom].get("traffic"),
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "peak_basis": "measured: cf_fp32_peak (independent FP32 FMA chains, CUDA events) on this GPU before the "
                          f"timed region; nominal {n_sm} SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz = {nominal_fp32:.1f}",
            "achieved_basis": "algorithmic FLOP per launch (full-scan / dense-tableau definition) / CUDA-event time; "
                              "frac_kernel_count uses the kernel's own work count",
            "kernels": kernels}


def run_ours(args):
    import numpy as np
    import torch

    import paper_2511_07418_b300 as cf
    import synth

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)

    w = synth.workload(args.workload, seed=rank, P=args.poses or None)
    F = w.hand.F
    q = torch.from_numpy(w.q).to(dev)
    soa = torch.from_numpy(w.obj.soa()).to(dev)
    poses = torch.from_numpy(w.poses).to(dev)
    prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed)
    prm_given = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed, tuples_given=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    peak_measured = cf.fp32_peak()
    tuning = None
    if args.autotune:
        # the project's autotuner picks the launch shapes on this request (untimed): poses per query block,
        # the scorer's refill point and blocks per SM
        t0 = time.perf_counter()
        tune_field = cf.build(w.hand, w.inv_h, w.bins, q)
        item = cf.batch_item(tune_field, soa, poses, prm)
        shapes, tune_ms = cf.autotune([item], reps=3)
        tuning = {"shapes": shapes, "query_ms": tune_ms[0], "sample_score_ms": tune_ms[1],
                  "seconds": time.perf_counter() - t0}
        del item, tune_field
    sampler = ClockSampler(str(props.uuid) if hasattr(props, "uuid") else None)
    main = main_leg(cf, torch, dev, w, args.steps, args.warmup, flush, barrier, sampler)
    masks, counts, tuples, fingers = main["masks"], main["counts"], main["tuples"], main["fingers"]
    ms, total_ms, accepted, t_wall = main["ms"], main["total_ms"], main["accepted"], main["t_wall"]
    clocks, status, counters = main["clocks"], main["status"], main["counters"]

    # ---- e2e: the same step through the host-buffer plan ----------------
    # page-locked inputs written by one thread (np.copyto), as a caller filling its buffers would.  Filled
    # by torch's multi-threaded copy (tensor.pin_memory()), their lines stay dirty in many cores' caches and
    # every host-to-device copy snoops them: ~10 GB/s on the B300 hosts against ~45 GB/s
    def pinned(a: np.ndarray) -> torch.Tensor:
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0]).dtype, pin_memory=True)
        np.copyto(t.numpy(), a)
        return t

    q_h = pinned(w.q)
    soa_h = pinned(np.ascontiguousarray(w.obj.soa())).numpy()
    poses_h = pinned(w.poses).numpy()
    ht = torch.empty((w.P, w.T, w.k), dtype=torch.int32, pin_memory=True).numpy()
    hm = torch.empty((w.P, w.T), dtype=torch.float32, pin_memory=True).numpy()
    ha = torch.empty((w.P, w.T), dtype=torch.uint8, pin_memory=True).numpy()
    # the accepted grasps (24-byte records, room for every tuple) are what a caller keeps
    hg = torch.empty(w.P * w.T * cf.GRASP_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True).numpy()
    hg = hg.view(cf.GRASP_DTYPE)
    plan = cf.Plan(F, w.obj.N, w.P, prm)
    q_d = torch.empty_like(q)

    def e2e_step(all_outputs: bool):
        q_d.copy_(q_h, non_blocking=True)
        field = cf.build(w.hand, w.inv_h, w.bins, q_d)
        if all_outputs:
            return plan.run_host(field, soa_h, poses_h, ht, hm, ha)
        return plan.run_host_accepted(field, soa_h, poses_h, hg)

    def e2e_leg(all_outputs: bool):
        # the host-driven path needs more warm-up than the device loop: its step time falls for ~40 calls
        # (2.5 -> 2.1 ms on the B300 hosts) before it settles
        for _ in range(max(40, args.warmup)):
            e2e_step(all_outputs)
        t_s, n_acc = 0.0, 0
        for i in range(n_e2e):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n_acc += e2e_step(all_outputs)
            t_s += time.perf_counter() - t0
        return t_s, n_acc

    n_e2e = max(1, min(args.e2e_steps, args.steps))
    e2e_s, e2e_acc = e2e_leg(False)
    all_s, all_acc = e2e_leg(True)
    h2d = w.q.nbytes + 6 * 4 * w.obj.N + 12 * 4 * w.P
    d2h_all = w.P * w.T * (4 * w.k + 4 + 1)

    # ---- reduce over ranks ------------------------------------------------
    (total_ms, e2e_s, all_s), (accepted, e2e_acc, all_acc) = reduce_over_ranks([total_ms, e2e_s, all_s],
                                                                                [accepted, e2e_acc, all_acc], dev)
    d2h = 8 + cf.GRASP_DTYPE.itemsize * e2e_acc / (world * n_e2e)  # the count, then the records (mean)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    value = accepted / (total_ms / 1e3)
    per = ms.mean(axis=0)  # build, query, sample, score ms per step (rank 0)
    sm_mhz = (clocks or {}).get("sm_mhz") or 2032.0
    n_sm = props.multi_processor_count
    nominal_fp32 = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s: FP32 lanes x FMA x clock
    peak_fp32 = peak_measured
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(w),
            "value_field_cached": accepted / ((total_ms - float(ms[:, 0].sum())) / 1e3),
            "accept_rate": accepted / (world * args.steps * w.P * w.T),
            "breakdown_ms": {"build": per[0], "query": per[1], "sample": per[2], "score": per[3]},
            "wall_s_timed_region": t_wall,
            "gpu_launches": 5 * args.steps,
            "device_status": status,
            "lp": {"pivots_per_tuple": counters["lp_pivots"] / max(1, counters["tuples_scored"]),
                   "lps_per_tuple": counters["lps"] / max(1, counters["tuples_scored"])},
            "e2e": {"value": e2e_acc / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": n_e2e, "ms_per_step": 1e3 * e2e_s / n_e2e, "call": "cf_plan_run_host_accepted",
                    "gpu_launches_per_step": 8,  # field build 2, query, sample, score, gather 3
                    "all_outputs": {"value": all_acc / all_s, "d2h_bytes_per_step": d2h_all,
                                    "ms_per_step": 1e3 * all_s / n_e2e, "call": "cf_plan_run_host"}},
            "clocks": clocks, "tuning": tuning or {"shapes": cf.get_tuning(), "autotuned": False}}
    if world == 1 and args.realized_steps > 0:
        line["realized"] = run_realized(cf, torch, dev, w, args.realized_steps, soa, poses, masks, counts, tuples,
                                        fingers, prm, prm_given, flush)
        ikr = line["realized"]["ik_roofline"]
        ikr["peak"] = peak_fp32
        ikr["frac"] = ikr["achieved"] / peak_fp32
    if world == 1 and args.optimized_steps > 0:
        line["optimized"] = run_optimized(cf, torch, dev, w, args.optimized_steps, soa, poses, masks, counts, tuples,
                                          fingers, prm, flush)
        # the same without the warm start (every candidate's LPs from c' = 0): the free lunch's effect
        line["optimized"]["cold_start"] = run_optimized(cf, torch, dev, w, 1, soa, poses, masks, counts, tuples,
                                                        fingers, prm, flush, warm_start=False)
    if world == 1 and args.gswo_steps > 0:
        line["gswo"] = run_gswo(cf, torch, dev, w, args.gswo_steps, soa, poses, masks, counts, tuples, fingers, prm,
                                prm_given, flush)
        line["gswo"]["frac_of_fp32"] = line["gswo"]["gswo_tflops"] / peak_fp32
    if world == 1 and (args.batch_objects > 0 or args.served_seconds > 0):
        ws, fields = _hand_fields(cf, torch, dev)
        if args.batch_objects > 0:
            line["batched"] = run_batched(cf, torch, dev, args.batch_objects, ws, fields)
            # a mix where most objects leave the GPU idle in a launch of their own
            line["batched_small_objects"] = run_batched(cf, torch, dev, 4 * args.batch_objects, ws, fields,
                                                        n_range=(1024, 8192), p_range=(256, 2048), tune=False)
        if args.served_seconds > 0:
            rates = [float(x) for x in args.served_rates.split(",") if x]
            line["served"] = run_served(cf, torch, dev, ws, fields, rates, args.served_seconds,
                                        max_active=args.served_slots, pose_chunk=args.served_chunk,
                                        pose_chunk_max=args.served_chunk_max,
                                        chunk_pairs_max=args.served_chunk_pairs,
                                        reserve_bytes=int(args.served_reserve_gb * 2**30))
    if world == 1 and args.extra_workload and args.extra_workload != w.name:
        we = synth.workload(args.extra_workload)
        ex = main_leg(cf, torch, dev, we, args.extra_steps, args.warmup, flush, barrier)
        per_e = ex["ms"].mean(axis=0)
        line[we.name] = {"value": ex["accepted"] / (ex["total_ms"] / 1e3), "unit": UNIT, "steps": args.extra_steps,
                         "ms_per_step": ex["total_ms"] / args.extra_steps, "config": _config(we),
                         "accept_rate": ex["accepted"] / (args.extra_steps * we.P * we.T),
                         "breakdown_ms": {"build": per_e[0], "query": per_e[1], "sample": per_e[2], "score": per_e[3]},
                         "roofline": roofline(we, per_e, ex["counters"], args.extra_steps, peak_fp32, n_sm, sm_mhz,
                                              nominal_fp32),
                         "device_status": ex["status"]}
        del ex
    if world == 1 and args.parity_poses > 0:
        line["parity"] = parity_leg(w, masks, counts, tuples, main["margin"], main["accept"], args.parity_poses)
    piv = None
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_poses)
        piv = line["cpu_baseline"].get("lp_iterations_per_tuple")
    line["roofline"] = roofline(w, per, counters, args.steps, peak_fp32, n_sm, sm_mhz, nominal_fp32, piv)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# end to end through the kinematics rows: IK, re-scoring, realization
# ---------------------------------------------------------------------------

SDF_H = 0.004        # object SDF grid spacing (m)
SDF_MARGIN = 0.02    # grid margin around the object (> largest capsule radius + penetration margin)
PEN_MARGIN = 2e-3    # tolerated capsule penetration (m)


def run_realized(cf, torch, dev, w, steps, soa, poses, masks, counts, tuples, fingers, prm, prm_given, flush):
    """Valid grasps/s after kinematics optimisation and post-processing.  One
    step = domain query, tuple sampling, closure scoring, the object's SDF grid,
    reverse lookup + DLS IK of every accepted tuple, closure re-scoring of the
    realised contacts, and the realization filter (random free joints,
    capsule-vs-SDF penetration, finger-finger capsule intersection).  The
    hand's field (with its reverse-lookup table) is built once, outside."""
    import numpy as np
    F, k = w.hand.F, w.k
    n = w.P * w.T
    q = torch.from_numpy(w.q).to(dev)
    field = cf.build(w.hand, w.inv_h, w.bins, q, want_rep=True)
    lo, h, dims = cf.sdf_box(w.obj.soa(), SDF_H, SDF_MARGIN)
    ikp = cf.ik_params()
    rp = cf.realize_params(PEN_MARGIN, 0.5 / float(w.inv_h), w.seed)
    prm_re = cf.score_params(1, k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed, tuples_given=True)
    tot = torch.zeros(5, dtype=torch.int64, device=dev)  # accepted, ik ok, re-accepted, valid, scored
    n_ev = 8

    def step(ev):
        ev[0].record()
        cf.query_domains(field, soa, poses, masks, counts)
        ev[1].record()
        cf.sample_tuples(soa, F, masks, counts, prm, tuples, fingers)
        ev[2].record()
        _, _, _, accept = cf.score_tuples(soa, F, None, None, prm_given, tuples)
        ev[3].record()
        sdf = cf.Sdf(soa, lo, h, dims)
        ev[4].record()
        ik = cf.ik_dls(field, soa, poses, w.T, k, tuples, fingers, accept, ikp)
        ev[5].record()
        _, _, _, acc2 = cf.score_tuples(ik["contacts"], F, None, None, prm_re, tuples=ik["rtuples"].view(n, 1, k))
        ev[6].record()
        flags = cf.realize(field, sdf, poses, w.T, ik["q"], ik["used"], ik["ok"], acc2.view(n), rp)
        ev[7].record()
        tot[0].add_(accept.sum())
        tot[1].add_(ik["ok"].sum())
        tot[2].add_(acc2.sum())
        tot[3].add_((flags == 0).sum())
        return sdf

    for _ in range(3):
        step([torch.cuda.Event(enable_timing=True) for _ in range(n_ev)])
    tot.zero_()
    cf.device_status()
    evs = []
    for i in range(steps):
        flush.fill_(float(i))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
        step(ev)
        evs.append(ev)
    torch.cuda.synchronize()
    ms = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(n_ev - 1)] for e in evs])
    t = tot.cpu().numpy()
    total_ms = float(ms.sum())
    per = ms.mean(axis=0)
    names = ["query", "sample", "score", "sdf_build", "ik_dls", "rescore", "realize"]
    # algorithmic FP32 work of the IK per contact (FMA-equivalents; J joints):
    # a DLS step = chain 72J + Jacobian 24J + normal equations 3J(J+1) + 6J + Cholesky J^3/6 + solves J^2
    # + targets 51; a projection = chain 72J + 40
    J = w.hand.J
    n_steps, n_proj = 16 + 4 * 4, 4 + 1
    fma_contact = n_steps * (72 * J + 24 * J + 3 * J * (J + 1) + 6 * J + J ** 3 / 6 + J * J + 51) + n_proj * (72 * J + 40)
    ik_tflops = t[0] / steps * k * 2 * fma_contact / (per[4] * 1e-3) / 1e12
    return {"metric": "valid grasps/s after IK + realization", "value": float(t[3]) / (total_ms / 1e3),
            "unit": UNIT, "steps": steps, "ms_per_step": total_ms / steps,
            "breakdown_ms": {nm: float(v) for nm, v in zip(names, per)},
            "per_step": {"accepted": t[0] / steps, "ik_ok": t[1] / steps, "re_accepted": t[2] / steps,
                         "valid": t[3] / steps},
            "ik_roofline": {"bound": "alu", "achieved": ik_tflops, "unit": "TFLOP/s",
                            "flop_per_contact": 2 * fma_contact, "contacts_per_step": t[0] / steps * k},
            "gpu_launches_per_step": 10,
            "params": {"sdf_h": SDF_H, "sdf_dims": [int(x) for x in dims], "pen_margin": PEN_MARGIN,
                       "axis_step": 0.5 / float(w.inv_h), "ik": {"beta": 0.01, "lambda": 1e-4, "phase1": 16,
                                                                  "rounds": 4, "phase2": 4, "tol_pos": 2e-3,
                                                                  "tol_deg": 20.0}},
            "device_status": cf.device_status()}


# ---------------------------------------------------------------------------
# contact optimisation (Alg. 2) on top of the sampled tuples
# ---------------------------------------------------------------------------

OPT = dict(n_outer=2, n_inner=8, sigma=0.005, zero_tol=1e-6, min_gain=1e-2)


def run_optimized(cf, torch, dev, w, steps, soa, poses, masks, counts, tuples, fingers, prm, flush, warm_start=True):
    """Valid grasps/s when every sampled tuple goes through the blockwise
    zeroth-order contact optimisation of Alg. 2 (which scores the tuples it
    starts from).  One step = domain query, tuple sampling, optimisation; the
    hand's field is built once, outside."""
    import numpy as np
    F = w.hand.F
    q = torch.from_numpy(w.q).to(dev)
    field = cf.build(w.hand, w.inv_h, w.bins, q)
    prm_opt = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, w.obj.centroid, w.obj.rho, w.seed, tuples_given=True)
    opt = cf.opt_params(**OPT, warm_start=warm_start)
    tot = torch.zeros(1, dtype=torch.int64, device=dev)
    n_ev = 4

    def step(ev):
        ev[0].record()
        cf.query_domains(field, soa, poses, masks, counts)
        ev[1].record()
        cf.sample_tuples(soa, F, masks, counts, prm, tuples, fingers)
        ev[2].record()
        _, accept = cf.optimize_tuples(soa, F, masks, prm_opt, opt, tuples, fingers)
        ev[3].record()
        tot.add_(accept.sum())

    for _ in range(3):
        step([torch.cuda.Event(enable_timing=True) for _ in range(n_ev)])
    tot.zero_()
    cf.device_counters(reset=True)
    evs = []
    for i in range(steps):
        flush.fill_(float(i))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
        step(ev)
        evs.append(ev)
    torch.cuda.synchronize()
    counters = cf.device_counters()
    ms = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(n_ev - 1)] for e in evs])
    acc = int(tot.item())
    total_ms = float(ms.sum())
    per = ms.mean(axis=0)
    return {"metric": "valid grasps/s with Alg. 2 contact optimisation", "value": acc / (total_ms / 1e3),
            "unit": UNIT, "steps": steps, "ms_per_step": total_ms / steps,
            "breakdown_ms": {"query": float(per[0]), "sample": float(per[1]), "optimize": float(per[2])},
            "accept_rate": acc / (steps * w.P * w.T), "params": dict(OPT, warm_start=warm_start),
            "lp_per_tuple": counters["lps"] / max(1, counters["tuples_scored"]),
            "pivots_per_lp": counters["lp_pivots"] / max(1, counters["lps"]),
            "warm_starts_per_tuple": counters["warm_starts"] / max(1, counters["tuples_scored"]),
            "gpu_launches_per_step": 2 + opt_launches(w.k, OPT["n_outer"], warm_start),
            "device_status": cf.device_status()}


def opt_launches(k: int, n_outer: int, warm_start: bool) -> int:
    """Kernels of one cf_optimize_tuples call: word and chunk boxes, begin, the
    tuples' own LPs and their selection, then per step (n_outer x k) the
    projection, the candidate job list (count, scan, write), the candidates'
    LPs, the selection and, with the warm start, the winners' job list and
    replay, and the finish."""
    return 5 + n_outer * k * (10 if warm_start else 6) + 1


# ---------------------------------------------------------------------------
# the paper's own metric: Eq. GSWO with true friction cones
# ---------------------------------------------------------------------------

GSWO_ITERS = 256
GSWO_EPS = 1e-4   # on the squared objective (the LP's eps = 1e-2 on the max-norm, squared)


def run_gswo(cf, torch, dev, w, steps, soa, poses, masks, counts, tuples, fingers, prm, prm_given, flush):
    """Valid grasps/s when the sampled tuples are scored with Eq. GSWO (true
    cones, squared L2, accelerated projected gradient) instead of the
    linearised LP.  One step = domain query, tuple sampling, GSWO scoring; the
    field is built once, outside.  Also reports how often the two metrics agree
    on acceptance (LP scores computed outside the timed steps)."""
    import numpy as np
    F = w.hand.F
    q = torch.from_numpy(w.q).to(dev)
    field = cf.build(w.hand, w.inv_h, w.bins, q)
    tot = torch.zeros(1, dtype=torch.int64, device=dev)
    n_ev = 4

    def step(ev):
        ev[0].record()
        cf.query_domains(field, soa, poses, masks, counts)
        ev[1].record()
        cf.sample_tuples(soa, F, masks, counts, prm, tuples, fingers)
        ev[2].record()
        _, accept = cf.score_gswo(soa, prm_given, tuples, GSWO_ITERS, GSWO_EPS)
        ev[3].record()
        tot.add_(accept.sum())
        return accept

    for _ in range(3):
        step([torch.cuda.Event(enable_timing=True) for _ in range(n_ev)])
    tot.zero_()
    evs = []
    for i in range(steps):
        flush.fill_(float(i))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
        acc_g = step(ev)
        evs.append(ev)
    torch.cuda.synchronize()
    _, _, _, acc_lp = cf.score_tuples(soa, F, None, None, prm_given, tuples)
    agree = float((acc_lp.view(-1) == acc_g.view(-1)).float().mean().item())
    ms = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(n_ev - 1)] for e in evs])
    acc = int(tot.item())
    total_ms = float(ms.sum())
    per = ms.mean(axis=0)
    k = w.k
    # FMA per tuple: k subproblems x (Q y 9k^2 + step 3k + momentum 6k + projections 10k) per iteration
    fma_tuple = k * GSWO_ITERS * (9 * k * k + 19 * k)
    return {"metric": "valid grasps/s under Eq. GSWO (true cones)", "value": acc / (total_ms / 1e3),
            "unit": UNIT, "steps": steps, "ms_per_step": total_ms / steps,
            "breakdown_ms": {"query": float(per[0]), "sample": float(per[1]), "gswo": float(per[2])},
            "accept_rate": acc / (steps * w.P * w.T), "agreement_with_lp_accept": agree,
            "params": {"n_iter": GSWO_ITERS, "eps_g": GSWO_EPS},
            "gswo_tflops": w.P * w.T * 2 * fma_tuple / (per[2] * 1e-3) / 1e12,
            "gpu_launches_per_step": 3, "device_status": cf.device_status()}


# ---------------------------------------------------------------------------
# batched and served forms (same GPU, against the plain one-object-per-launch form)
# ---------------------------------------------------------------------------

def _hand_fields(cf, torch, dev):
    import synth
    ws, fields = [], []
    for name in ["tiny_sphere", "hand16_superquadric", "hand20_tool"]:
        w = synth.workload(name, P=1, N=64)
        ws.append(w)
        fields.append(cf.build(w.hand, w.inv_h, w.bins, torch.from_numpy(w.q).to(dev)))
    torch.cuda.synchronize()
    return ws, fields


def run_batched(cf, torch, dev, n_objects, ws, fields, n_range=(2048, 131072), p_range=(4096, 32768),
                tune=True):
    """The many-object batch: every object's query + sampling + scoring, once as
    plain per-object calls on one stream, once as the batch's graph replay
    (one persistent launch per stage)."""
    import numpy as np

    import synth
    names = ["tiny_sphere", "hand16_superquadric", "hand20_tool"]
    t_gen = time.perf_counter()
    specs = synth.batch_objects(n_objects, seed=0, n_range=n_range, p_range=p_range)
    items = []
    for j, sp in enumerate(specs):
        hi = names.index(sp["hand"])
        w = ws[hi]
        obj, poses = synth.batch_object_inputs(sp, w.hand)
        prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, obj.centroid, obj.rho, 7000 + j)
        it = cf.batch_item(fields[hi], torch.from_numpy(obj.soa()).to(dev), torch.from_numpy(poses).to(dev), prm)
        it["F"] = w.hand.F
        items.append(it)
    t_gen = time.perf_counter() - t_gen
    pairs = sum(int(it["soa"].shape[1]) * int(it["poses"].shape[0]) for it in items)
    tuples = sum(int(it["tuples"].numel()) // int(it["prm"].k) for it in items)

    def plain():
        for it in items:
            cf.query_domains(it["field"], it["soa"], it["poses"], it["masks"], it["counts"])
            cf.score_tuples(it["soa"], it["F"], it["masks"], it["counts"], it["prm"], it["tuples"], it["fingers"])

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = None
        for _ in range(reps):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best

    default_tuning = cf.get_tuning()
    t_plain = timed(plain)
    # the plain calls above allocate margin/accept per call; the batch writes into the items' own buffers
    batch = cf.Batch(items)
    t_batch_default = timed(batch.run)
    batch.close()
    out = {"objects": n_objects, "pose_point_pairs": pairs, "tuples": tuples,
           "plain_ms": t_plain, "default_tuning": default_tuning, "batched_ms_default_tuning": t_batch_default,
           "plain_launches": 3 * n_objects, "generate_s": t_gen,
           "workload": f"{n_objects} objects (superquadrics / tool composites), points log-uniform "
                       f"{n_range[0]:,}-{n_range[1]:,}, poses log-uniform {p_range[0]:,}-{p_range[1]:,}, hand per "
                       "object from the 3/4/5-finger hands (fields cached)"}
    t_batch = t_batch_default
    if tune:
        # the autotuner picks the launch shapes on these objects; the batch is re-created under them
        t_tune = time.perf_counter()
        tuning, tune_ms = cf.autotune(items, reps=2)
        out.update(autotuned=tuning, autotune_s=time.perf_counter() - t_tune, autotune_query_score_ms=list(tune_ms),
                   plain_ms_autotuned=timed(plain))
        batch = cf.Batch(items)
        t_batch = timed(batch.run)
        batch.close()
        cf.set_tuning(*default_tuning.values())
    batch = cf.Batch(items)
    batch.run()
    torch.cuda.synchronize()
    accepted = sum(int(it["accept"].sum()) for it in items)
    n_launch, n_groups = batch.launches()
    batch.close()
    out.update(accepted=accepted, batched_ms=t_batch, plain_grasps_per_s=accepted / (t_plain / 1e3),
               batched_grasps_per_s=accepted / (t_batch / 1e3), batched_launches=n_launch)
    return out


def run_served(cf, torch, dev, ws, fields, rates, seconds, pool=24, max_active=64, pose_chunk=256, pose_chunk_max=0,
               chunk_pairs_max=0, reserve_bytes=0):
    """Poisson request streams against the engine (continuous batching) and
    against the same engine with one slot (one request at a time, plain
    per-request launches); p50 / p99 latency and valid grasps/s per rate."""
    import numpy as np

    import synth
    rng = np.random.default_rng(11)
    names = ["tiny_sphere", "hand16_superquadric", "hand20_tool"]
    objs = []
    for o in range(pool):
        N = int(round(np.exp(rng.uniform(np.log(1024), np.log(65536)))))
        obj = synth.superquadric(N, 3000 + o) if o % 2 == 0 else synth.tool_composite(N, 3000 + o)
        hi = int(rng.integers(3))
        poses = synth.palm_poses(8192, 4000 + o, ws[hi].hand.grasp_centre, obj.centroid)
        objs.append((hi, obj.soa(), poses, obj))

    def stream(max_active, rate, seconds=seconds, budget=64 << 30, chunk_max=pose_chunk_max):
        eng = cf.Engine(fields, hbm_budget_bytes=budget, max_active=max_active, pose_chunk=pose_chunk, pose_cap=65536,
                        pose_chunk_max=chunk_max, chunk_pairs_max=chunk_pairs_max, reserve_bytes=min(budget, reserve_bytes))
        r = np.random.default_rng(int(rate) * 7 + max_active)
        t = 0.0
        arrivals = []
        while t < seconds:
            t += r.exponential(1.0 / rate)
            arrivals.append(t)
        done = []
        t0 = time.perf_counter()
        for j, ta in enumerate(arrivals):
            while time.perf_counter() - t0 < ta:
                done += eng.poll()
                time.sleep(0.0002)
            hi, soa, poses, obj = objs[int(r.integers(pool))]
            w = ws[hi]
            prm = cf.score_params(w.T, w.k, w.mu, w.K, w.eps, obj.centroid, obj.rho, 90000 + j)
            eng.submit(hi, soa, poses, prm, int(r.integers(100, 5001)), j)
        eng.drain(600000)
        done += eng.poll(4096)
        wall = time.perf_counter() - t0
        st = eng.stats()
        eng.close()
        lat = np.array([d["t_done"] - d["t_submit"] for d in done]) * 1e3
        acc = sum(d["n_accepted"] for d in done)
        # where a request's time goes: waiting for admission, its upload until its first round, its rounds
        wait = np.array([d["t_admit"] - d["t_submit"] for d in done]) * 1e3
        upload = np.array([d["t_first_round"] - d["t_admit"] for d in done]) * 1e3
        inrounds = np.array([d["t_done"] - d["t_first_round"] for d in done]) * 1e3
        nr = np.array([d["n_rounds"] for d in done])
        tail = lat >= np.percentile(lat, 99)
        pct = lambda a: {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99))}
        return {"rate": rate, "seconds": seconds, "requests": len(arrivals), "completed": len(done),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "grasps_per_s": acc / wall, "rounds": st["rounds"], "peak_active": st["peak_active"],
                "peak_gb": st["peak_bytes_in_use"] / 1e9, "hbm_budget_gb": budget / 1e9,
                "breakdown_ms": {"queue_wait": pct(wait), "admission_upload": pct(upload), "in_rounds": pct(inrounds),
                                 "rounds_per_request": pct(nr)},
                "tail_mean_ms": {"queue_wait": float(wait[tail].mean()), "admission_upload": float(upload[tail].mean()),
                                 "in_rounds": float(inrounds[tail].mean()), "rounds": float(nr[tail].mean())},
                "worker_s": {"admit": st["admit_s"], "round_host": st["round_host_s"], "round_wait": st["round_wait_s"],
                             "wall": wall},
                "round_ms_mean": 1e3 * (st["round_host_s"] + st["round_wait_s"]) / max(1, st["rounds"])}

    out = {"continuous_batching": [], "one_at_a_time": [],
           "workload": f"Poisson arrivals, {seconds:g} s per rate; objects drawn from {pool} generated objects "
                       "(superquadric / tool, 1,024-65,536 points) with a random hand; 100-5,000 grasps requested; "
                       f"8,192 candidate poses per request (pose cap 65,536), chunk {pose_chunk} poses "
                       f"(adaptive_chunks: up to {pose_chunk_max} poses and {chunk_pairs_max} point-pose pairs after "
                       f"the first round), {max_active} slots, HBM budget 64 GiB, {reserve_bytes / 2**30:g} GiB of the "
                       "library's pool reserved when each engine is created"}
    for rate in rates:
        out["continuous_batching"].append(stream(max_active, rate, chunk_max=0))
        out["one_at_a_time"].append(stream(1, rate, seconds=min(seconds, 5.0), chunk_max=0))
    # adaptive chunks: fewer rounds for requests that need many poses, at the price of longer rounds
    # for the requests they share them with; with the pool reserved at engine creation the fewer
    # rounds win at every rate measured (10 s per rate here, beside the fixed-chunk streams)
    if pose_chunk_max > pose_chunk:
        out["adaptive_chunks"] = [stream(max_active, rate, seconds=min(seconds, 10.0)) for rate in rates]
    # admission by HBM budget that binds: a 128 MiB budget holds only a few dozen requests' device state
    # (fixed chunks: each request holds one chunk's state)
    out["budget_gated"] = stream(max_active, max(rates), seconds=min(seconds, 10.0), budget=128 << 20, chunk_max=0)
    out["engine"] = {"max_active": max_active, "pose_chunk": pose_chunk, "pose_chunk_max": pose_chunk_max,
                     "chunk_pairs_max": chunk_pairs_max, "reserve_bytes": reserve_bytes}
    return out


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
