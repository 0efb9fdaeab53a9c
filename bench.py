#!/usr/bin/env python
"""Benchmark of the dynamic coherence-based EM ray tracer on one GB300.

Workload: highway V2I -- 2 km six-lane road with concrete barriers
(about 4.0k triangles), 200 moving vehicles with one receiver on each roof,
one roadside transmitter, 1M Fibonacci-sphere rays, 4 reflections, 28 GHz,
frames at 10 Hz. One step = one frame of the whole hot path (transform and
refit, coherence marking, shooting and bouncing, capture, dedupe,
image-method validation, field, per-receiver reduction) in COHERENT mode.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0. `value` is coherent frames/s with inputs
resident in HBM (device pointers through the C ABI); `e2e` is the same
through the C ABI with host buffers (copies inside the timed region). The
full-retrace rate, ray-segments/s, per-stage times, the roofline of the
dominant kernel, the received-power error against the FP64 oracle, and the
oracle's own rate on the host cores are reported alongside.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ray-segments/s & frames/s, coherent vs full retrace; Rx power err (dB) vs FP64"
WORKLOAD = "highway V2I: 2 km 6-lane road + barriers, 200 vehicles, 200 roof Rx, 1M rays, 4 reflections, 28 GHz, 10 Hz frames"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rays", type=int, default=1_000_000)
    ap.add_argument("--freq", type=float, default=28e9)
    ap.add_argument("--no-baseline", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched multi-transmitter workload")
    ap.add_argument("--batched-frames", type=int, default=8)
    ap.add_argument("--toy-frames", type=int, default=300)
    ap.add_argument("--no-multi-scene", action="store_true", help="skip the multi-scene batch workload")
    ap.add_argument("--no-transmission", action="store_true", help="skip the indoor transmission workload")
    ap.add_argument("--no-diffraction", action="store_true", help="skip the diffraction measurement")
    ap.add_argument("--no-toy", action="store_true", help="skip the toy-street workload")
    ap.add_argument("--no-band", action="store_true", help="skip the highway at 5.9 GHz")
    ap.add_argument("--no-roadside", action="store_true", help="skip the highway with static roadside receivers")
    ap.add_argument("--no-gradient", action="store_true", help="skip the differentiable urban workload")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args, n_frames):
    from paper_2112_07115_gb300 import scenes
    sc = scenes.highway(seed=0, n_frames=n_frames, n_rays=args.rays, max_refl=4, freq_hz=args.freq)
    return sc, scenes.fibonacci_sphere(sc.n_rays)


def config(args, sc, extra=None):
    c = {"workload": WORKLOAD, "triangles": sc.ntri, "vehicles": sc.nobj, "receivers": sc.nrx,
         "rays": sc.n_rays, "max_reflections": sc.max_refl, "freq_hz": sc.freq_hz,
         "mode": "coherent", "l2": "flushed before every timed step (256 MiB write)",
         "parallelism": f"replicas x{args.gpus}"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.lines, self.proc = [], None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# The sources a kernel is compiled from: its translation unit and the
# headers it includes (a traffic figure is stale once one of them changed).
_TRACE_SRC = ["paper_2112_07115_gb300/csrc/trace.cu", "paper_2112_07115_gb300/csrc/trace.cuh",
              "paper_2112_07115_gb300/csrc/bvh.cuh", "paper_2112_07115_gb300/csrc/dcem_internal.cuh",
              "include/dcem.h"]
KERNEL_SOURCES = {"k_trace_q": _TRACE_SRC, "k_trace": _TRACE_SRC, "k_capture": _TRACE_SRC, "k_mark": _TRACE_SRC}


_COMMENTS = re.compile(r"//[^\n]*|/\*.*?\*/", re.S)


def code_text(text: str) -> str:
    """C/C++ source without its comments and blank lines (trailing blanks
    dropped): what the compiler sees, so that a documentation edit leaves a
    capture current."""
    code = _COMMENTS.sub("", text)
    return "\n".join(ln.rstrip() for ln in code.splitlines() if ln.strip())


def src_sha(kernel: str, read=None) -> str:
    """Hash of the code (comments and blank lines dropped) of the sources a
    kernel is compiled from; `read(path)` gives a file's text (default: the
    working tree)."""
    read = read or (lambda f: open(os.path.join(ROOT, f), encoding="utf-8").read())
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        h.update(f.encode() + code_text(read(f)).encode())
    return h.hexdigest()[:16]


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU baseline."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_metrics(kernel: str, workload: str, mode: str):
    """The one-launch ncu counters of `kernel` on `workload` in `mode`
    (profiles/ncu_metrics.json), if they were taken on the current source:
    DRAM and L2 bytes per launch, L2 hit rate, threads per warp instruction."""
    p = os.path.join(ROOT, "profiles", "ncu_metrics.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(f"{kernel}|{workload}|{mode}")
    if not e or kernel not in KERNEL_SOURCES or e.get("src_sha") != src_sha(kernel):
        return None
    return e


def _measured_forms(kernel, workload, mode, ms, peak):
    """DRAM and L2 forms of a kernel's bandwidth from its ncu counters and the
    kernel's CUDA-event time (ms), plus the L2 hit rate and warp execution
    efficiency; None without a current capture."""
    e = ncu_metrics(kernel, workload, mode)
    if not e:
        return None
    dram = e["dram_bytes"] / (ms * 1e-3) / 1e9
    l2 = e["lts_bytes"] / (ms * 1e-3) / 1e9
    return {"dram_bytes_per_launch": e["dram_bytes"], "dram_gbs": round(dram, 1),
            "dram_frac_of_hbm": round(dram / peak, 4), "l2_bytes_per_launch": e["lts_bytes"],
            "l2_gbs": round(l2, 1), "l2_hit_rate_pct": e["l2_hit_pct"],
            "warp_exec_efficiency": round(e["threads_per_inst"] / 32.0, 4),
            "threads_per_warp_instruction": e["threads_per_inst"], "profile": e.get("profile")}


def max_over_ranks(values, device=None):
    """Element-wise maximum of per-rank timings over the process group (the
    values themselves when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


# ---------------------------------------------------------------- ours
def run_ours(args):
    import ctypes as C
    import torch
    from paper_2112_07115_gb300 import build as B
    from paper_2112_07115_gb300 import dcem

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    K, W = args.steps, args.warmup
    sc, rays = workload(args, n_frames=W + K + 2)
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", local)
    xf_d = torch.from_numpy(sc.xf).to(dev)
    rx_d = torch.from_numpy(sc.rx).to(dev)
    tx = sc.tx
    nrx = sc.nrx
    max_paths = 1 << 17
    field_d = torch.empty((nrx, 2), dtype=torch.float64, device=dev)
    pc_d = torch.empty(nrx, dtype=torch.float64, device=dev)
    pi_d = torch.empty(nrx, dtype=torch.float64, device=dev)
    paths_d = torch.empty(max_paths * C.sizeof(dcem.Path), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def new_result():
        r = dcem.Result()
        r.ptr_kind = dcem.PTR_DEVICE
        r.max_paths = max_paths
        r.field, r.p_coh_dbm, r.p_inc_dbm = field_d.data_ptr(), pc_d.data_ptr(), pi_d.data_ptr()
        r.paths = paths_d.data_ptr()
        return r

    def run(mode, frames, timed, timing, graphs=True):
        # timing 2: only the closest-hit kernel is bracketed by events (the
        # timed loops); timing 1: every stage (the instrumented pass)
        s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
        s.set_rays(rays)
        s.set_graph_replay(graphs)
        prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, mode=mode, timing=timing)
        res = new_result()
        stats, ms = [], []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i, f in enumerate(frames):
            is_t = i >= W and timed
            if is_t:
                flush.zero_()
            e0.record(stream)
            dcem.dcem_scene_update_transforms(s.h, xf_d[f])
            rc = dcem.dcem_trace_frame(s.h, tx, rx_d[f], prm, res)
            e1.record(stream)
            e1.synchronize()
            if rc != dcem.OK:
                raise dcem.DcemError(rc, f"frame {f}")
            if is_t:
                ms.append(e0.elapsed_time(e1))
                stats.append(dcem.stats_dict(res.stats))
        return s, ms, stats

    frames = list(range(1, W + K + 1))
    # coherent (the headline)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    s_coh, ms_coh, st_coh = run(dcem.MODE_COHERENT, frames, True, 2)
    torch.cuda.synchronize()
    # full retrace of the same frames
    s_full, ms_full, st_full = run(dcem.MODE_FULL, frames, True, 2)
    torch.cuda.synchronize()
    # the coherent frames again, every operation launched on its own
    s_dir, ms_dir, _ = run(dcem.MODE_COHERENT, frames, True, 2, graphs=False)
    s_dir.close()
    clocks = clk.stop()
    # instrumented pass over the same frames (not timed): per-stage breakdown
    si, _, ist_coh = run(dcem.MODE_COHERENT, frames, True, 1)
    si.close()
    si, _, ist_full = run(dcem.MODE_FULL, frames, True, 1)
    si.close()
    t_coh = sum(ms_coh) / 1e3
    t_full = sum(ms_full) / 1e3
    t_dir = sum(ms_dir) / 1e3
    t_coh, t_full, t_dir = max_over_ranks([t_coh, t_full, t_dir], dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    fps_coh = world * K / t_coh
    fps_full = world * K / t_full
    seg_full = world * sum(x["segments_traced"] for x in st_full) / t_full
    seg_coh_traced = world * sum(x["segments_traced"] for x in st_coh) / t_coh
    seg_coh_repr = world * sum(x["segments_traced"] + x["segments_reused"] for x in st_coh) / t_coh

    # stage times and roofline of the dominant kernel (coherent frames)
    stage_names = dcem.STAGES
    mean_stage = {n: float(np.mean([x["ms_stage"][n] for x in ist_coh])) for n in stage_names}
    mean_stage_full = {n: float(np.mean([x["ms_stage"][n] for x in ist_full])) for n in stage_names}
    dom = max(["mark", "trace", "capture", "dedupe", "validate", "reduce"], key=lambda n: mean_stage[n])
    # the closest-hit kernel's own time inside the timed loops
    trace_timed = float(np.mean([x["ms_stage"]["trace"] for x in st_coh]))
    trace_timed_full = float(np.mean([x["ms_stage"]["trace"] for x in st_full]))
    mean_stage["trace"] = trace_timed
    mean_stage_full["trace"] = trace_timed_full
    R = sc.n_rays
    peak, peak_kind = measured_peaks()

    def bytes_trace(x):
        q = x["rays_retraced"]
        return (q * (32 + 4) + x["segments_traced"] * 36 + x["node_visits"] * 64 + x["tri_tests"] * 48)

    def bytes_mark(x):
        examined = x["segments_reused"] + x["rays_retraced"]
        return R * 8 + examined * 32 + x["rays_retraced"] * 4

    def bytes_capture(x):
        # log entry (origin, D, direction, t) and segment count per tested
        # segment, 8 B per emitted candidate
        return x["segments_traced"] * 36 + (x["candidates"] - x["candidates_reused"]) * 8

    tname = ["k_trace", "k_trace_q", "k_trace_qg"][st_coh[-1]["trace_kernel"]]
    kern = {"trace": (tname, bytes_trace), "mark": ("k_mark", bytes_mark), "capture": ("k_capture", bytes_capture)}
    roof = None
    if dom in kern:
        kname, fb = kern[dom]
        b = float(np.mean([fb(x) for x in st_coh]))
        ach = b / (mean_stage[dom] * 1e-3) / 1e9
        meas = _measured_forms(kname, "highway", "coherent", mean_stage[dom], peak)
        roof = {"kernel": kname, "bound": "latency", "achieved": round(ach, 1), "peak": peak,
                "unit": "GB/s", "frac": round(ach / peak, 4), "peak_kind": peak_kind,
                "bytes": "algorithmic: 64 B per node visit and 48 B per triangle test as if read, plus ray "
                         "state and log; nodes come from shared memory and triangles from L2, so DRAM "
                         "traffic is far lower and the kernel is bound by latency and issue, not HBM",
                "algorithmic_bytes_per_launch": int(b),
                "traffic": (meas or {}).get("dram_bytes_per_launch"),
                "measured": meas,
                "traffic_note": "ncu dram__bytes_read+write of one launch on the current source"
                                if meas else "no ncu capture on the current source"}
    # full-retrace traversal roofline (context)
    bf = float(np.mean([bytes_trace(x) for x in st_full]))
    roof_full_trace = {"kernel": tname, "bound": "latency",
                       "achieved": round(bf / (mean_stage_full["trace"] * 1e-3) / 1e9, 1),
                       "unit": "GB/s", "frac": None, "bytes": "algorithmic (as the headline roofline)"}
    roof_full_trace["frac"] = round(roof_full_trace["achieved"] / peak, 4)
    roof_full_trace["measured"] = _measured_forms(tname, "highway", "full", mean_stage_full["trace"], peak)
    seg_mean = float(np.mean([x["segments_traced"] for x in st_full]))
    nodes_per_seg = float(np.mean([x["node_visits"] for x in st_full])) / max(seg_mean, 1)
    tris_per_seg = float(np.mean([x["tri_tests"] for x in st_full])) / max(seg_mean, 1)

    # received power error vs the FP64 oracle on the same path keys (last frame)
    err = None
    if rank == 0:
        err = power_error_vs_oracle(sc, s_coh, frames[-1], max_paths, paths_d, pc_d, pi_d, res_n=st_coh[-1])

    # field derivatives over the last frame's paths (device in, device out)
    grads = grad_timing(s_coh, sc, rx_d[frames[-1]], paths_d, int(st_coh[-1]["paths_valid"]), stream, dev)

    # validation arithmetic: FP64 and double-float, full frames with every
    # stage timed, each checked against the oracle on its last frame
    precs = {}
    if rank == 0:
        sub = frames[-min(len(frames), 60):]
        for name, prec in (("f64", dcem.PREC_F64), ("df32", dcem.PREC_DF32)):
            sp = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
            sp.set_rays(rays)
            prm_p = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, mode=dcem.MODE_FULL,
                                        timing=1, prec=prec)
            res_p = new_result()
            vms, last = [], None
            for f in sub:
                dcem.dcem_scene_update_transforms(sp.h, xf_d[f])
                rc = dcem.dcem_trace_frame(sp.h, tx, rx_d[f], prm_p, res_p)
                if rc != dcem.OK:
                    raise dcem.DcemError(rc, f"frame {f} ({name})")
                last = dcem.stats_dict(res_p.stats)
                vms.append(last["ms_stage"]["validate"])
            torch.cuda.synchronize()
            e_p = power_error_vs_oracle(sc, sp, sub[-1], max_paths, paths_d, pc_d, pi_d, res_n=last)
            precs[name] = {"validate_ms": round(float(np.mean(vms[1:] or vms)), 4),
                           "max_abs_p_coh_db": e_p["max_abs_p_coh"], "max_abs_p_inc_db": e_p["max_abs_p_inc"],
                           "max_len_err_m": e_p["max_len_err_m"], "paths": e_p["paths"]}
            sp.close()

    batched = None
    if not args.no_batched:
        batched = run_batched(args, stream, dev, world, flush)
    multi = None
    if not args.no_multi_scene:
        multi = run_multi_scene(args, stream, dev, world, flush)
    trans = None
    if not args.no_transmission:
        trans = run_transmission(args, stream, dev, world, flush, rank)
    diff = None
    if not args.no_diffraction:
        diff = run_diffraction(args, sc, rays, stream, dev, world, flush)
        diff["orders"] = run_diffraction_orders(args, sc, stream, dev, world, flush)

    toy = None
    if not args.no_toy:
        toy = run_toy(args, stream, dev, world, flush, rank)
    band = None
    if not args.no_band:
        band = run_band(args, stream, dev, world, flush, rank)
    roadside = None
    if not args.no_roadside:
        roadside = run_roadside(args, stream, dev, world, flush, rank)
    gradw = None
    if not args.no_gradient:
        gradw = run_gradient(args, stream, dev, world, flush, rank)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, sc, rays, stream, W, K, world, dev, flush)
    base = None
    if rank == 0 and world == 1 and not args.no_baseline:
        base = cpu_baseline(sc, rays, frames[W])
    launches = int(np.mean([x["kernel_launches"] for x in st_coh]))
    s_coh.close()
    s_full.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(fps_coh, 2), "unit": "frames/s", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": round(1e3 * t_coh / K, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 geometry / f64 field",
            "data": "synthetic (seeded highway generator)", "impl": "ours",
            "config": config(args, sc),
            "coherent": {"frames_per_s": round(fps_coh, 2), "ms_per_frame": round(1e3 * t_coh / K, 4),
                         "ray_segments_traced_per_s": round(seg_coh_traced, 0),
                         "ray_segments_represented_per_s": round(seg_coh_repr, 0),
                         "rays_retraced_frac": round(float(np.mean([x["rays_retraced"] for x in st_coh])) / R, 4),
                         "segments_reused_frac": round(float(np.mean(
                             [x["segments_reused"] / max(1, x["segments_reused"] + x["segments_traced"])
                              for x in st_coh])), 4),
                         "stage_ms": {k: round(v, 4) for k, v in mean_stage.items()},
                         "stage_ms_note": "trace: CUDA events around the closest-hit kernel inside the timed "
                                          "loop; other stages: an instrumented pass over the same frames "
                                          "(events around every stage, not timed)",
                         "frame_ms_p50_max": [round(float(np.median(ms_coh)), 4), round(float(max(ms_coh)), 4)],
                         "nodes_per_segment": round(float(np.sum([x["node_visits"] for x in st_coh])) /
                                                    max(1.0, float(np.sum([x["segments_traced"] for x in st_coh]))), 2),
                         "max_segment_nodes": int(max(x["max_segment_nodes"] for x in st_coh)),
                         "bvh_rebuilds": int(sum(x["bvh_rebuilt"] for x in st_coh))},
            "gradients": grads,
            "validation_precision": precs,
            "toy_street": toy,
            "highway_5p9ghz": band,
            "highway_roadside_rx": roadside,
            "differentiable_urban": gradw,
            "batched": batched,
            "multi_scene": multi,
            "transmission": trans,
            "diffraction": diff,
            "full": {"frames_per_s": round(fps_full, 2), "ms_per_frame": round(1e3 * t_full / K, 4),
                     "ray_segments_per_s": round(seg_full, 0), "segments_per_frame": int(seg_mean),
                     "nodes_per_segment": round(nodes_per_seg, 2), "tris_per_segment": round(tris_per_seg, 2),
                     "max_segment_nodes": int(max(x["max_segment_nodes"] for x in st_full)),
                     "stage_ms": {k: round(v, 4) for k, v in mean_stage_full.items()},
                     "frame_ms_p50_max": [round(float(np.median(ms_full)), 4), round(float(max(ms_full)), 4)],
                     "trace_roofline": roof_full_trace},
            "graph_replay": {"frames_replayed_frac": round(float(np.mean([x["graph_replayed"] for x in st_coh])), 4),
                             "direct_launch_frames_per_s": round(world * K / t_dir, 2),
                             "note": "coherent frames launched as one replayed CUDA graph each (value) vs "
                                     "operation by operation (direct)"},
            "coherent_speedup": round(fps_coh / fps_full, 3),
            "paths_per_frame": int(np.mean([x["paths_valid"] for x in st_coh])),
            "rx_power_err_db": err,
            "roofline": roof,
            "e2e": e2e,
            "cpu_baseline": base,
            "clocks": clocks,
            "gpu_launches": launches * K,
            "gpu_launches_per_step": launches,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _frames_timed(s, sc, frames, prm, stream, flush, xf_d, rx_d, res, warmup):
    """Runs update + trace over `frames` (device inputs and outputs), the L2
    flushed before each; returns (ms per timed frame, stats per timed frame)."""
    import torch
    from paper_2112_07115_gb300 import dcem
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, st = [], []
    for i, f in enumerate(frames):
        flush.zero_()
        e0.record(stream)
        if sc.nobj:
            dcem.dcem_scene_update_transforms(s.h, xf_d[f])
        rc = dcem.dcem_trace_frame(s.h, sc.tx, rx_d[f], prm, res)
        e1.record(stream)
        e1.synchronize()
        if rc != dcem.OK:
            raise dcem.DcemError(rc, f"frame {f}")
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
            st.append(dcem.stats_dict(res.stats))
    return ms, st


def _device_result(nrx, max_paths, dev):
    import ctypes as C
    import torch
    from paper_2112_07115_gb300 import dcem
    bufs = (torch.empty((max(nrx, 1), 2), dtype=torch.float64, device=dev),
            torch.empty(max(nrx, 1), dtype=torch.float64, device=dev),
            torch.empty(max(nrx, 1), dtype=torch.float64, device=dev),
            torch.empty(max_paths * C.sizeof(dcem.Path), dtype=torch.uint8, device=dev))
    r = dcem.Result()
    r.ptr_kind = dcem.PTR_DEVICE
    r.max_paths = max_paths
    r.field, r.p_coh_dbm, r.p_inc_dbm, r.paths = [x.data_ptr() for x in bufs]
    return r, bufs


def _mode_summary(ms, st, world, n_rays, dev, workload=None, mode=None):
    """Rates of timed frames (ms: CUDA-event times, st: their stats); with
    `workload` and `mode`, the closest-hit kernel's ncu counters (DRAM and L2
    bytes, L2 hit rate, warp execution efficiency) when a capture of the
    current source exists."""
    t = max_over_ranks([sum(ms) / 1e3], dev)[0]
    K = len(ms)
    segs = float(np.mean([x["segments_traced"] for x in st]))
    rep = float(np.mean([x["segments_traced"] + x["segments_reused"] for x in st]))
    return {"frames_per_s": round(world * K / t, 2), "ms_per_frame": round(1e3 * t / K, 4),
            "ray_segments_traced_per_s": round(world * K * segs / t, 0),
            "ray_segments_represented_per_s": round(world * K * rep / t, 0),
            "rays_retraced_frac": round(float(np.mean([x["rays_retraced"] for x in st])) / max(n_rays, 1), 4),
            "keys_reused_frac": round(float(np.mean([x["keys_reused"] / max(1, x["unique_candidates"])
                                                     for x in st])), 4),
            "closest_hit_ms": round(float(np.mean([x["ms_stage"]["trace"] for x in st])), 4),
            "paths_per_frame": int(np.mean([x["paths_valid"] for x in st])),
            "closest_hit_measured": (_measured_forms("k_trace_q", workload, mode,
                                                     float(np.mean([x["ms_stage"]["trace"] for x in st])),
                                                     measured_peaks()[0]) if workload else None)}


def run_toy(args, stream, dev, world, flush, rank, warmup=5):
    """The toy street (58 triangles, 4 moving metal vehicles, 8 static
    receivers, 10k rays, 3 reflections, 28 GHz, 10 frames at 10 Hz): full and
    coherent frames over the scene's frames in turn, L2 flushed before each;
    every frame's received power against the FP64 oracle (its own trace,
    dedupe and validation)."""
    import torch
    from oracle import oracle as O
    from paper_2112_07115_gb300 import dcem, scenes
    sc = scenes.toy_street()
    rays = scenes.fibonacci_sphere(sc.n_rays)
    K = max(args.toy_frames, 10)
    frames = [1 + i % (sc.nframes - 1) for i in range(warmup + K)]
    xf_d = torch.from_numpy(sc.xf).to(dev)
    rx_d = torch.from_numpy(sc.rx).to(dev)
    res, bufs = _device_result(sc.nrx, 1 << 14, dev)
    out = {"workload": "toy street: %d triangles (2 buildings, 4 moving metal vehicles), %d static Rx, %d rays, "
                       "%d reflections, 28 GHz, %d frames at 10 Hz taken in turn" % (sc.ntri, sc.nrx, sc.n_rays,
                                                                                      sc.max_refl, sc.nframes)}
    for name, mode in (("full", dcem.MODE_FULL), ("coherent", dcem.MODE_COHERENT)):
        s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
        s.set_rays(rays)
        prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, mode=mode, timing=2)
        ms, st = _frames_timed(s, sc, frames, prm, stream, flush, xf_d, rx_d, res, warmup)
        s.close()
        out[name] = _mode_summary(ms, st, world, sc.n_rays, dev, "toy", name)
    out["coherent_speedup"] = round(out["coherent"]["frames_per_s"] / out["full"]["frames_per_s"], 3)
    if rank == 0:
        # every frame in order, coherent, against the oracle
        s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
        s.set_rays(rays)
        prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, mode=dcem.MODE_COHERENT)
        oprm = O.OracleParams(freq_hz=sc.freq_hz, n_rays=sc.n_rays, max_refl=sc.max_refl)
        dc, di, diff, npaths = 0.0, 0.0, 0, 0
        for f in range(sc.nframes):
            s.update_transforms(sc.xf[f])
            fr = s.trace(sc.tx, sc.rx[f], prm)
            ref = O.frame(sc, f, rays, oprm)
            fin = np.isfinite(ref.p_coh_dbm) & np.isfinite(fr.p_coh_dbm)
            dc = max(dc, float(np.max(np.abs(ref.p_coh_dbm[fin] - fr.p_coh_dbm[fin]), initial=0.0)))
            dc_inf = np.isfinite(ref.p_coh_dbm) != np.isfinite(fr.p_coh_dbm)
            di = max(di, float(np.max(np.abs(ref.p_inc_dbm[fin] - fr.p_inc_dbm[fin]), initial=0.0)))
            want = {tuple(k) for k, p in zip(ref.keys.tolist(), ref.paths) if p["valid"]}
            got = set()
            for p in fr.paths:
                got.add((int(p["rx"]), int(p["depth"])) + tuple(int(x) for x in p["tri"][:sc.max_refl]))
            diff += len(got ^ want) + int(dc_inf.sum())
            npaths += len(got)
        s.close()
        out["rx_power_err_db"] = {"frames": sc.nframes, "paths": npaths, "max_abs_p_coh": dc, "max_abs_p_inc": di,
                                  "path_set_differences": diff,
                                  "against": "FP64 oracle frames (own trace, dedupe, validation), all frames"}
    return out


def run_band(args, stream, dev, world, flush, rank, freq=5.9e9, warmup=5):
    """The headline highway frames at 5.9 GHz (1M rays, 4 reflections, 200
    roof receivers): coherent and full, L2 flushed before each frame; the last
    frame's paths re-validated by the FP64 oracle."""
    import torch
    from paper_2112_07115_gb300 import dcem, scenes
    K = min(args.steps, 100)
    sc = scenes.highway(seed=0, n_frames=warmup + K + 2, n_rays=args.rays, max_refl=4, freq_hz=freq)
    rays = scenes.fibonacci_sphere(sc.n_rays)
    frames = list(range(1, warmup + K + 1))
    xf_d = torch.from_numpy(sc.xf).to(dev)
    rx_d = torch.from_numpy(sc.rx).to(dev)
    max_paths = 1 << 17
    res, bufs = _device_result(sc.nrx, max_paths, dev)
    out = {"workload": "highway V2I as the headline, at %.1f GHz" % (freq / 1e9)}
    for name, mode in (("full", dcem.MODE_FULL), ("coherent", dcem.MODE_COHERENT)):
        s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
        s.set_rays(rays)
        prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, mode=mode, timing=2)
        ms, st = _frames_timed(s, sc, frames, prm, stream, flush, xf_d, rx_d, res, warmup)
        wl = "highway_5p9ghz" if abs(freq - 5.9e9) < 1e6 else None
        out[name] = _mode_summary(ms, st, world, sc.n_rays, dev, wl, name)
        if name == "coherent" and rank == 0:
            out["rx_power_err_db"] = power_error_vs_oracle(sc, s, frames[-1], max_paths, bufs[3], bufs[1], bufs[2],
                                                           res_n=st[-1])
        s.close()
    out["coherent_speedup"] = round(out["coherent"]["frames_per_s"] / out["full"]["frames_per_s"], 3)
    return out


def run_roadside(args, stream, dev, world, flush, rank, warmup=5):
    """The headline highway with its 200 receivers as static roadside units
    (2.5 m high, 2 m beyond the outer barriers) instead of on the vehicles'
    roofs: the same moving traffic, so the coherent frame re-tests no reused
    segment against moved receivers and copies the validation of keys that
    no moved object touches. Coherent and full frames (L2 flushed before
    each), the stage times of an instrumented pass of both, and the last
    frame's paths re-validated by the FP64 oracle."""
    import torch
    from paper_2112_07115_gb300 import dcem, scenes
    K = min(args.steps, 100)
    sc = scenes.highway(seed=0, n_frames=warmup + K + 2, n_rays=args.rays, max_refl=4, freq_hz=args.freq,
                        roadside_rx=200)
    rays = scenes.fibonacci_sphere(sc.n_rays)
    frames = list(range(1, warmup + K + 1))
    xf_d = torch.from_numpy(sc.xf).to(dev)
    rx_d = torch.from_numpy(sc.rx).to(dev)
    max_paths = 1 << 17
    res, bufs = _device_result(sc.nrx, max_paths, dev)
    out = {"workload": "highway V2I as the headline (1M rays, 4 reflections, 200 moving vehicles), 200 static "
                       "roadside receivers instead of roof receivers"}
    for name, mode in (("full", dcem.MODE_FULL), ("coherent", dcem.MODE_COHERENT)):
        s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
        s.set_rays(rays)
        prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, mode=mode, timing=2)
        ms, st = _frames_timed(s, sc, frames, prm, stream, flush, xf_d, rx_d, res, warmup)
        out[name] = _mode_summary(ms, st, world, sc.n_rays, dev, "roadside", name)
        if name == "coherent" and rank == 0:
            out["rx_power_err_db"] = power_error_vs_oracle(sc, s, frames[-1], max_paths, bufs[3], bufs[1], bufs[2],
                                                           res_n=st[-1])
        s.close()
        # instrumented pass (events around every stage; not timed)
        s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
        s.set_rays(rays)
        prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, mode=mode, timing=1)
        _, sti = _frames_timed(s, sc, frames[:warmup + 10], prm, stream, flush, xf_d, rx_d, res, warmup)
        s.close()
        out[name]["stage_ms"] = {n: round(float(np.mean([x["ms_stage"][n] for x in sti])), 4) for n in dcem.STAGES}
    out["coherent_speedup"] = round(out["coherent"]["frames_per_s"] / out["full"]["frames_per_s"], 3)
    return out


def run_gradient(args, stream, dev, world, flush, rank, reps=10):
    """The differentiable urban workload: the urban grid (10 x 10 blocks, 1000
    moving metal vehicles) with eight (eps_r, sigma) classes, one roadside
    transmitter with 1M rays, 4 reflections, 256 roadside receivers; the
    gradient of the summed received power (dB) with respect to every
    material's (eps_r, sigma) and every vehicle's (x, y) over one frame's
    path topology, by the adjoint kernel (dcem_path_adjoint: field, powers,
    Jacobian and the vector-Jacobian product) and, for comparison, the
    forward-mode kernel; a sample of derivatives against the FP64 oracle's
    central differences."""
    import ctypes as C
    import torch
    from oracle import oracle as O
    from paper_2112_07115_gb300 import dcem, scenes
    sc = scenes.urban_gradient(n_rays=args.rays)
    f = 1
    s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(sc.n_rays))
    s.update_transforms(sc.xf[f])
    prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz)
    fr = s.trace(sc.tx, sc.rx[f], prm)
    paths = fr.paths
    n = paths.shape[0]
    nrx = sc.nrx
    npar = dcem.dcem_scene_gradient_size(s.h)
    pd = torch.from_numpy(paths.view(np.uint8).copy()).to(dev)
    rxd = torch.from_numpy(sc.rx[f]).to(dev)
    th = torch.from_numpy(s.theta(sc.xf[f])).to(dev)
    fin = np.isfinite(fr.p_coh_dbm)
    pbar = torch.from_numpy(fin.astype(np.float64)).to(dev)   # d(sum of finite P_coh[dBm]) / d P
    fd_ = torch.empty((nrx, 2), dtype=torch.float64, device=dev)
    pc_ = torch.empty(nrx, dtype=torch.float64, device=dev)
    dfd = torch.empty((nrx, npar, 2), dtype=torch.float64, device=dev)
    dpd = torch.empty((nrx, npar), dtype=torch.float64, device=dev)
    tb = torch.empty(npar, dtype=torch.float64, device=dev)

    def adj():
        return dcem.dcem_path_adjoint(s.h, sc.tx, rxd, pd.data_ptr(), prm, dcem.PTR_DEVICE, th.data_ptr(),
                                      pbar.data_ptr(), fd_.data_ptr(), pc_.data_ptr(), dfd.data_ptr(),
                                      dpd.data_ptr(), tb.data_ptr(), n_paths=n)

    def fwd():
        return dcem.dcem_path_gradients(s.h, sc.tx, rxd, pd.data_ptr(), prm, dcem.PTR_DEVICE, fd_.data_ptr(),
                                         dfd.data_ptr(), dpd.data_ptr(), n_paths=n)

    out = {"workload": "urban grid 10x10 blocks, %d triangles, %d moving metal vehicles, 8 (eps_r, sigma) "
                       "classes, 1 Tx with %d rays, %d reflections, %d roadside Rx; d(sum P_coh[dBm]) / d theta "
                       "over one frame's paths" % (sc.ntri, sc.nobj, sc.n_rays, sc.max_refl, nrx),
           "paths": int(n), "receivers_with_paths": int(fin.sum()), "params": int(npar)}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, fn in (("adjoint", adj), ("forward_mode", fwd)):
        for _ in range(3):
            if fn() != dcem.OK:
                raise dcem.DcemError(dcem.ERR_ARG, name)
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[name + "_ms"] = round(float(np.mean(ts)), 4)
    adj()
    torch.cuda.synchronize()
    g = tb.cpu().numpy()
    dE = dfd.cpu().numpy()
    dE = dE[..., 0] + 1j * dE[..., 1]
    nm2 = 2 * sc.materials.shape[0]
    out["grad_sum_p_coh"] = {"nonzero": int(np.count_nonzero(g)), "max_abs_material": float(np.abs(g[:nm2]).max()),
                             "max_abs_vehicle_xy_db_per_m": float(np.abs(g[nm2:]).max(initial=0.0))}
    # a sample of d E / d theta against the oracle's central differences (FP64)
    if rank == 0 and n:
        keys = np.full((n, 2 + sc.max_refl), -1, np.int32)
        keys[:, 0], keys[:, 1] = paths["rx"], paths["depth"]
        keys[:, 2:] = np.where(np.arange(sc.max_refl)[None] < paths["depth"][:, None],
                               paths["tri"][:, :sc.max_refl], -1)
        wt = np.asarray(O.transform(sc.tris, sc.tri_obj, sc.xf[f]), np.float64).reshape(-1, 3, 3)
        mats = sc.materials.astype(np.float64)
        oprm = O.OracleParams(freq_hz=sc.freq_hz, n_rays=sc.n_rays, max_refl=sc.max_refl)
        nz = np.flatnonzero(np.abs(dE).max(0))
        rng = np.random.default_rng(0)
        pick = np.concatenate([rng.permutation(nz[nz < nm2])[:6], rng.permutation(nz[nz >= nm2])[:6]])
        base = O.path_amp_d(wt, sc.tri_mat, mats, sc.tx, sc.rx[f], keys, oprm)
        worst, checked = 0.0, 0
        for i in pick:
            tp, tm, mp, mm = wt.copy(), wt.copy(), mats.copy(), mats.copy()
            if i < nm2:
                h = 1e-6 * max(1.0, abs(mats[i // 2, i % 2]))
                mp[i // 2, i % 2] += h
                mm[i // 2, i % 2] -= h
            else:
                h = 1e-6
                sel = sc.tri_obj == (i - nm2) // 2
                tp[sel, :, (i - nm2) % 2] += h
                tm[sel, :, (i - nm2) % 2] -= h
            pp = O.path_amp_d(tp, sc.tri_mat, mp, sc.tx, sc.rx[f], keys, oprm)
            pm = O.path_amp_d(tm, sc.tri_mat, mm, sc.tx, sc.rx[f], keys, oprm)
            ok = (base["valid"] != 0) & (pp["valid"] != 0) & (pm["valid"] != 0)
            for q in (pp, pm):
                q["valid"] = ok
            fdv = (O.field_of(keys, pp, nrx) - O.field_of(keys, pm, nrx)) / (2 * h)
            scale = np.abs(dE).max(1)
            for r in np.flatnonzero(np.abs(fdv) > 0):
                err = abs(dE[r, i] - fdv[r]) / (abs(fdv[r]) + 1e-9 * scale[r])
                worst = max(worst, float(err))
                checked += 1
        out["oracle_check"] = {"params_sampled": int(len(pick)), "elements": checked,
                               "max_rel_err": worst, "bar": 1e-4,
                               "note": "per element |dE - fd| / (|fd| + 1e-9 max_r |dE|), central differences "
                                       "of the FP64 oracle's path amplitudes (h = 1e-6)"}
    s.close()
    return out


def run_batched(args, stream, dev, world, flush, warmup=2):
    """The batched multi-transmitter workload: an urban grid (10 x 10 blocks,
    ~51k static and 10k moving triangles, 1000 vehicles), 64 roadside
    transmitters with log-uniform budgets of 64k-2M rays (~31M rays in all),
    4096 receivers (262,144 links), 5 reflections, every transmitter traced in
    the same launches per frame (dcem_trace_links). Full and coherent frames,
    L2 flushed before each, timed with CUDA events; max over ranks."""
    import ctypes as C
    import torch
    from paper_2112_07115_gb300 import dcem, scenes
    K = args.batched_frames
    sc = scenes.urban_grid(seed=0, n_frames=warmup + K + 1)
    txs, budgets = sc.meta["tx"], sc.meta["budgets"]
    sets = [scenes.fibonacci_sphere(n) for n in budgets]
    nl = len(budgets) * sc.nrx
    xf_d = torch.from_numpy(sc.xf).to(dev)
    rx_d = torch.from_numpy(sc.rx).to(dev)
    max_paths = 1 << 22
    field_d = torch.empty((nl, 2), dtype=torch.float64, device=dev)
    pc_d = torch.empty(nl, dtype=torch.float64, device=dev)
    pi_d = torch.empty(nl, dtype=torch.float64, device=dev)
    paths_d = torch.empty(max_paths * C.sizeof(dcem.Path), dtype=torch.uint8, device=dev)
    out = {"workload": "urban grid 10x10 blocks (100 m pitch, 20 m streets), %d triangles (%d moving), "
                       "%d vehicles, %d Tx with %d-%d rays each (%d rays), %d Rx, %d links, %d reflections, "
                       "28 GHz" % (sc.ntri, int((sc.tri_obj >= 0).sum()), sc.nobj, len(budgets), min(budgets),
                                   max(budgets), sum(budgets), sc.nrx, nl, sc.max_refl)}
    # closest-hit configuration: the autotuner on the first frame (untimed)
    s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
    s.set_ray_sets(sets)
    s.update_transforms(sc.xf[1])
    tune = s.autotune(txs, sc.rx[1], dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz), reps=1)
    s.close()
    out["closest_hit_config"] = {"kernel": ["binary nodes, global", "4-wide copy, shared memory",
                                            "4-wide copy, global"][tune[0]],
                                 "block": tune[1], "stack": tune[2], "chosen_by": "dcem_scene_autotune"}
    for name, mode in (("full", dcem.MODE_FULL), ("coherent", dcem.MODE_COHERENT)):
        s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
        s.set_ray_sets(sets)
        s.set_trace_config(tune[0], tune[1] if tune[0] != 1 else 256, tune[2] if tune[0] != 1 else 24)
        prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, mode=mode, timing=2)
        res = dcem.Result()
        res.ptr_kind = dcem.PTR_DEVICE
        res.max_paths = max_paths
        res.field, res.p_coh_dbm, res.p_inc_dbm = field_d.data_ptr(), pc_d.data_ptr(), pi_d.data_ptr()
        res.paths = paths_d.data_ptr()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, st = [], []
        for i in range(warmup + K):
            f = i + 1
            flush.zero_()
            e0.record(stream)
            dcem.dcem_scene_update_transforms(s.h, xf_d[f])
            rc = dcem.dcem_trace_links(s.h, txs, rx_d[f], prm, res)
            e1.record(stream)
            e1.synchronize()
            if rc != dcem.OK:
                raise dcem.DcemError(rc, f"batched frame {f}")
            if i >= warmup:
                ms.append(e0.elapsed_time(e1))
                st.append(dcem.stats_dict(res.stats))
        s.close()
        t = max_over_ranks([sum(ms) / 1e3], dev)[0]
        segs = float(np.mean([x["segments_traced"] for x in st]))
        trace_ms = float(np.mean([x["ms_stage"]["trace"] for x in st]))
        tb = float(np.mean([x["rays_retraced"] * 36 + x["segments_traced"] * 36 + x["node_visits"] * 64 +
                            x["tri_tests"] * 48 for x in st]))
        peak, _ = measured_peaks()
        out[name] = {"frames_per_s": round(world * K / t, 3), "ms_per_frame": round(1e3 * t / K, 3),
                     "trace_roofline": {"bound": "latency",
                                        "achieved_algorithmic": round(tb / (trace_ms * 1e-3) / 1e9, 1),
                                        "unit": "GB/s",
                                        "algorithmic_over_hbm_peak": round(tb / (trace_ms * 1e-3) / 1e9 / peak, 4),
                                        "note": "algorithmic bytes of the closest-hit kernel, served mostly "
                                                "by L2; a ratio to the HBM peak above 1 counts L2 and "
                                                "shared-memory bytes, not an HBM fraction"},
                     "rays_per_s": round(world * K * sum(budgets) / t, 0),
                     "segments_traced_per_frame": int(segs),
                     "ray_segments_traced_per_s": round(world * K * segs / t, 0),
                     "links_per_s": round(world * K * nl / t, 0),
                     "paths_per_frame": int(np.mean([x["paths_valid"] for x in st])),
                     "unique_candidates_per_frame": int(np.mean([x["unique_candidates"] for x in st])),
                     "closest_hit_ms": round(trace_ms, 3),
                     "closest_hit_kernel": ["k_trace", "k_trace_q", "k_trace_qg"][st[-1]["trace_kernel"]],
                     "nodes_per_segment": round(float(np.mean([x["node_visits"] for x in st])) / max(segs, 1.0), 2),
                     "segments_reused_frac": round(float(np.mean(
                         [x["segments_reused"] / max(1, x["segments_reused"] + x["segments_traced"]) for x in st])), 4),
                     "graph_replayed_frac": round(float(np.mean([x["graph_replayed"] for x in st])), 3)}
    return out


def run_multi_scene(args, stream, dev, world, flush, warmup=2):
    """The multi-scene batch: 32 independent urban grids (1k-200k triangles,
    10-2000 vehicles, 1-16 transmitters each with 16k-512k rays; 1.2M
    triangles, 296 transmitters, 43.5M rays, 367k links in all), 4
    reflections, refit and traced together (dcem_batch_update_transforms +
    dcem_batch_trace: one graph launch per frame once the plans repeat),
    device outputs, L2 flushed before each frame. Also the same frames with
    the scenes traced one after another (dcem_trace_links each) for the
    concurrency gain."""
    import ctypes as C
    import torch
    from paper_2112_07115_gb300 import dcem, scenes
    K = args.batched_frames
    nf = warmup + K + 1
    scs = scenes.scene_batch(seed=0, n_frames=2 * nf + 1)
    objs, res, keep = [], [], []
    for sc in scs:
        s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
        s.set_ray_sets([scenes.fibonacci_sphere(n) for n in sc.meta["budgets"]])
        objs.append(s)
        nl = len(sc.meta["budgets"]) * sc.nrx
        mp = max(1024, 8 * nl)
        bufs = (torch.empty((nl, 2), dtype=torch.float64, device=dev), torch.empty(nl, dtype=torch.float64, device=dev),
                torch.empty(nl, dtype=torch.float64, device=dev),
                torch.empty(mp * C.sizeof(dcem.Path), dtype=torch.uint8, device=dev))
        keep.append(bufs)
        r = dcem.Result()
        r.ptr_kind = dcem.PTR_DEVICE
        r.max_paths = mp
        r.field, r.p_coh_dbm, r.p_inc_dbm, r.paths = [x.data_ptr() for x in bufs]
        res.append(r)
    xf_d = [torch.from_numpy(sc.xf).to(dev) if sc.nobj else None for sc in scs]
    rx_d = [torch.from_numpy(sc.rx).to(dev) for sc in scs]
    txs = [sc.meta["tx"] for sc in scs]
    prm = dcem.default_params(max_refl=4, freq_hz=28e9, mode=dcem.MODE_FULL)
    b = dcem.Batch(objs, stream=stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, st = [], []
    for i in range(warmup + K):
        f = i + 1
        flush.zero_()
        e0.record(stream)
        b.update_transforms([x[f] if x is not None else None for x in xf_d])
        rc, failed = b.trace_raw(txs, [x[f] for x in rx_d], prm, res)
        e1.record(stream)
        e1.synchronize()
        if rc != dcem.OK:
            raise dcem.DcemError(rc, f"multi-scene frame {f} (scene {failed})")
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
            st.append([dcem.stats_dict(r.stats) for r in res])
    b.close()
    # the same scenes, one after another
    ms_seq = []
    for i in range(warmup + K):
        f = nf + i + 1
        flush.zero_()
        e0.record(stream)
        for k, s in enumerate(objs):
            if xf_d[k] is not None:
                dcem.dcem_scene_update_transforms(s.h, xf_d[k][f])
            rc = dcem.dcem_trace_links(s.h, txs[k], rx_d[k][f], prm, res[k])
            if rc != dcem.OK:
                raise dcem.DcemError(rc, f"multi-scene sequential frame {f} (scene {k})")
        e1.record(stream)
        e1.synchronize()
        if i >= warmup:
            ms_seq.append(e0.elapsed_time(e1))
    for s in objs:
        s.close()
    t = max_over_ranks([sum(ms) / 1e3], dev)[0]
    t_seq = max_over_ranks([sum(ms_seq) / 1e3], dev)[0]
    rays = sum(sum(sc.meta["budgets"]) for sc in scs)
    links = sum(len(sc.meta["budgets"]) * sc.nrx for sc in scs)
    segs = float(np.mean([sum(x["segments_traced"] for x in fr) for fr in st]))
    return {"workload": "%d independent urban grids: %d-%d triangles (%d in all), %d-%d vehicles (%d), %d "
                        "transmitters with %d-%d rays (%d rays), %d links, 4 reflections, 28 GHz, full frames"
                        % (len(scs), min(x.ntri for x in scs), max(x.ntri for x in scs), sum(x.ntri for x in scs),
                           min(x.nobj for x in scs), max(x.nobj for x in scs), sum(x.nobj for x in scs),
                           sum(len(x.meta["budgets"]) for x in scs), min(min(x.meta["budgets"]) for x in scs),
                           max(max(x.meta["budgets"]) for x in scs), rays, links),
            "frames_per_s": round(world * K / t, 3), "ms_per_frame": round(1e3 * t / K, 3),
            "rays_per_s": round(world * K * rays / t, 0),
            "ray_segments_traced_per_s": round(world * K * segs / t, 0),
            "paths_per_frame": int(np.mean([sum(x["paths_valid"] for x in fr) for fr in st])),
            "graph_replayed_frac": round(float(np.mean([min(x["graph_replayed"] for x in fr) for fr in st])), 3),
            "one_after_another": {"frames_per_s": round(world * K / t_seq, 3),
                                  "ms_per_frame": round(1e3 * t_seq / K, 3)}}


def _trace_roof(st):
    """Closest-hit roofline of timed frames (stats with timing=2): the
    algorithmic bytes (36 B per ray and per segment, 64 B per node pair,
    48 B per triangle test) over the kernel time, of the measured HBM copy
    bandwidth."""
    peak, _ = measured_peaks()
    b = float(np.mean([(x["n_rays"] + x["child_rays"]) * 36 + x["segments_traced"] * 36 + x["node_visits"] * 64 +
                       x["tri_tests"] * 48 for x in st]))
    ms = float(np.mean([x["ms_stage"]["trace"] for x in st]))
    ach = b / (ms * 1e-3) / 1e9
    return {"bound": "latency", "achieved_algorithmic": round(ach, 1), "unit": "GB/s",
            "algorithmic_over_hbm_peak": round(ach / peak, 4),
            "note": "algorithmic bytes (nodes and triangles from L2 and shared memory); a ratio above 1 is "
                    "not an HBM fraction"}


def run_transmission(args, stream, dev, world, flush, rank, warmup=3):
    """Transmission (Table II penetration losses): the indoor office (12
    rooms, 262 triangles, indoor walls 20 dB, glass 5 dB, 4 moving metal
    carts, 48 receivers), 1M rays, 2 reflections and 2 transmissions per
    path, 30 GHz, 0.5 W; full frames (frames with transmission are always
    traced in full), L2 flushed before each. The last frame's paths are
    re-validated by the FP64 oracle and the per-receiver power compared."""
    import ctypes as C
    import torch
    from oracle import oracle as O
    from paper_2112_07115_gb300 import dcem, scenes
    K = args.batched_frames
    sc = scenes.office(n_frames=warmup + K + 1)
    tdb, T = sc.meta["trans_db"], sc.meta["max_trans"]
    s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(sc.n_rays))
    s.set_transmission(tdb, T)
    prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, tx_power_w=0.5, timing=2)
    xf_d = torch.from_numpy(sc.xf).to(dev)
    rx_d = torch.from_numpy(sc.rx).to(dev)
    nrx, max_paths = sc.nrx, 1 << 16
    pc_d = torch.empty(nrx, dtype=torch.float64, device=dev)
    pi_d = torch.empty(nrx, dtype=torch.float64, device=dev)
    fd = torch.empty((nrx, 2), dtype=torch.float64, device=dev)
    paths_d = torch.empty(max_paths * C.sizeof(dcem.Path), dtype=torch.uint8, device=dev)
    res = dcem.Result()
    res.ptr_kind = dcem.PTR_DEVICE
    res.max_paths = max_paths
    res.field, res.p_coh_dbm, res.p_inc_dbm, res.paths = (fd.data_ptr(), pc_d.data_ptr(), pi_d.data_ptr(),
                                                          paths_d.data_ptr())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, st = [], []
    for i in range(warmup + K):
        f = i + 1
        flush.zero_()
        e0.record(stream)
        dcem.dcem_scene_update_transforms(s.h, xf_d[f])
        rc = dcem.dcem_trace_frame(s.h, sc.tx, rx_d[f], prm, res)
        e1.record(stream)
        e1.synchronize()
        if rc != dcem.OK:
            raise dcem.DcemError(rc, f"transmission frame {f}")
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
            st.append(dcem.stats_dict(res.stats))
    s.close()
    t = max_over_ranks([sum(ms) / 1e3], dev)[0]
    segs = float(np.mean([x["segments_traced"] for x in st]))
    out = {"workload": "indoor office, %d rooms, %d triangles (indoor walls 20 dB, glass 5 dB, Table II), %d "
                       "moving carts, %d Rx, %d rays, %d reflections + %d transmissions per path, 30 GHz, full "
                       "frames" % (12, sc.ntri, sc.nobj, nrx, sc.n_rays, sc.max_refl, T),
           "frames_per_s": round(world * K / t, 2), "ms_per_frame": round(1e3 * t / K, 4),
           "child_rays_per_frame": int(np.mean([x["child_rays"] for x in st])),
           "segments_traced_per_frame": int(segs),
           "ray_segments_traced_per_s": round(world * K * segs / t, 0),
           "closest_hit_ms_all_passes": round(float(np.mean([x["ms_stage"]["trace"] for x in st])), 4),
           "trace_roofline": _trace_roof(st),
           "paths_per_frame": int(np.mean([x["paths_valid"] for x in st]))}
    if rank == 0:
        # the last frame's paths re-validated by the FP64 oracle
        f = warmup + K
        n = min(int(st[-1]["paths_valid"]), max_paths)
        raw = paths_d[: n * dcem.PATH_DTYPE.itemsize].cpu().numpy().view(dcem.PATH_DTYPE)
        width = sc.max_refl + T
        keys = np.full((n, 2 + width), -1, np.int32)
        keys[:, 0] = raw["rx"]
        keys[:, 1] = raw["depth"]
        keys[:, 2:] = raw["tri"][:, :width]
        order = np.lexsort(keys.T[::-1])
        keys = keys[order]
        oprm = O.OracleParams(freq_hz=sc.freq_hz, tx_power_w=0.5, n_rays=sc.n_rays, max_refl=sc.max_refl,
                              max_trans=T, trans_db=tuple(tdb))
        wt = O.transform(sc.tris, sc.tri_obj, sc.xf[f])
        ref = O.validate(wt, sc.tri_mat, sc.materials, sc.tx, sc.rx[f], keys, oprm)
        _, pc, pi = O.reduce(keys, ref, nrx, 0.5)
        gc, gi = pc_d.cpu().numpy(), pi_d.cpu().numpy()
        fin = np.isfinite(pc) & np.isfinite(gc)
        out["rx_power_err_db"] = {"paths": int(n), "transmission_paths": int(np.sum(np.any(
            (keys[:, 2:] >= 0) & ((keys[:, 2:] & O.TRANS) != 0), axis=1))),
            "oracle_invalid": int((ref["valid"] == 0).sum()),
            "max_abs_p_coh": float(np.max(np.abs(pc[fin] - gc[fin]))) if fin.any() else 0.0,
            "max_abs_p_inc": float(np.max(np.abs(pi[fin] - gi[fin]))) if fin.any() else 0.0}
    return out


def run_diffraction(args, sc, rays, stream, dev, world, flush, warmup=3):
    """First-order edge diffraction on the headline highway frames (coherent
    mode, every frame adds the diffraction paths of every (receiver, wedge)
    pair): frames/s with and without it, the wedge count and the
    diffraction paths per frame."""
    import ctypes as C
    import torch
    from paper_2112_07115_gb300 import dcem
    K = args.batched_frames * 4
    xf_d = torch.from_numpy(sc.xf).to(dev)
    rx_d = torch.from_numpy(sc.rx).to(dev)
    nrx, max_paths = sc.nrx, 1 << 17
    bufs = [torch.empty((nrx, 2), dtype=torch.float64, device=dev), torch.empty(nrx, dtype=torch.float64, device=dev),
            torch.empty(nrx, dtype=torch.float64, device=dev),
            torch.empty(max_paths * C.sizeof(dcem.Path), dtype=torch.uint8, device=dev)]
    out = {}
    for on in ("refl", True, False):
        s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
        s.set_rays(rays)
        nw = s.set_diffraction(bool(on))
        nrp = s.set_diffraction_reflections(True) if on == "refl" else 0
        prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, mode=dcem.MODE_COHERENT)
        res = dcem.Result()
        res.ptr_kind = dcem.PTR_DEVICE
        res.max_paths = max_paths
        res.field, res.p_coh_dbm, res.p_inc_dbm, res.paths = [x.data_ptr() for x in bufs]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, nd = [], []
        for i in range(warmup + K):
            f = 1 + i % (sc.nframes - 1)  # short runs have fewer frames than this loop
            flush.zero_()
            e0.record(stream)
            dcem.dcem_scene_update_transforms(s.h, xf_d[f])
            rc = dcem.dcem_trace_frame(s.h, sc.tx, rx_d[f], prm, res)
            e1.record(stream)
            e1.synchronize()
            if rc != dcem.OK:
                raise dcem.DcemError(rc, f"diffraction frame {f}")
            if i >= warmup:
                ms.append(e0.elapsed_time(e1))
                if on:
                    n = min(res.n_paths, max_paths)
                    p = bufs[3][: n * C.sizeof(dcem.Path)].cpu().numpy().view(dcem.PATH_DTYPE)
                    first = (p["depth"] == 1) & ((p["tri"][:, 0] & dcem.TRI_DIFFRACT) != 0)
                    comb = (p["depth"] == 2) & ((((p["tri"][:, 0] | p["tri"][:, 1]) & dcem.TRI_DIFFRACT)) != 0)
                    nd.append((int(first.sum()), int(comb.sum())))
        s.close()
        t = max_over_ranks([sum(ms) / 1e3], dev)[0]
        if on == "refl":
            out["with_one_reflection"] = {
                "reflector_planes": nrp, "frames_per_s": round(world * K / t, 2), "ms_per_frame": round(1e3 * t / K, 4),
                "combined_paths_per_frame": round(float(np.mean([x[1] for x in nd])), 1),
                "candidates_per_frame": nw * nrx * nrp * 2,
                "note": "first-order diffraction plus one reflection on a static plane before or after it"}
        elif on:
            out.update({"wedges": nw, "frames_per_s": round(world * K / t, 2), "ms_per_frame": round(1e3 * t / K, 4),
                        "diffraction_paths_per_frame": round(float(np.mean([x[0] for x in nd])), 1),
                        "receiver_wedge_pairs_per_frame": nw * nrx})
        else:
            out["without_diffraction_frames_per_s"] = round(world * K / t, 2)
    out["workload"] = ("highway frames (coherent), first-order UTD diffraction at every wedge (barrier tops and "
                       "vehicle edges) for all 200 receivers")
    return out


def run_diffraction_orders(args, hw, stream, dev, world, flush, warmup=2, K=8):
    """Diffraction of order 1-3 (Sec. III step 5, bound 3): frames/s of the
    city blocks (8 x 8 box buildings, 512 wedges, 64 receivers, 200k rays,
    3 reflections) with diffraction up to order 1, 2 and 3, up to order 2
    with one reflection before or after each chain (the ground and every
    building face as reflector planes), and first order with up to two
    reflections around it; the highway frames with order 2, and with first
    order and up to two reflections around it; both workloads up to order 2
    with every combination of reflections (around a first-order diffraction,
    before or after a chain, between its two wedges); the
    pre-test candidates and wedge pairs/triples per frame, and order 2 on 8
    of the city's receivers against the oracle."""
    import torch
    from oracle import oracle as O
    from paper_2112_07115_gb300 import dcem, scenes
    city = scenes.city_blocks()

    def frames(sc, order, n_rays, max_refl, mode, refl=0):
        s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
        s.set_rays(scenes.fibonacci_sphere(n_rays))
        nw = s.set_diffraction(True)
        nrp = s.set_diffraction_reflections(refl) if refl else 0
        s.set_diffraction_order(order)
        prm = dcem.default_params(max_refl=max_refl, freq_hz=sc.freq_hz, mode=mode)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, fr = [], None
        for i in range(warmup + K):
            f = min(1 + i, sc.nframes - 1)
            flush.zero_()
            e0.record(stream)
            if sc.nobj:
                s.update_transforms(sc.xf[f])
            fr = s.trace(sc.tx, sc.rx[f], prm)
            e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                ms.append(e0.elapsed_time(e1))
        s.close()
        p = fr.paths
        by = [int(((p["depth"] == m) & np.all((p["tri"][:, :m] & dcem.TRI_DIFFRACT) != 0, axis=1)).sum())
              for m in (1, 2, 3)]
        t = max_over_ranks([sum(ms) / 1e3], dev)[0]
        st = fr.stats
        d = np.zeros(len(p), np.int32)
        for i in range(4):
            d += ((p["tri"][:, i] >= 0) & ((p["tri"][:, i] & dcem.TRI_DIFFRACT) != 0)).astype(np.int32)
        with_refl = [int(((p["depth"] == m + 1) & (d == m)).sum()) for m in (1, 2, 3)]
        out = {"frames_per_s": round(world * K / t, 2), "ms_per_frame": round(1e3 * t / K, 3), "wedges": nw,
               "diffraction_paths_by_order": by, "wedge_pairs": st["diff_pairs"],
               "wedge_triples": st["diff_triples"], "fp64_candidates": st["diff_candidates"]}
        if refl:
            out.update({"reflector_planes": nrp, "with_one_reflection_by_order": with_refl})
        if refl >= 2:
            t3 = p["tri"][:, :3]
            nd = ((t3 >= 0) & ((t3 & dcem.TRI_DIFFRACT) != 0)).sum(axis=1)
            sel = (p["depth"] == 3) & (nd == 1)
            at = [int((sel & ((t3[:, i] & dcem.TRI_DIFFRACT) != 0)).sum()) for i in range(3)]
            out["with_two_reflections"] = {"both_before": at[2], "one_each_side": at[1], "both_after": at[0]}
        if refl >= 3:
            t3 = p["tri"][:, :3]
            dd = (t3 >= 0) & ((t3 & dcem.TRI_DIFFRACT) != 0)
            out["with_a_reflection_between_two_wedges"] = int(((p["depth"] == 3) & dd[:, 0] & ~dd[:, 1] &
                                                                dd[:, 2]).sum())
        return out, fr

    out = {"city_workload": "8 x 8 box buildings (642 triangles, 512 wedges), 1 Tx at 10 m, 64 Rx at 1.5 m, "
                            "200000 rays, 3 reflections, 28 GHz, full frames (static scene)"}
    last = None
    for order in (1, 2, 3):
        r, fr = frames(city, order, 200_000, 3, dcem.MODE_FULL)
        out[f"city_order_{order}"] = r
        if order == 2:
            last = fr
    r, _ = frames(city, 2, 200_000, 3, dcem.MODE_FULL, refl=1)
    out["city_order_2_with_reflections"] = r
    r, _ = frames(city, 1, 200_000, 3, dcem.MODE_FULL, refl=2)
    out["city_order_1_with_two_reflections"] = r
    r, _ = frames(city, 2, 200_000, 3, dcem.MODE_FULL, refl=3)
    out["city_order_2_with_reflections_around_and_between"] = r
    r, _ = frames(hw, 2, hw.n_rays, hw.max_refl, dcem.MODE_COHERENT)
    out["highway_order_2"] = r
    r, _ = frames(hw, 1, hw.n_rays, hw.max_refl, dcem.MODE_COHERENT, refl=2)
    out["highway_order_1_with_two_reflections"] = r
    r, _ = frames(hw, 2, hw.n_rays, hw.max_refl, dcem.MODE_COHERENT, refl=3)
    out["highway_order_2_with_reflections_around_and_between"] = r
    # order 2 against the oracle on 8 receivers of the city (the oracle is brute force)
    sub = city.rx[0][:8]
    prm = O.OracleParams(freq_hz=city.freq_hz, max_refl=3)
    ck, cp = O.diffract_multi(city.tris.reshape(-1, 9), city.tri_mat, city.tri_obj, city.materials, city.tx, sub,
                              prm, 2)
    g = last.paths[(last.paths["depth"] == 2) & np.all((last.paths["tri"][:, :2] & dcem.TRI_DIFFRACT) != 0, axis=1)
                   & (last.paths["rx"] < 8)]
    gk = {(int(x["rx"]), int(x["tri"][0]), int(x["tri"][1])): x for x in g}
    ok = {(int(k[0]), int(k[2]), int(k[3])): p for k, p in zip(ck, cp)}
    common = set(gk) & set(ok)
    err = [abs(complex(gk[k]["amp_re"], gk[k]["amp_im"]) - complex(ok[k]["amp_re"], ok[k]["amp_im"])) /
           abs(complex(ok[k]["amp_re"], ok[k]["amp_im"])) for k in common]
    out["oracle_check_order_2"] = {"receivers": 8, "gpu_paths": len(gk), "oracle_paths": len(ok),
                                   "set_differences": len(set(gk) ^ set(ok)),
                                   "max_rel_amp_err": float(max(err)) if err else None}
    return out


def grad_timing(s, sc, rx_f, paths_d, n_paths, stream, dev, reps=20):
    """dcem_path_gradients on one frame's device paths: d E / d theta and
    d P_coh / d theta for every material's (eps_r, sigma) and every vehicle's
    (x, y), timed with CUDA events over `reps` calls after 3 warm-up calls."""
    import torch
    from paper_2112_07115_gb300 import dcem
    nrx = sc.nrx
    npar = dcem.dcem_scene_gradient_size(s.h)
    prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz)
    fd = torch.empty((nrx, 2), dtype=torch.float64, device=dev)
    dfd = torch.empty((nrx, npar, 2), dtype=torch.float64, device=dev)
    dpd = torch.empty((nrx, npar), dtype=torch.float64, device=dev)

    def call():
        return dcem.dcem_path_gradients(s.h, sc.tx, rx_f, paths_d.data_ptr(), prm, dcem.PTR_DEVICE,
                                         fd.data_ptr(), dfd.data_ptr(), dpd.data_ptr(), n_paths=n_paths)
    for _ in range(3):
        if call() != dcem.OK:
            return {"error": "dcem_path_gradients failed"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        call()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nz = int(torch.count_nonzero(dfd).item()) // 2
    return {"ms_per_call": round(ms, 4), "paths": n_paths, "receivers": nrx, "params": npar,
            "nonzero_derivatives": nz,
            "note": "forward-mode FP64 derivatives of the received field over the frame's path topology "
                    "(materials eps_r, sigma; vehicle x, y); parity vs FP64 central differences in tests"}


def power_error_vs_oracle(sc, s, f, max_paths, paths_d, pc_d, pi_d, res_n):
    """Validate the GPU's distinct path keys with the FP64 oracle and compare
    the per-receiver power (same path set, FP64 vs the GPU)."""
    from oracle import oracle as O
    from paper_2112_07115_gb300 import dcem
    n = min(int(res_n["paths_valid"]), max_paths)
    raw = paths_d[: n * dcem.PATH_DTYPE.itemsize].cpu().numpy().view(dcem.PATH_DTYPE)
    N = sc.max_refl
    keys = np.full((n, 2 + N), -1, np.int32)
    keys[:, 0] = raw["rx"]
    keys[:, 1] = raw["depth"]
    keys[:, 2:] = raw["tri"][:, :N]
    order = np.lexsort(keys.T[::-1])
    keys = keys[order]
    wt = O.transform(sc.tris, sc.tri_obj, sc.xf[f])
    prm = O.OracleParams(freq_hz=sc.freq_hz, n_rays=sc.n_rays, max_refl=N)
    ref = O.validate(wt, sc.tri_mat, sc.materials, sc.tx, sc.rx[f], keys, prm)
    _, pc, pi = O.reduce(keys, ref, sc.nrx, prm.tx_power_w)
    gc, gi = pc_d.cpu().numpy(), pi_d.cpu().numpy()
    fin = np.isfinite(pc) & np.isfinite(gc)
    return {"frame": int(f), "paths": int(n), "oracle_invalid": int((ref["valid"] == 0).sum()),
            "max_abs_p_coh": float(np.max(np.abs(pc[fin] - gc[fin]))) if fin.any() else 0.0,
            "max_abs_p_inc": float(np.max(np.abs(pi[fin] - gi[fin]))) if fin.any() else 0.0,
            "max_len_err_m": float(np.max(np.abs(ref["len_m"][ref["valid"] == 1] -
                                                 raw["len_m"][order][ref["valid"] == 1]))) if n else 0.0,
            "against": "FP64 oracle validation of the same path keys"}


def run_e2e(args, sc, rays, stream, W, K, world, dev, flush):
    """Same frames through the C ABI with host buffers: per step the
    transforms and receivers are copied host->device and the per-receiver
    results and paths device->host inside the timed region. The L2 is
    flushed before every step, outside the timed region, as for `value`."""
    import torch
    from paper_2112_07115_gb300 import dcem
    s = dcem.Scene.from_scene(sc, stream=stream.cuda_stream)
    s.set_rays(rays)
    prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, mode=dcem.MODE_COHERENT)
    xf_h = torch.from_numpy(sc.xf).pin_memory()
    rx_h = torch.from_numpy(sc.rx).pin_memory()
    nrx = sc.nrx
    max_paths = 1 << 17
    field = torch.empty((nrx, 2), dtype=torch.float64).pin_memory()
    pc = torch.empty(nrx, dtype=torch.float64).pin_memory()
    pi = torch.empty(nrx, dtype=torch.float64).pin_memory()
    paths = torch.empty(max_paths * dcem.PATH_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    res = dcem.Result()
    res.ptr_kind = dcem.PTR_HOST
    res.max_paths = max_paths
    res.field, res.p_coh_dbm, res.p_inc_dbm, res.paths = (field.data_ptr(), pc.data_ptr(), pi.data_ptr(),
                                                          paths.data_ptr())
    h2d = d2h = 0
    t = 0.0
    for i, f in enumerate(range(1, W + K + 1)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dcem.dcem_scene_update_transforms(s.h, xf_h[f])
        rc = dcem.dcem_trace_frame(s.h, sc.tx, rx_h[f], prm, res)
        t1 = time.perf_counter()
        if rc != dcem.OK:
            raise dcem.DcemError(rc, "e2e")
        if i >= W:
            t += t1 - t0
            h2d += sc.nobj * 48 + nrx * 12
            d2h += nrx * 32 + res.n_paths * dcem.PATH_DTYPE.itemsize + 2 * 96
    s.close()
    t = max_over_ranks([t], dev)[0]
    return {"value": round(world * K / t, 2), "unit": "frames/s", "h2d_bytes_per_step": int(h2d / K),
            "d2h_bytes_per_step": int(d2h / K),
            "l2": "flushed before every step (outside the timed region)",
            "note": "C-ABI calls with pinned host transforms/receivers and host outputs; wall clock"}


def cpu_baseline(sc, rays, f, nframes=2):
    """The FP64 oracle on the host cores, on a bounded sample of the workload:
    `nframes` whole highway frames (every ray traced, its distinct keys
    validated), about 10 s on 16 Arm cores."""
    from oracle import oracle as O
    prm = O.OracleParams(freq_hz=sc.freq_hz, n_rays=sc.n_rays, max_refl=sc.max_refl)
    t0 = time.perf_counter()
    segs = 0
    for g in range(f, f + nframes):
        wt = O.transform(sc.tris, sc.tri_obj, sc.xf[g])
        tr = O.trace(wt, sc.tri_mat, sc.materials, sc.tx, rays, sc.rx[g], prm)
        keys = O.unique_keys(O.candidate_keys(tr["cands"], tr["hit_id"], prm.max_refl))
        O.validate(wt, sc.tri_mat, sc.materials, sc.tx, sc.rx[g], keys, prm)
        segs += int(tr["nseg"].sum())
    dt = time.perf_counter() - t0
    return {"value": round(nframes / dt, 5), "unit": "frames/s", "cores": os.cpu_count(),
            "cpu_model": cpu_model(), "kind": "oracle", "ray_segments_per_s": round(segs / dt, 0),
            "sample": f"highway frames {f}-{f + nframes - 1}, all {len(rays)} rays traced and their keys "
                      f"validated, {dt:.1f} s"}


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    K, W = args.steps, args.warmup
    sc, rays = workload(args, n_frames=W + K + 2)
    frac = 32
    prm = O.OracleParams(freq_hz=sc.freq_hz, n_rays=sc.n_rays, max_refl=sc.max_refl)
    times, segs = [], []
    for i, f in enumerate(range(1, W + K + 1)):
        sub = rays[(f % frac)::frac]
        t0 = time.perf_counter()
        wt = O.transform(sc.tris, sc.tri_obj, sc.xf[f])
        tr = O.trace(wt, sc.tri_mat, sc.materials, sc.tx, sub, sc.rx[f], prm)
        keys = O.unique_keys(O.candidate_keys(tr["cands"], tr["hit_id"], prm.max_refl))
        O.validate(wt, sc.tri_mat, sc.materials, sc.tx, sc.rx[f], keys, prm)
        dt = time.perf_counter() - t0
        if i >= W:
            times.append(dt)
            segs.append(int(tr["nseg"].sum()))
    # each step processes 1/frac of a frame: the rate is frames (fractions
    # included) per second of measured time, nothing extrapolated
    t = sum(times)
    v = (K / frac) / t
    line = {"metric": METRIC, "value": round(v, 6), "unit": "frames/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": round(1e3 * t / K, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "impl": "reference",
            "data": "synthetic (seeded highway generator)", "config": config(args, sc, {"mode": "full retrace"}),
            "step": f"1/{frac} of one frame's rays (every {frac}th ray from an offset that changes per frame), "
                    f"traced and their distinct keys validated",
            "ray_segments_per_s": round(sum(segs) / t, 0),
            "cpu_baseline": {"value": round(v, 6), "unit": "frames/s", "cores": os.cpu_count(),
                             "cpu_model": cpu_model(), "kind": "oracle",
                             "sample": f"{K} steps of 1/{frac} of a frame each, {t:.1f} s measured"},
            "e2e": {"value": round(v, 6), "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
