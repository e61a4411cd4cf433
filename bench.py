#!/usr/bin/env python3
"""Benchmark of the visibility color map (VCM) path on GB300.

Workload (one step = one whole VCM: grid-index cull, slab tests, visible
measure, quantisation): the 3D plain VCM - 512 x 512 viewpoints at 1.7 m
plus 4 layers spaced 10 m, 5,000 boxes (footprints 10-60 m, lognormal
heights, median 20 m, sigma 0.6, centres from a 16-component Gaussian
mixture over 2 km x 2 km), a 20 m x 10 m target at 30 m split into 32 x 16
patches, 16 color levels.  Seeded synthetic inputs stand in for the paper's
city datasets.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
Under torchrun each rank runs its own full copy of the workload (weak
scaling, no data-path collective) and the slowest rank's time is reported.
"""

import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "viewpoint-patch occlusion tests/sec and VCM cells/sec at ≤1e-5 rel err; p50/p99 latency"
UNIT = "segments/s"
WORKLOAD = "3D plain VCM: 512x512 viewpoints x 5 layers, 5,000 mixture boxes over 2 km, 20x10 m target, 32x16 patches"
# Algorithmic work of one segment/box slab test: per axis the entry and exit
# parameters (a multiply each; the differences to the box faces are shared
# per viewpoint and box), their min/max, and the running max of entries and
# min of exits, then one compare: 6 FMUL + 12 FMNMX + 1 compare = 19 FP32
# operations in 3D, 13 in 2D.  Every test the tile kernel counts (row tests
# of the sweep, corner tests of the one-box checks) decides one
# segment/box pair.  The separable sweep itself issues only ~7 lane
# operations per row test, sharing the u and n parts across a column's rows;
# those are reported beside the fraction.
OPS_PER_SLAB_TEST = {3: 19, 2: 13}
ISSUED_OPS_PER_ROW_TEST = 7
ISSUED_OPS_PER_CORNER_TEST = 15
L2_FLUSH_BYTES = 512 << 20
# kernels of ours that one step launches: k_prologue, k_tiles (two passes:
# the tiles, then the open viewpoints they published), k_quantise
LAUNCHES_PER_STEP = 4


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return {}


def hbm_peak():
    """Copy bandwidth measured on the GB300s, else the recipe's
    fallback figure."""
    v = peaks().get("hbm_gbs")
    if v:
        return {"value": float(v), "basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    return {"value": 6800.0, "basis": "fallback 6.8 TB/s (no measured peak file)"}


PROFILE = os.path.join(ROOT, "profiles", "k_tiles_3d_512x512x5_5000boxes.md")
KERNEL_SRC = os.path.join(ROOT, "paper_1310_7297_gb300", "csrc", "vcm_kernels.cu")


def profiled_traffic():
    """DRAM bytes per k_tiles launch from the committed ncu summary, or None
    if the kernel source has changed since that capture."""
    import hashlib

    try:
        text = open(PROFILE).read()
        digest = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        line = line.strip().lstrip("-* ")
        if ":" in line and line.startswith(("kernel_source_sha256", "dram_bytes_per_launch")):
            k, v = line.split(":", 1)
            vals[k.strip().strip("`* ")] = v.strip().strip("`* ")
    if vals.get("kernel_source_sha256") != digest:
        return None
    try:
        return int(float(vals["dram_bytes_per_launch"]))
    except (KeyError, ValueError):
        return None


def alu_peak_ops(sm_count, mhz):
    """Issue-limited lane-operation rate: 4 schedulers x 32 lanes per SM per clock."""
    return sm_count * 4 * 32 * mhz * 1e6


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self, t_from=None, t_to=None):
        """Summary of the samples taken between t_from and t_to
        (time.monotonic()); all samples when not given."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        rows = []
        for ts, l in self.lines:
            if (t_from is not None and ts < t_from) or (t_to is not None and ts > t_to):
                continue
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0]:
                continue
            rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def reduce_max(x, pg, device=None):
    """Largest value of x over all ranks (identity without a process group)."""
    if pg is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_rate(scene, req, seconds, seed=0):
    """Segments/s of the CPU oracle on seeded random viewpoint samples that
    add up to about `seconds` of wall time, on all host cores.  A probe sets
    the first sample's size; further samples (at most four in all) top the
    time up, each sized from the rate measured so far."""
    from oracle import oracle as O

    O.build()
    n = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    P = req["patches_u"] * req["patches_w"]
    rng = np.random.default_rng(seed)
    probe = np.sort(rng.choice(n, 64, replace=False))
    t0 = time.perf_counter()
    O.run(scene, req, indices=probe)
    rate = 64 / max(time.perf_counter() - t0, 1e-6)
    m_all, t_all = 0, 0.0
    for _ in range(4):
        if t_all >= 0.9 * seconds:
            break
        m = int(min(n, max(64, rate * (seconds - t_all))))
        idx = np.sort(rng.choice(n, m, replace=False))
        t0 = time.perf_counter()
        O.run(scene, req, indices=idx)
        t_all += time.perf_counter() - t0
        m_all += m
        rate = m_all / t_all
    return {"value": m_all * P / t_all, "cells_per_s": m_all / t_all, "seconds": t_all, "viewpoints": m_all,
            "cores": O.default_threads()}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import synth

    scene, req = synth.workload_3d()
    per_step = max(2.0, 120.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup):
        oracle_rate(scene, req, per_step / 4, seed=100 + i)
    rates, secs, vps, cores = [], [], 0, 1
    for i in range(args.steps):
        r = oracle_rate(scene, req, per_step, seed=i)
        rates.append(r["value"])
        secs.append(r["seconds"])
        vps += r["viewpoints"]
        cores = r["cores"]
    value = float(np.mean(rates))
    P = req["patches_u"] * req["patches_w"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(scene, req),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d random viewpoints of the workload over %d steps (%d patches each)"
                                   % (vps, args.steps, P)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(scene, req):
    n_vp = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    return {"workload": WORKLOAD, "viewpoints": n_vp, "grid": [req["grid_nx"], req["grid_ny"]],
            "layers_m": [z / 1024 for z in req["layer_z"]], "patches": [req["patches_u"], req["patches_w"]],
            "boxes": scene.n, "scene_digest": scene.digest(), "color_levels": req["color_levels"],
            "segments_per_step": n_vp * req["patches_u"] * req["patches_w"],
            "l2": "512 MB buffer written between timed steps", "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch

    import synth
    from paper_1310_7297_gb300 import Context, stats_from_tensor
    from paper_1310_7297_gb300 import build as B
    from paper_1310_7297_gb300.vcm import STATS_BYTES

    world, rank, local = dist_setup()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    scene, req = synth.workload_3d()
    n_vp = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    P = req["patches_u"] * req["patches_w"]
    seg = n_vp * P
    ctx = Context(local)
    ctx.load_scene(scene)
    ctx.vcm_build(0.0)
    stream = torch.cuda.current_stream(dev)
    v = torch.empty(n_vp, dtype=torch.float32, device=dev)
    col = torch.empty(n_vp, dtype=torch.uint8, device=dev)
    st = torch.empty(STATS_BYTES, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        ctx.vcm_compute(req, v.data_ptr(), col.data_ptr(), None, st.data_ptr(), stream.cuda_stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    uuid = None
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = u[4:] if u.startswith("GPU-") else u
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    # The timed region of a few ms is shorter than the 200 ms sampling
    # period, so the same step also runs untimed for about half a second
    # right before it; the clock summary covers that load and the timed
    # region.
    t_load = time.monotonic()
    while time.monotonic() - t_load < 0.6:
        for _ in range(20):
            flush.zero_()
            step()
        torch.cuda.synchronize()
    K = args.steps
    s_ev = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    e_ev = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    kb = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ka = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for e in kb + ka:
        e.record(stream)   # torch creates the CUDA event on first record; the library re-records it
    torch.cuda.synchronize()
    for i in range(K):
        flush.zero_()
        ctx.vcm_set_timing_events(kb[i], ka[i])
        s_ev[i].record(stream)
        step()
        e_ev[i].record(stream)
    torch.cuda.synchronize()
    t_end = time.monotonic()
    ctx.vcm_set_timing_events(None, None)
    clocks = sampler.stop(t_load, t_end)
    if clocks is not None:
        clocks["window"] = "%.2f s: the same step untimed, then the timed region" % (t_end - t_load)
    step_ms = [s.elapsed_time(e) for s, e in zip(s_ev, e_ev)]
    kern_ms = [b.elapsed_time(a) for b, a in zip(kb, ka)]
    total_ms = reduce_max(float(sum(step_ms)), pg, dev)
    if pg:
        pg.barrier()
    stats = stats_from_tensor(st)

    # End to end through the public API with host buffers.  Headline: the
    # scene is a resident database (uploaded and indexed once, as the
    # paper's obstacle set is), and each step submits the request, waits for
    # it and reads its values and colours back into host memory.  Also
    # reported: the same with the scene uploaded and re-indexed every step.
    lo = torch.from_numpy(scene.lo_f32()[:, :3].copy()).pin_memory().numpy()
    hi = torch.from_numpy(scene.hi_f32()[:, :3].copy()).pin_memory().numpy()

    def e2e_loop(with_scene):
        ms, chk = [], 0.0
        for i in range(args.warmup + K):
            t0 = time.perf_counter()
            if with_scene:
                ctx.vcm_scene_load_mem(lo, hi, 3)
                ctx.vcm_build(0.0)
            t = ctx.vcm_submit(req)
            ctx.vcm_poll(t, -1)
            hv, hc, _, _ = ctx.vcm_result_get(t, copy=False)
            chk += float(hv[-1]) + int(hc[-1])
            ctx.vcm_result_release(t)
            if i >= args.warmup:
                ms.append(1e3 * (time.perf_counter() - t0))
        return ms

    e2e_scene_ms = e2e_loop(True)
    e2e_ms = e2e_loop(False)
    e2e_scene_total = reduce_max(float(sum(e2e_scene_ms)), pg, dev)
    e2e_total = reduce_max(float(sum(e2e_ms)), pg, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_rate(scene, req, args.cpu_seconds)
        cpu = {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
               "sample": "%d random viewpoints of the workload (%d patches each), %.1f s of CPU work"
                         % (r["viewpoints"], P, r["seconds"])}

    # the request as uploaded: its descriptor and the coordinates the library
    # derives from it (patch centres, viewpoint x, y, layer heights)
    from paper_1310_7297_gb300.vcm import vcm_request
    req_bytes = int(ctypes.sizeof(vcm_request) + 4 * (req["patches_u"] + req["patches_w"] + req["grid_nx"] +
                                                       req["grid_ny"] + len(req["layer_z"])))
    if rank == 0:
        pk = peaks()
        props = torch.cuda.get_device_properties(dev)
        sm_count = props.multi_processor_count
        max_mhz = float(pk.get("sm_max_mhz", 2070.0))
        peak = alu_peak_ops(sm_count, max_mhz)
        kern_avg_s = float(np.mean(kern_ms)) / 1e3
        units = stats["slab_tests"] + stats["corner_tests"]
        achieved = units * OPS_PER_SLAB_TEST[req["dims"]] / kern_avg_s
        issued = (stats["slab_tests"] * ISSUED_OPS_PER_ROW_TEST +
                  stats["corner_tests"] * ISSUED_OPS_PER_CORNER_TEST) / kern_avg_s
        value = world * seg * K / (total_ms / 1e3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": config_dict(scene, req),
            "cells_per_s": world * n_vp * K / (total_ms / 1e3),
            "kernel_ms": float(np.mean(kern_ms)),
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": profiled_traffic(),
                         "kernel": "k_tiles", "work_unit": "segment/box slab test",
                         "ops_per_unit": OPS_PER_SLAB_TEST[req["dims"]],
                         "issued_slab_ops": {"value": issued / 1e12, "frac": issued / peak,
                                             "ops_per_row_test": ISSUED_OPS_PER_ROW_TEST,
                                             "ops_per_corner_test": ISSUED_OPS_PER_CORNER_TEST},
                         "units_per_launch": units,
                         "peak_basis": "%d SMs x 128 lane-instr/clk x %.0f MHz (issue limit)" % (sm_count, max_mhz)},
            "stats": {"slab_tests": stats["slab_tests"], "corner_tests": stats["corner_tests"],
                      "shortcut_viewpoints": stats["shortcut_viewpoints"], "rechecked": stats["rechecked"],
                      "shared_viewpoints": stats["shared_viewpoints"],
                      "boxes_listed": stats["boxes_listed"], "edge_cells": stats["edge_cells"],
                      "v_ref": stats["v_ref"], "nonzero_cells": int((v > 0).sum().item())},
            "cpu_baseline": cpu,
            "e2e": {"value": world * seg * K / (e2e_total / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": req_bytes, "d2h_bytes_per_step": int(n_vp * 5 + STATS_BYTES),
                    "ms_per_step": e2e_total / K,
                    "path": "vcm_submit, vcm_poll, vcm_result_get (values and colours into pinned host memory); "
                            "scene resident, uploaded and indexed once"},
            "e2e_scene_per_step": {"value": world * seg * K / (e2e_scene_total / 1e3), "unit": UNIT,
                                   "h2d_bytes_per_step": int(lo.nbytes + hi.nbytes) + req_bytes,
                                   "d2h_bytes_per_step": int(n_vp * 5 + STATS_BYTES),
                                   "ms_per_step": e2e_scene_total / K,
                                   "path": "vcm_scene_load_mem and vcm_build every step, then as e2e"},
            "gpu_launches": LAUNCHES_PER_STEP * K,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()


# ---------------------------------------------------------------------------
# batched uneven requests (one persistent launch) and serving
# ---------------------------------------------------------------------------

def _alloc_outputs(torch, dev, reqs):
    from paper_1310_7297_gb300 import n_viewpoints
    from paper_1310_7297_gb300.vcm import STATS_BYTES

    vs = [torch.empty(n_viewpoints(r), dtype=torch.float32, device=dev) for r in reqs]
    cs = [torch.empty(n_viewpoints(r), dtype=torch.uint8, device=dev) for r in reqs]
    st = torch.empty(STATS_BYTES * len(reqs), dtype=torch.uint8, device=dev)
    return vs, cs, st


def run_batched(args):
    """256 uneven requests over a shared 50,000-box scene: one persistent
    launch (default shapes, then autotuned shapes) against one launch per
    request (autotuned shapes)."""
    import torch

    import synth
    from paper_1310_7297_gb300 import Context, n_viewpoints
    from paper_1310_7297_gb300 import build as B
    from paper_1310_7297_gb300.vcm import STATS_BYTES

    B.build()
    dev = torch.device("cuda", 0)
    scene, reqs = synth.workload_batched(n_requests=args.batch_requests)
    seg = sum(n_viewpoints(r) * r["patches_u"] * r["patches_w"] for r in reqs)
    ctx = Context(0)
    ctx.load_scene(scene)
    ctx.vcm_build(50.0)
    vs, cs, st = _alloc_outputs(torch, dev, reqs)
    stream = torch.cuda.current_stream(dev)

    def batch():
        ctx.vcm_compute_batch(reqs, [t.data_ptr() for t in vs], [t.data_ptr() for t in cs], [None] * len(reqs),
                              st.data_ptr(), stream.cuda_stream)

    def singles():
        for i, r in enumerate(reqs):
            ctx.vcm_compute(r, vs[i].data_ptr(), cs[i].data_ptr(), None, st.data_ptr() + STATS_BYTES * i, stream.cuda_stream)

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return {"ms": float(np.median(ms)), "segments_per_s": seg / (float(np.median(ms)) / 1e3)}

    res = {"persistent_batch_default_shapes": timed(batch)}
    t0 = time.perf_counter()
    # 16 requests of the mix (a seeded sample) stand for it
    pick = np.random.default_rng(7).choice(len(reqs), size=min(16, len(reqs)), replace=False)
    samples = [reqs[i] for i in sorted(pick)]
    tuned = ctx.vcm_autotune(samples)
    tune_s = time.perf_counter() - t0
    res["persistent_batch"] = timed(batch)
    # roofline of the batched launch: slab-test operations counted on the
    # device over the batch's time (which also holds the small prologue and
    # colour kernels, so the fraction is a lower bound)
    from paper_1310_7297_gb300 import stats_from_tensor
    batch()
    torch.cuda.synchronize()
    per = [stats_from_tensor(st[i * STATS_BYTES:(i + 1) * STATS_BYTES]) for i in range(len(reqs))]
    ops = sum((p["slab_tests"] + p["corner_tests"]) * OPS_PER_SLAB_TEST[r["dims"]] for p, r in zip(per, reqs))
    props = torch.cuda.get_device_properties(dev)
    peak = alu_peak_ops(props.multi_processor_count, float(peaks().get("sm_max_mhz", 2070.0)))
    achieved = ops / (res["persistent_batch"]["ms"] / 1e3)
    res["persistent_batch"]["roofline"] = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                                           "unit": "Tops/s", "frac": achieved / peak}
    res["one_per_launch"] = timed(singles)
    print(json.dumps({"mode": "batched", "metric": METRIC, "unit": UNIT, "requests": len(reqs), "boxes": scene.n,
                      "segments": seg, "autotune_s": tune_s, "tuned_shapes": sorted(set(map(tuple, tuned))),
                      **res, "speedup": res["one_per_launch"]["ms"] / res["persistent_batch"]["ms"]}), flush=True)
    ctx.close()


def run_serve(args):
    """Poisson arrivals of requests from the batched mix against a resident
    100,000-box scene.  Continuous batching (vcm_submit / vcm_poll: queued
    requests are admitted into slots as memory and slots free up, and run as
    batched persistent launches that overlap on the device) against a FIFO
    server that runs one request per launch: a worker thread takes requests
    in arrival order, runs vcm_compute on one stream and copies v and colors
    back to pinned host memory.  Latency = completion minus arrival."""
    import queue as _queue

    import torch

    import synth
    from paper_1310_7297_gb300 import Context, n_viewpoints
    from paper_1310_7297_gb300 import build as B
    from paper_1310_7297_gb300.vcm import STATS_BYTES

    B.build()
    dev = torch.device("cuda", 0)
    scene, _ = synth.workload_3d_large(grid=64, layers=1)
    ctx = Context(0, 64 << 30)
    ctx.load_scene(scene)
    ctx.vcm_build(50.0)
    ctx.vcm_set_slots(args.slots, args.max_batch)
    pool = synth.serving_requests(scene, count=args.serve_pool)
    seg_of = [n_viewpoints(r) * r["patches_u"] * r["patches_w"] for r in pool]
    nmax = max(n_viewpoints(r) for r in pool)
    stream = torch.cuda.Stream(dev)
    d_v = torch.empty(nmax, dtype=torch.float32, device=dev)
    d_c = torch.empty(nmax, dtype=torch.uint8, device=dev)
    d_s = torch.empty(STATS_BYTES, dtype=torch.uint8, device=dev)
    h_v = torch.empty(nmax, dtype=torch.float32).pin_memory()
    h_c = torch.empty(nmax, dtype=torch.uint8).pin_memory()

    def fifo_one(r):
        n = n_viewpoints(r)
        with torch.cuda.stream(stream):
            ctx.vcm_compute(r, d_v.data_ptr(), d_c.data_ptr(), None, d_s.data_ptr(), stream.cuda_stream)
            h_v[:n].copy_(d_v[:n], non_blocking=True)
            h_c[:n].copy_(d_c[:n], non_blocking=True)
        stream.synchronize()

    for r in pool[:8]:
        fifo_one(r)
    # warm the scheduler path too
    for t in [ctx.vcm_submit(r) for r in pool[:8]]:
        ctx.vcm_poll(t, -1)
        ctx.vcm_result_release(t)
    out = []
    for rate in args.rates:
        n = int(min(args.serve_count, max(40, rate * args.serve_seconds)))
        arr = synth.poisson_arrivals(int(rate), float(rate), n)
        picks = [pool[i % len(pool)] for i in range(n)]
        seg = sum(seg_of[i % len(pool)] for i in range(n))

        # FIFO server, one request per launch
        q = _queue.Queue()
        done = [0.0] * n

        def worker():
            for _ in range(n):
                i, t0 = q.get()
                fifo_one(picks[i])
                done[i] = time.perf_counter() - t0

        th = threading.Thread(target=worker)
        th.start()
        t0 = time.perf_counter()
        for i in range(n):
            now = time.perf_counter() - t0
            if arr[i] > now:
                time.sleep(arr[i] - now)
            q.put((i, t0))
        th.join()
        lat = [1e3 * (done[i] - arr[i]) for i in range(n)]
        fifo = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "segments_per_s": seg / max(done)}

        # continuous batching through the scheduler
        tickets = [None] * n
        t0 = time.perf_counter()
        for i in range(n):
            now = time.perf_counter() - t0
            if arr[i] > now:
                time.sleep(arr[i] - now)
            ts = time.perf_counter() - t0   # the library times from here to completion
            tickets[i] = (ctx.vcm_submit(picks[i]), ts)
        lat2, last = [], 0.0
        for i, (t, ts) in enumerate(tickets):
            ctx.vcm_poll(t, -1)
            _, hc, _, stt = ctx.vcm_result_get(t, copy=False)
            lat2.append((ts - arr[i]) * 1e3 + stt["latency_ms"])
            last = max(last, arr[i] + lat2[-1] / 1e3)
            ctx.vcm_result_release(t)
        cont = {"p50_ms": float(np.percentile(lat2, 50)), "p99_ms": float(np.percentile(lat2, 99)),
                "segments_per_s": seg / last}
        out.append({"rate_per_s": rate, "requests": n, "continuous": cont, "one_per_launch_fifo": fifo})
    print(json.dumps({"mode": "serve", "metric": METRIC, "unit": UNIT, "boxes": scene.n, "budget_gb": 64,
                      "slots": args.slots, "max_batch": args.max_batch, "rates": out}), flush=True)
    ctx.close()


def run_large(args):
    """The large scene at full size: 100,000 boxes over 10 km x 10 km, one
    40 m x 20 m target split 64 x 32, 2048 x 2048 x 8 viewpoints, 50 m grid
    index.  Same timing rules as the default step."""
    import torch

    import synth
    from paper_1310_7297_gb300 import Context, stats_from_tensor
    from paper_1310_7297_gb300 import build as B
    from paper_1310_7297_gb300.vcm import STATS_BYTES

    B.build()
    dev = torch.device("cuda", 0)
    scene, req = synth.workload_3d_large()
    n_vp = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    seg = n_vp * req["patches_u"] * req["patches_w"]
    ctx = Context(0)
    ctx.load_scene(scene)
    ctx.vcm_build(50.0)
    stream = torch.cuda.current_stream(dev)
    v = torch.empty(n_vp, dtype=torch.float32, device=dev)
    c = torch.empty(n_vp, dtype=torch.uint8, device=dev)
    st = torch.empty(STATS_BYTES, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(1, args.warmup)):
        ctx.vcm_compute(req, v.data_ptr(), c.data_ptr(), None, st.data_ptr(), stream.cuda_stream)
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.vcm_compute(req, v.data_ptr(), c.data_ptr(), None, st.data_ptr(), stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    stats = stats_from_tensor(st)
    out = {"mode": "large", "metric": METRIC, "unit": UNIT, "boxes": scene.n, "viewpoints": n_vp,
           "patches": [req["patches_u"], req["patches_w"]], "segments": seg, "ms_per_step": float(np.mean(ms)),
           "value": seg / (float(np.mean(ms)) / 1e3), "cells_per_s": n_vp / (float(np.mean(ms)) / 1e3),
           "stats": {k: stats[k] for k in ("slab_tests", "corner_tests", "shortcut_viewpoints", "rechecked",
                                           "boxes_listed")},
           "nonzero_cells": int((v > 0).sum().item())}
    if not args.no_cpu_baseline:
        r = oracle_rate(scene, req, args.cpu_seconds)
        out["cpu_baseline"] = {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                               "sample": "%d random viewpoints, %.1f s" % (r["viewpoints"], r["seconds"])}
    print(json.dumps(out), flush=True)
    ctx.close()


def run_gaze(args):
    """Incremental gaze change on the 3D workload (512 x 512 x 5 viewpoints,
    5,000 boxes, 32 x 16 patches): occlusion bits once, then one recolour per
    gaze direction (a 120 degree field of view turned in steps around the
    vertical) against a full recompute with the same gaze.  The recolour
    kernel reads ceil(P/32) words and writes one float per viewpoint; its
    roofline is HBM."""
    import math

    import torch

    import synth
    from paper_1310_7297_gb300 import Context
    from paper_1310_7297_gb300 import build as B
    from paper_1310_7297_gb300.vcm import STATS_BYTES

    B.build()
    dev = torch.device("cuda", 0)
    scene, req = synth.workload_3d()
    n_vp = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    P = req["patches_u"] * req["patches_w"]
    words = (P + 31) // 32
    ctx = Context(0)
    ctx.load_scene(scene)
    ctx.vcm_build(0.0)
    stream = torch.cuda.current_stream(dev)
    _, _, bits, _ = ctx.compute(req, emit_bits=True)
    v = torch.empty(n_vp, dtype=torch.float32, device=dev)
    c = torch.empty(n_vp, dtype=torch.uint8, device=dev)
    st = torch.empty(STATS_BYTES, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def gaze_req(k):
        a = math.radians(-60.0 + 120.0 * k / max(1, args.steps - 1))
        return dict(req, fov_deg=120.0, gaze=[math.sin(a), math.cos(a), 0.0])

    for k in range(max(1, args.warmup)):
        ctx.vcm_recolor(gaze_req(k), bits.data_ptr(), v.data_ptr(), c.data_ptr(), st.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    kb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ka = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for e in kb + ka:
        e.record(stream)
    torch.cuda.synchronize()
    rec, kern, full = [], [], []
    for k in range(args.steps):
        r = gaze_req(k)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx.vcm_set_timing_events(kb[k], ka[k])
        a.record(stream)
        ctx.vcm_recolor(r, bits.data_ptr(), v.data_ptr(), c.data_ptr(), st.data_ptr(), stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        ctx.vcm_set_timing_events(None, None)
        rec.append(a.elapsed_time(b))
        kern.append(kb[k].elapsed_time(ka[k]))
        flush.zero_()
        a.record(stream)
        ctx.vcm_compute(r, v.data_ptr(), c.data_ptr(), None, st.data_ptr(), stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        full.append(a.elapsed_time(b))
    k_ms = float(np.mean(kern))
    # words are read for the viewpoints in front of the one-sided target only
    # (the target faces req["normal"]); one float is written per viewpoint
    ax, sgn = req["normal"] >> 1, (-1 if req["normal"] & 1 else 1)
    coords = [(req["grid_origin"][k] + (np.arange(n) + 0.5) * req["grid_step"][k]) for k, n in
              ((0, req["grid_nx"]), (1, req["grid_ny"]))] + [np.asarray(req["layer_z"], np.float64)]
    per_axis = [req["grid_nx"], req["grid_ny"], len(req["layer_z"])]
    n_front = int(np.sum(sgn * (coords[ax] - req["center"][ax]) > 0)) * n_vp // per_axis[ax]
    bytes_per_launch = n_front * 4 * words + n_vp * 4
    peak = hbm_peak()
    achieved = bytes_per_launch / (k_ms / 1e3) / 1e9
    out = {"mode": "gaze", "workload": "3D plain VCM 512x512x5, 5,000 boxes, 32x16 patches; 120 degree field of "
                                      "view turned over 120 degrees in %d steps" % args.steps,
           "recolor_ms": float(np.mean(rec)), "full_recompute_ms": float(np.mean(full)),
           "speedup": float(np.mean(full)) / float(np.mean(rec)),
           "cells_per_s": n_vp / (float(np.mean(rec)) / 1e3),
           "roofline": {"bound": "hbm", "kernel": "k_recolor", "achieved": achieved, "peak": peak["value"],
                        "unit": "GB/s", "frac": achieved / peak["value"], "peak_basis": peak["basis"],
                        "bytes_per_launch": bytes_per_launch, "front_viewpoints": n_front, "kernel_ms": k_ms,
                        "traffic": None},
           "l2": "512 MB buffer written between timed calls"}
    print(json.dumps(out), flush=True)
    ctx.close()


def mode_variants(req):
    """(name, request) of each variant `--mode modes` times, derived from a
    target-centric request: plain, strict, a 120 degree field of view gazing
    along +y, both, two-sided, and the viewer-centric map over the same grid
    from a viewer at the target's centre."""
    import synth
    from paper_1310_7297_gb300 import VCM_STRICT, VCM_TWO_SIDED, VCM_VIEWER

    fov = dict(fov_deg=120.0, gaze=[0.0, 1.0, 0.0])
    g0, gs = [x / 1024 for x in req["grid_origin"]], [x / 1024 for x in req["grid_step"]]
    viewer = synth.make_request(3, tuple(c / 1024 for c in req["center"]), 0, 2, 1.0, 1, g0, gs,
                                (req["grid_nx"], req["grid_ny"]), layers_m=[z / 1024 for z in req["layer_z"]],
                                height_m=1.0, color_levels=16, flags=VCM_VIEWER)
    return [("plain", req), ("strict", dict(req, flags=VCM_STRICT)), ("fov120", dict(req, **fov)),
            ("strict_fov120", dict(req, flags=VCM_STRICT, **fov)), ("two_sided", dict(req, flags=VCM_TWO_SIDED)),
            ("viewer", viewer)]


def run_modes(args):
    """The visibility variants on the 3D workload (512 x 512 x 5 viewpoints,
    5,000 boxes, 32 x 16 patches), each timed like the step (inputs resident,
    L2 flushed between steps) with its ALU roofline, and the CPU oracle on a
    bounded sample of the same variant: plain (the step), strict (completely
    visible), a 120 degree field of view, both, a two-sided target, and the
    viewer-centric map from a viewer at the target's centre (one segment per
    cell)."""
    import torch

    import synth
    from paper_1310_7297_gb300 import VCM_VIEWER, Context, stats_from_tensor
    from paper_1310_7297_gb300 import build as B
    from paper_1310_7297_gb300.vcm import STATS_BYTES

    B.build()
    dev = torch.device("cuda", 0)
    scene, req = synth.workload_3d()
    n_vp = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    variants = mode_variants(req)
    ctx = Context(0)
    ctx.load_scene(scene)
    ctx.vcm_build(0.0)
    stream = torch.cuda.current_stream(dev)
    v = torch.empty(n_vp, dtype=torch.float32, device=dev)
    c = torch.empty(n_vp, dtype=torch.uint8, device=dev)
    st = torch.empty(STATS_BYTES, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    pk = peaks()
    max_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak = alu_peak_ops(torch.cuda.get_device_properties(dev).multi_processor_count, max_mhz)
    results = []
    for name, r in variants:
        P = 1 if r.get("flags", 0) & VCM_VIEWER else r["patches_u"] * r["patches_w"]
        for _ in range(max(3, args.warmup)):
            ctx.vcm_compute(r, v.data_ptr(), c.data_ptr(), None, st.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        kb, ka = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kb.record(stream)   # torch creates an event's handle on its first record
        ka.record(stream)
        torch.cuda.synchronize()
        step, kern = [], []
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ctx.vcm_set_timing_events(kb, ka)
            a.record(stream)
            ctx.vcm_compute(r, v.data_ptr(), c.data_ptr(), None, st.data_ptr(), stream.cuda_stream)
            b.record(stream)
            torch.cuda.synchronize()
            ctx.vcm_set_timing_events(None, None)
            step.append(a.elapsed_time(b))
            kern.append(kb.elapsed_time(ka))
        stats = stats_from_tensor(st)
        ms, k_ms = float(np.mean(step)), float(np.mean(kern))
        ops = (stats["slab_tests"] + stats["corner_tests"]) * OPS_PER_SLAB_TEST[r["dims"]]
        row = {"name": name, "flags": int(r.get("flags", 0)), "ms_per_step": ms, "kernel_ms": k_ms,
               "segments_per_s": n_vp * P / (ms / 1e3), "cells_per_s": n_vp / (ms / 1e3),
               "nonzero_cells": int((v > 0).sum().item()),
               "roofline": {"bound": "alu", "achieved": ops / (k_ms / 1e3) / 1e12, "peak": peak / 1e12,
                            "unit": "Tops/s", "frac": ops / (k_ms / 1e3) / peak}}
        if not args.no_cpu_baseline:
            o = oracle_rate(scene, r, max(1.0, args.cpu_seconds / len(variants)), seed=len(results))
            row["cpu_oracle"] = {"segments_per_s": o["cells_per_s"] * P, "cells_per_s": o["cells_per_s"],
                                 "cores": o["cores"], "sample": "%d random viewpoints, %.1f s" % (o["viewpoints"],
                                                                                               o["seconds"])}
        results.append(row)
    print(json.dumps({"mode": "modes", "workload": WORKLOAD, "steps": args.steps,
                      "l2": "512 MB buffer written between timed steps", "results": results}), flush=True)
    ctx.close()


def run_equivisible(args):
    """The paper's own equi-visible colouring (distance and angle partition,
    a colour per cell from its centre; CPU) against the dense GPU map of the
    same 2D target, by the error of Eq. 6, for the angular resolutions of
    Table II.  No obstacles: the partition is the paper's step before it
    accounts for them.  Target: a 10 m segment facing +y; grid: 1024 x 1024
    cells over 1 km; 16 colour levels, each map normalised by its own
    maximum; the near point is 1 m."""
    import torch

    import synth
    from paper_1310_7297_gb300 import Context
    from paper_1310_7297_gb300 import build as B
    from paper_1310_7297_gb300 import equivisible as E

    B.build()
    S, n, half, levels = 10.0, 1024, 500.0, 16
    scene = synth.Scene(2, np.zeros((0, 3), np.int64), np.zeros((0, 3), np.int64))
    req = synth.make_request(2, (0.0, 0.0), synth.AXIS_PX, synth.AXIS_PY, S, 64, (-half, -half),
                             (2 * half / n, 2 * half / n), (n, n), color_levels=levels)
    ctx = Context(0)
    ctx.load_scene(scene)
    ctx.vcm_build(0.0)
    t0 = time.perf_counter()
    v, c, _, _ = ctx.compute(req)
    torch.cuda.synchronize()
    gpu_ms = 1e3 * (time.perf_counter() - t0)
    c_dense = c.cpu().numpy().astype(np.int64)
    xs = -half + (np.arange(n) + 0.5) * (2 * half / n)
    X, Y = np.meshgrid(xs, xs)
    X, Y = X.ravel(), Y.ravel()

    def subtended(D, a_deg):
        # exact angle subtended by the segment from a point at distance D and
        # viewing angle a (the limit of the dense map's sum)
        a = np.radians(a_deg)
        px, py = D * np.cos(a), D * np.sin(a)
        return np.abs(np.arctan2(py, px - S / 2) - np.arctan2(py, px + S / 2))

    rows = []
    for mu in (1, 2, 4, 8, 16):
        t1 = time.perf_counter()
        P = E.Partition(S, mu, 1.0)
        vp = P.values_at(X, Y)
        cpu_s = time.perf_counter() - t1
        c_paper = E.quantise(vp, levels)
        c_same = E.quantise(P.values_at(X, Y, subtended), levels)
        inside = np.hypot(X, Y) < P.d_edges[-1]
        rows.append({"mu_deg": mu, "cells": P.n_cells(), "d_max_m": float(P.d_edges[-1]), "cpu_s": cpu_s,
                     "eq6_paper_measure": E.eq6_error(c_dense, c_paper),
                     "eq6_paper_measure_within_d_max": E.eq6_error(c_dense[inside], c_paper[inside]),
                     "eq6_same_measure": E.eq6_error(c_dense, c_same),
                     "eq6_same_measure_within_d_max": E.eq6_error(c_dense[inside], c_same[inside]),
                     "mean_abs_colour_diff_within_d_max": float(np.mean(np.abs(c_dense[inside] - c_same[inside])))})
    print(json.dumps({"mode": "equivisible", "workload": "2D, 10 m target, 1024 x 1024 cells over 1 km, no "
                      "obstacles, 16 levels", "dense_gpu_ms": gpu_ms, "rows": rows}), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=["step", "batched", "serve", "large", "gaze", "equivisible", "modes"],
                    default="step",
                    help="step: the timed VCM step (default); batched / serve: the batching and serving runs; "
                         "large: the 100,000-box scene at full size; gaze: recolouring for new gazes; "
                         "equivisible: the paper's equi-visible cells against the dense map (Eq. 6); "
                         "modes: strict, field of view, two-sided and viewer-centric variants of the step")
    ap.add_argument("--batch-requests", type=int, default=256)
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--serve-count", type=int, default=400)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--rates", type=float, nargs="+", default=[50, 100, 200, 500, 1000, 2000])
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=8)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "large":
        run_large(args)
    elif args.mode == "gaze":
        run_gaze(args)
    elif args.mode == "equivisible":
        run_equivisible(args)
    elif args.mode == "modes":
        run_modes(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
