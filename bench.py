#!/usr/bin/env python3
"""Benchmark of the visibility color map (VCM) path on GB300.

Headline workload (one step = one whole VCM: grid-index cull, slab tests,
visible measure, quantisation): the large 3D scene - 100,000 boxes over
10 km x 10 km (footprints 10-60 m, lognormal heights with median 20 m and
sigma 0.6, centres from a 64-component Gaussian mixture), one 40 m x 20 m
target at 30 m split into 64 x 32 patches, 2048 x 2048 viewpoints on 8
layers from 1.7 m spaced 10 m, a 50 m uniform-grid index, 16 color levels.
It is the largest of the single-GPU workloads.  Seeded synthetic inputs
stand in for the paper's city datasets.

The same JSON line carries sub-records, each with its own clock window:
the 3D workload of 5,000 boxes (512 x 512 x 5 viewpoints, 32 x 16
patches), the 256-request uneven mix in one persistent launch against one
launch per request, and serving (Poisson arrivals at 50-2,000 req/s against
the resident 100,000-box scene) against a FIFO of one launch per request.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
Under torchrun each rank runs its own full copy of the headline workload
(weak scaling, no data-path collective) and the slowest rank's time is
reported; the sub-records run at N = 1 only.
"""

import argparse
import ctypes
import gc
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
WORKLOAD = ("3D large scene: {g}x{g} viewpoints x {l} layers, 100,000 mixture boxes over 10 km, "
            "40x20 m target, 64x32 patches, 50 m grid index")
WORKLOAD_3D = "3D plain VCM: 512x512 viewpoints x 5 layers, 5,000 mixture boxes over 2 km, 20x10 m target, 32x16 patches"
GRID_CELL_LARGE_M = 50.0
# Algorithmic work of one segment/box slab test: per axis the entry and exit
# parameters (a multiply each; the differences to the box faces are shared
# per viewpoint and box), their min/max, and the running max of entries and
# min of exits, then one compare: 6 FMUL + 12 FMNMX + 1 compare = 19 FP32
# operations in 3D, 13 in 2D.  Every test the tile kernel counts (row tests
# of the sweep, corner tests of the one-box checks) decides one
# segment/box pair.  The separable sweep itself issues only ~6 lane
# operations per row test (two selects, two fused w-margins, their max and a
# compare), sharing the u and n parts across a column's rows; those are
# reported beside the fraction.
OPS_PER_SLAB_TEST = {3: 19, 2: 13}
ISSUED_OPS_PER_ROW_TEST = 6
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


KERNEL_SRC = os.path.join(ROOT, "paper_1310_7297_gb300", "csrc", "vcm_kernels.cu")
PROFILE_LARGE = os.path.join(ROOT, "profiles", "k_tiles_3d_large_2048x2048x8_100000boxes.md")
PROFILE_3D = os.path.join(ROOT, "profiles", "k_tiles_3d_512x512x5_5000boxes.md")


def profiled_traffic(profile):
    """DRAM bytes per k_tiles launch (both passes) of the workload a
    committed ncu summary covers, or None if the kernel source has changed
    since that capture."""
    import hashlib

    try:
        text = open(profile).read()
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
    """nvidia-smi clocks and throttle reasons sampled every 200 ms for the
    whole run; ``window`` summarises the samples of one timed region."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.t = None
        self.lock = threading.Lock()

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return self
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            with self.lock:
                self.lines.append((time.monotonic(), line.strip()))

    def window(self, t_from, t_to, what=""):
        """Summary of the samples taken between t_from and t_to (monotonic)."""
        if self.proc is None:
            return None
        # a sample of the last 200 ms may still be in the pipe
        deadline = time.monotonic() + 0.5
        while time.monotonic() < deadline:
            with self.lock:
                if self.lines and self.lines[-1][0] >= t_to:
                    break
            time.sleep(0.05)
        with self.lock:
            lines = list(self.lines)
        rows = []
        for ts, l in lines:
            if ts < t_from or ts > t_to:
                continue
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 9 or (self.uuid and self.uuid not in parts[0]):
                continue
            rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = sorted({self.NAMES[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        out = {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": reasons, "samples": len(rows)}
        if what:
            out["window"] = "%.2f s: %s" % (t_to - t_from, what)
        return out

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)


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


def headline_workload(grid=2048, layers=8):
    import synth

    return synth.workload_3d_large(grid=grid, layers=layers)


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_rate(scene, req, seconds, seed=0, rate_hint=None):
    """Segments/s of the CPU oracle on seeded random viewpoint samples that
    add up to about `seconds` of wall time, on all host cores.  A probe of
    64 viewpoints (skipped when a viewpoint rate is given) sets the first
    sample's size; further samples (at most four in all) top the time up,
    each sized from the rate measured so far."""
    from oracle import oracle as O

    O.build()
    n = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    P = req["patches_u"] * req["patches_w"]
    rng = np.random.default_rng(seed)
    if rate_hint:
        rate = float(rate_hint)
    else:
        probe = np.sort(rng.choice(n, min(n, 64), replace=False))
        t0 = time.perf_counter()
        O.run(scene, req, indices=probe)
        rate = probe.size / max(time.perf_counter() - t0, 1e-6)
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


def config_dict(scene, req, workload=WORKLOAD, grid_cell_m=GRID_CELL_LARGE_M):
    n_vp = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    return {"workload": workload.format(g=req["grid_nx"], l=len(req["layer_z"])), "viewpoints": n_vp, "grid": [req["grid_nx"], req["grid_ny"]],
            "layers_m": [z / 1024 for z in req["layer_z"]], "patches": [req["patches_u"], req["patches_w"]],
            "boxes": scene.n, "scene_digest": scene.digest(), "color_levels": req["color_levels"],
            "grid_index_cell_m": grid_cell_m,
            "segments_per_step": n_vp * req["patches_u"] * req["patches_w"],
            "l2": "512 MB buffer written between timed steps (outputs of 168 MB also exceed L2)",
            "parallelism": "replicas"}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    scene, req = headline_workload(args.grid, args.layers)
    # bounded: the whole run takes about 90 s of oracle time
    per_step = max(1.5, 90.0 / max(1, args.steps + args.warmup))
    rate = None
    for i in range(args.warmup):
        rate = oracle_rate(scene, req, per_step / 2, seed=100 + i, rate_hint=rate)["cells_per_s"]
    rates, secs, vps, cores = [], [], 0, 1
    for i in range(args.steps):
        r = oracle_rate(scene, req, per_step, seed=i, rate_hint=rate)
        rate = r["cells_per_s"]
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


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def _device_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u[4:] if u.startswith("GPU-") else u
    except Exception:
        return None


def time_direct(ctx, req, steps, warmup, stream, flush, sampler, what, preload_s=0.6, pg=None):
    """Time `steps` direct calls (vcm_compute into device buffers) after
    `warmup` untimed ones; L2 flushed before every call.  The same call also
    runs untimed for about `preload_s` just before the timed region, so that
    the clock samples (every 200 ms) cover that load; the clock window spans
    both.  Returns per-step and per-k_tiles times (CUDA events on the launch
    stream), the device counters and the output tensors."""
    import torch

    from paper_1310_7297_gb300 import n_viewpoints, stats_from_tensor
    from paper_1310_7297_gb300.vcm import STATS_BYTES

    dev = torch.device("cuda", ctx.device)
    n_vp = n_viewpoints(req)
    v = torch.empty(n_vp, dtype=torch.float32, device=dev)
    col = torch.empty(n_vp, dtype=torch.uint8, device=dev)
    st = torch.empty(STATS_BYTES, dtype=torch.uint8, device=dev)

    def step():
        ctx.vcm_compute(req, v.data_ptr(), col.data_ptr(), None, st.data_ptr(), stream.cuda_stream)

    for _ in range(warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t_load = time.monotonic()
    while time.monotonic() - t_load < preload_s:
        for _ in range(4):
            flush.zero_()
            step()
        torch.cuda.synchronize()
    s_ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e_ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    kb = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ka = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for e in kb + ka:
        e.record(stream)   # torch creates the CUDA event on first record; the library re-records it
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        ctx.vcm_set_timing_events(kb[i], ka[i])
        s_ev[i].record(stream)
        step()
        e_ev[i].record(stream)
    torch.cuda.synchronize()
    t_end = time.monotonic()
    ctx.vcm_set_timing_events(None, None)
    return {"step_ms": [s.elapsed_time(e) for s, e in zip(s_ev, e_ev)],
            "kern_ms": [b.elapsed_time(a) for b, a in zip(kb, ka)],
            "stats": stats_from_tensor(st), "v": v, "color": col,
            "clocks": sampler.window(t_load, t_end, what) if sampler else None}


def alu_roofline(stats, dims, kern_ms, sm_count, profile=None):
    """ALU roofline of k_tiles (both passes): the device-counted slab tests
    x their algorithmic operations over the passes' CUDA-event time."""
    max_mhz = float(peaks().get("sm_max_mhz", 2070.0))
    peak = alu_peak_ops(sm_count, max_mhz)
    kern_s = float(np.mean(kern_ms)) / 1e3
    units = stats["slab_tests"] + stats["corner_tests"]
    achieved = units * OPS_PER_SLAB_TEST[dims] / kern_s
    issued = (stats["slab_tests"] * ISSUED_OPS_PER_ROW_TEST + stats["corner_tests"] * ISSUED_OPS_PER_CORNER_TEST) / kern_s
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
            "frac": achieved / peak, "traffic": profiled_traffic(profile) if profile else None,
            "kernel": "k_tiles (both passes)", "work_unit": "segment/box slab test",
            "ops_per_unit": OPS_PER_SLAB_TEST[dims],
            "issued_slab_ops": {"value": issued / 1e12, "frac": issued / peak,
                                "ops_per_row_test": ISSUED_OPS_PER_ROW_TEST,
                                "ops_per_corner_test": ISSUED_OPS_PER_CORNER_TEST},
            "units_per_launch": units, "kernel_ms": float(np.mean(kern_ms)),
            "peak_basis": "%d SMs x 128 lane-instr/clk x %.0f MHz (issue limit; derived, "
                          "MEASURED_PEAKS.json has no ALU figure)" % (sm_count, max_mhz)}


def executed(stats, v, ms):
    """What the device actually did, beside the nominal segment rate."""
    s = ms / 1e3
    return {"nonzero_cells": int((v > 0).sum().item()), "slab_tests": stats["slab_tests"],
            "corner_tests": stats["corner_tests"], "slab_tests_per_s": stats["slab_tests"] / s,
            "corner_tests_per_s": stats["corner_tests"] / s,
            "shortcut_viewpoints": stats["shortcut_viewpoints"], "shared_viewpoints": stats["shared_viewpoints"],
            "rechecked": stats["rechecked"], "boxes_listed": stats["boxes_listed"],
            "edge_cells": stats["edge_cells"], "v_ref": stats["v_ref"]}


def run_gpu(args):
    import torch

    from paper_1310_7297_gb300 import Context
    from paper_1310_7297_gb300 import build as B
    from paper_1310_7297_gb300.vcm import STATS_BYTES, vcm_request

    world, rank, local = dist_setup()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    scene, req = headline_workload(args.grid, args.layers)
    n_vp = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    P = req["patches_u"] * req["patches_w"]
    seg = n_vp * P
    ctx = Context(local)
    ctx.load_scene(scene)
    ctx.vcm_build(GRID_CELL_LARGE_M)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sampler = ClockSampler(_device_uuid(torch, dev)).start()
    time.sleep(0.3)
    K = args.steps
    head = time_direct(ctx, req, K, args.warmup, stream, flush, sampler,
                       "the same step untimed, then the timed region", preload_s=args.preload_s, pg=pg)
    total_ms = reduce_max(float(sum(head["step_ms"])), pg, dev)
    if pg:
        pg.barrier()
    stats = head["stats"]

    # End to end through the public API with host buffers.  Headline: the
    # scene is a resident database (uploaded and indexed once, as the
    # paper's obstacle set is), and each step submits the request, waits for
    # it and reads its values and colours back into host memory, with two
    # steps in flight as a server keeps them (the scheduler chains their
    # launches, so one step's read-back overlaps the next one's kernels).
    # Also reported: one step at a time, and the scene uploaded and
    # re-indexed every step (a scene load waits for an idle context, so that
    # loop runs one step at a time).
    lo = torch.from_numpy(scene.lo_f32()[:, :3].copy()).pin_memory().numpy()
    hi = torch.from_numpy(scene.hi_f32()[:, :3].copy()).pin_memory().numpy()

    def e2e_loop(with_scene):
        ms, chk = [], 0.0
        for i in range(args.warmup + K):
            t0 = time.perf_counter()
            if with_scene:
                ctx.vcm_scene_load_mem(lo, hi, 3)
                ctx.vcm_build(GRID_CELL_LARGE_M)
            t = ctx.vcm_submit(req)
            ctx.vcm_poll(t, -1)
            hv, hc, _, _ = ctx.vcm_result_get(t, copy=False)
            chk += float(hv[-1]) + int(hc[-1])
            ctx.vcm_result_release(t)
            if i >= args.warmup:
                ms.append(1e3 * (time.perf_counter() - t0))
        return ms

    def e2e_pipelined(depth=2):
        chk = 0.0

        def run(n):
            nonlocal chk
            pending = []
            for _ in range(n):
                pending.append(ctx.vcm_submit(req))
                if len(pending) == depth:
                    t = pending.pop(0)
                    ctx.vcm_poll(t, -1)
                    hv, hc, _, _ = ctx.vcm_result_get(t, copy=False)
                    chk += float(hv[-1]) + int(hc[-1])
                    ctx.vcm_result_release(t)
            for t in pending:
                ctx.vcm_poll(t, -1)
                hv, hc, _, _ = ctx.vcm_result_get(t, copy=False)
                chk += float(hv[-1]) + int(hc[-1])
                ctx.vcm_result_release(t)

        run(args.warmup)
        t0 = time.perf_counter()
        run(K)
        return [1e3 * (time.perf_counter() - t0) / K] * K

    t_e2e = time.monotonic()
    e2e_scene_ms = e2e_loop(True)
    e2e_seq_ms = e2e_loop(False)
    e2e_ms = e2e_pipelined()
    e2e_clocks = sampler.window(t_e2e, time.monotonic(), "both end-to-end loops")
    e2e_scene_total = reduce_max(float(sum(e2e_scene_ms)), pg, dev)
    e2e_total = reduce_max(float(sum(e2e_ms)), pg, dev)
    e2e_seq_total = reduce_max(float(sum(e2e_seq_ms)), pg, dev)

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras["config_3d_5000_boxes"] = sub_3d(ctx, args, stream, flush, sampler)
        extras["batched"] = sub_batched(ctx, args, stream, sampler)
        extras["serve"] = sub_serve(ctx, args, sampler)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_rate(scene, req, args.cpu_seconds)
        cpu = {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
               "sample": "%d random viewpoints of the workload (%d patches each), %.1f s of CPU work"
                         % (r["viewpoints"], P, r["seconds"])}
    sampler.stop()

    # the request as uploaded: its descriptor and the coordinates the library
    # derives from it (patch centres, viewpoint x, y, layer heights)
    req_bytes = int(ctypes.sizeof(vcm_request) + 4 * (req["patches_u"] + req["patches_w"] + req["grid_nx"] +
                                                       req["grid_ny"] + len(req["layer_z"])))
    if rank == 0:
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        value = world * seg * K / (total_ms / 1e3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": config_dict(scene, req),
            "cells_per_s": world * n_vp * K / (total_ms / 1e3),
            "kernel_ms": float(np.mean(head["kern_ms"])),
            "roofline": alu_roofline(stats, req["dims"], head["kern_ms"], sm_count, PROFILE_LARGE),
            "executed": executed(stats, head["v"], total_ms / K),
            "cpu_baseline": cpu,
            "e2e": {"value": world * seg * K / (e2e_total / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": req_bytes, "d2h_bytes_per_step": int(n_vp * 5 + STATS_BYTES),
                    "ms_per_step": e2e_total / K,
                    "path": "vcm_submit, vcm_poll, vcm_result_get (values and colours into pinned host memory); "
                            "scene resident, uploaded and indexed once; two steps in flight",
                    "one_at_a_time_ms_per_step": e2e_seq_total / K,
                    "clocks": e2e_clocks},
            "e2e_scene_per_step": {"value": world * seg * K / (e2e_scene_total / 1e3), "unit": UNIT,
                                   "h2d_bytes_per_step": int(lo.nbytes + hi.nbytes) + req_bytes,
                                   "d2h_bytes_per_step": int(n_vp * 5 + STATS_BYTES),
                                   "ms_per_step": e2e_scene_total / K,
                                   "path": "vcm_scene_load_mem and vcm_build every step, then as e2e"},
            "gpu_launches": LAUNCHES_PER_STEP * K,
            "clocks": head["clocks"],
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()


def sub_3d(ctx, args, stream, flush, sampler):
    """The 3D workload of 5,000 boxes (512 x 512 x 5 viewpoints, 32 x 16
    patches), timed like the headline."""
    import torch

    import synth

    scene, req = synth.workload_3d()
    ctx.load_scene(scene)
    ctx.vcm_build(0.0)
    n_vp = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    seg = n_vp * req["patches_u"] * req["patches_w"]
    r = time_direct(ctx, req, args.steps, args.warmup, stream, flush, sampler,
                    "the same step untimed, then the timed region", preload_s=args.preload_s)
    ms = float(np.mean(r["step_ms"]))
    sm_count = torch.cuda.get_device_properties(stream.device).multi_processor_count
    return {"workload": WORKLOAD_3D, "boxes": scene.n, "scene_digest": scene.digest(), "value": seg / (ms / 1e3),
            "unit": UNIT, "ms_per_step": ms, "cells_per_s": n_vp / (ms / 1e3),
            "roofline": alu_roofline(r["stats"], 3, r["kern_ms"], sm_count, PROFILE_3D),
            "executed": executed(r["stats"], r["v"], ms), "clocks": r["clocks"]}


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


def sub_batched(ctx, args, stream, sampler, autotune=False):
    """The 256-request uneven mix over a shared 50,000-box scene: one
    persistent launch (default shapes; with autotune also the tuned shapes)
    against one launch per request, each timed with CUDA events on the
    launch stream; the persistent launch's ALU roofline from the device
    counters over the tile kernel's event time."""
    import torch

    import synth
    from paper_1310_7297_gb300 import n_viewpoints, stats_from_tensor
    from paper_1310_7297_gb300.vcm import STATS_BYTES

    dev = torch.device("cuda", ctx.device)
    scene, reqs = synth.workload_batched(n_requests=args.batch_requests)
    seg = sum(n_viewpoints(r) * r["patches_u"] * r["patches_w"] for r in reqs)
    ctx.load_scene(scene)
    ctx.vcm_build(50.0)
    vs, cs, st = _alloc_outputs(torch, dev, reqs)
    steps = max(1, min(args.steps, 10))

    def batch():
        ctx.vcm_compute_batch(reqs, [t.data_ptr() for t in vs], [t.data_ptr() for t in cs], [None] * len(reqs),
                              st.data_ptr(), stream.cuda_stream)

    def singles():
        for i, r in enumerate(reqs):
            ctx.vcm_compute(r, vs[i].data_ptr(), cs[i].data_ptr(), None, st.data_ptr() + STATS_BYTES * i,
                            stream.cuda_stream)

    def timed(fn, what):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        t0 = time.monotonic()
        ms, kern = [], []
        kb, ka = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kb.record(stream)
        ka.record(stream)
        torch.cuda.synchronize()
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ctx.vcm_set_timing_events(kb, ka)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ctx.vcm_set_timing_events(None, None)
            ms.append(a.elapsed_time(b))
            kern.append(kb.elapsed_time(ka))
        m = float(np.median(ms))
        return {"ms": m, "segments_per_s": seg / (m / 1e3), "steps": steps, "kern_ms": kern,
                "clocks": sampler.window(t0, time.monotonic(), what) if sampler else None}

    res = {"workload": "256 uneven requests (2-50 m targets, 64^2-1024^2 x 1-8 layer grids, 8x4-64x32 patches) "
                       "over a shared 50,000-box scene", "requests": len(reqs), "boxes": scene.n, "segments": seg,
           "unit": UNIT}
    res["persistent_batch"] = timed(batch, "the persistent batch, timed")
    if autotune:
        t0 = time.perf_counter()
        pick = np.random.default_rng(7).choice(len(reqs), size=min(16, len(reqs)), replace=False)
        tuned = ctx.vcm_autotune([reqs[i] for i in sorted(pick)])
        res["autotune_s"] = time.perf_counter() - t0
        res["tuned_shapes"] = sorted(set(map(tuple, tuned)))
        res["persistent_batch_tuned"] = timed(batch, "the persistent batch with tuned shapes, timed")
    batch()
    torch.cuda.synchronize()
    per = [stats_from_tensor(st[i * STATS_BYTES:(i + 1) * STATS_BYTES]) for i in range(len(reqs))]
    tot = {k: sum(p[k] for p in per) for k in ("slab_tests", "corner_tests", "shortcut_viewpoints",
                                               "shared_viewpoints", "rechecked")}
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    pb = res["persistent_batch"]
    pb["roofline"] = alu_roofline(tot, 3, pb.pop("kern_ms"), sm_count)
    pb["executed"] = {k: tot[k] for k in tot}
    pb["executed"]["nonzero_cells"] = int(sum(int((t > 0).sum().item()) for t in vs))
    if "persistent_batch_tuned" in res:
        res["persistent_batch_tuned"].pop("kern_ms")
    res["one_per_launch"] = timed(singles, "one launch per request, timed")
    res["one_per_launch"].pop("kern_ms")
    res["speedup"] = res["one_per_launch"]["ms"] / res["persistent_batch"]["ms"]
    del vs, cs, st
    return res


def sub_serve(ctx, args, sampler):
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
    from paper_1310_7297_gb300 import n_viewpoints
    from paper_1310_7297_gb300.vcm import STATS_BYTES

    dev = torch.device("cuda", ctx.device)
    scene, _ = synth.workload_3d_large(grid=64, layers=1)
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

    def sched_one(r):
        t = ctx.vcm_submit(r)
        ctx.vcm_poll(t, -1)
        ctx.vcm_result_release(t)

    def busy(run_one, seconds=0.5):
        t_end, k = time.monotonic() + seconds, 0
        while time.monotonic() < t_end:
            run_one(pool[k % len(pool)])
            k += 1

    for r in pool:
        fifo_one(r)
    # warm the scheduler path too: every request once, alone and in a burst
    for r in pool[:16]:
        t = ctx.vcm_submit(r)
        ctx.vcm_poll(t, -1)
        ctx.vcm_result_release(t)
    for t in [ctx.vcm_submit(r) for r in pool]:
        ctx.vcm_poll(t, -1)
        ctx.vcm_result_release(t)
    out = []
    t_start = time.monotonic()
    for rate in args.rates:
        n = int(min(args.serve_count, max(40, rate * args.serve_seconds)))
        arr = synth.poisson_arrivals(int(rate), float(rate), n)
        picks = [pool[i % len(pool)] for i in range(n)]
        seg = sum(seg_of[i % len(pool)] for i in range(n))
        # No garbage collection during the arms (a stalled harness thread is
        # not a latency of either path), and each arm starts on a busy GPU:
        # 0.5 s of back-to-back requests through its own path first.  After
        # half a second idle the next large request ran up to twice as long
        # (3.9-6.6 ms against 3.34), in either arm.
        gc.collect()
        gc.disable()
        busy(fifo_one)

        # FIFO server, one request per launch
        q = _queue.Queue()
        done = [0.0] * n
        began = [0.0] * n

        def worker():
            for _ in range(n):
                i, t0 = q.get()
                began[i] = time.perf_counter() - t0
                fifo_one(picks[i])
                done[i] = time.perf_counter() - t0

        th = threading.Thread(target=worker)
        t_w = time.monotonic()
        th.start()
        t0 = time.perf_counter()
        for i in range(n):
            now = time.perf_counter() - t0
            if arr[i] > now:
                time.sleep(arr[i] - now)
            q.put((i, t0))
        th.join()
        t_fifo = (t_w, time.monotonic())
        lat = [1e3 * (done[i] - arr[i]) for i in range(n)]
        slow = np.argsort(lat)[-3:][::-1]
        fifo = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "segments_per_s": seg / max(done),
                "median_wait_ms": float(np.median([1e3 * (began[i] - arr[i]) for i in range(n)])),
                "median_service_ms": float(np.median([1e3 * (done[i] - began[i]) for i in range(n)])),
                "slowest": [{"request": int(i), "arrival_ms": 1e3 * arr[i], "latency_ms": lat[i],
                             "wait_ms": 1e3 * (began[i] - arr[i]), "service_ms": 1e3 * (done[i] - began[i]),
                             "segments": seg_of[i % len(pool)]} for i in slow]}

        # continuous batching through the scheduler; a consumer thread takes
        # each result as it is done and releases it, as a server would
        q2 = _queue.Queue()
        lat2, info = [0.0] * n, [None] * n

        def consumer():
            for _ in range(n):
                i, t, ts = q2.get()
                ctx.vcm_poll(t, -1)
                _, hc, _, stt = ctx.vcm_result_get(t, copy=False)
                lat2[i] = (ts - arr[i]) * 1e3 + stt["latency_ms"]
                info[i] = {k: stt[k] for k in ("queue_ms", "device_ms", "chain_ms", "launch_ms", "group_size",
                                               "launch_form")}
                ctx.vcm_result_release(t)

        busy(sched_one)
        th2 = threading.Thread(target=consumer)
        th2.start()
        t_w = time.monotonic()
        t0 = time.perf_counter()
        for i in range(n):
            now = time.perf_counter() - t0
            if arr[i] > now:
                time.sleep(arr[i] - now)
            ts = time.perf_counter() - t0   # the library times from here to completion
            q2.put((i, ctx.vcm_submit(picks[i]), ts))
        th2.join()
        t_cont = (t_w, time.monotonic())
        gc.enable()
        # clock windows once both arms are done (their wait for the last
        # sample would otherwise idle the GPU before the second arm)
        fifo["clocks"] = sampler.window(*t_fifo, "FIFO arm")
        last = max(arr[i] + lat2[i] / 1e3 for i in range(n))
        slow = np.argsort(lat2)[-3:][::-1]
        cont = {"p50_ms": float(np.percentile(lat2, 50)), "p99_ms": float(np.percentile(lat2, 99)),
                "segments_per_s": seg / last, "clocks": sampler.window(*t_cont, "continuous arm"),
                "persistent_launch_share": float(np.mean([x["launch_form"] == 0 for x in info])),
                "mean_group_size": float(np.mean([x["group_size"] for x in info])),
                "median_queue_ms": float(np.median([x["queue_ms"] for x in info])),
                "median_device_ms": float(np.median([x["device_ms"] for x in info])),
                "median_chain_ms": float(np.median([x["chain_ms"] for x in info])),
                "median_host_ms": float(np.median([lat2[i] - info[i]["queue_ms"] - info[i]["device_ms"]
                                                   for i in range(n)])),
                "slowest": [dict(request=int(i), arrival_ms=1e3 * arr[i], latency_ms=lat2[i], fifo_latency_ms=lat[i],
                                 segments=seg_of[i % len(pool)], **info[i]) for i in slow]}
        for x in fifo["slowest"]:   # the same requests in the other arm
            x["continuous_latency_ms"] = lat2[x["request"]]
        out.append({"rate_per_s": rate, "requests": n, "continuous": cont, "one_per_launch_fifo": fifo})
    ctx.vcm_set_slots(2, 64)
    return {"workload": "Poisson arrivals of requests from the batched mix against a resident 100,000-box scene",
            "unit": UNIT, "boxes": scene.n, "budget_gb": 64, "slots": args.slots, "max_batch": args.max_batch,
            "rates": out, "clocks": sampler.window(t_start, time.monotonic(), "all rates, both arms")}


def _standalone(args, fn, **kw):
    """Run one sub-record on its own (a --mode) with its own context."""
    import torch

    from paper_1310_7297_gb300 import Context
    from paper_1310_7297_gb300 import build as B

    B.build()
    dev = torch.device("cuda", 0)
    sampler = ClockSampler(_device_uuid(torch, dev)).start()
    time.sleep(0.3)
    ctx = Context(0, 64 << 30)
    try:
        return fn(ctx, args, sampler=sampler, **kw)
    finally:
        sampler.stop()
        ctx.close()


def run_batched(args):
    import torch

    out = _standalone(args, lambda ctx, a, sampler: sub_batched(ctx, a, torch.cuda.current_stream(), sampler,
                                                                autotune=True))
    print(json.dumps(dict(mode="batched", metric=METRIC, **out)), flush=True)


def run_serve(args):
    out = _standalone(args, sub_serve)
    print(json.dumps(dict(mode="serve", metric=METRIC, **out)), flush=True)


def run_step3d(args):
    import torch

    def fn(ctx, a, sampler):
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        return sub_3d(ctx, a, torch.cuda.current_stream(), flush, sampler)

    out = _standalone(args, fn)
    print(json.dumps(dict(mode="step3d", metric=METRIC, **out)), flush=True)


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
    sampler = ClockSampler(_device_uuid(torch, dev)).start()
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
    t_w = time.monotonic()
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
    clocks = sampler.window(t_w, time.monotonic(), "recolours and full recomputes, alternating")
    sampler.stop()
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
           "l2": "512 MB buffer written between timed calls", "clocks": clocks}
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
    from paper_1310_7297_gb300 import VCM_VIEWER, Context
    from paper_1310_7297_gb300 import build as B

    B.build()
    dev = torch.device("cuda", 0)
    scene, req = synth.workload_3d()
    n_vp = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    variants = mode_variants(req)
    sampler = ClockSampler(_device_uuid(torch, dev)).start()
    ctx = Context(0)
    ctx.load_scene(scene)
    ctx.vcm_build(0.0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    results = []
    for name, r in variants:
        P = 1 if r.get("flags", 0) & VCM_VIEWER else r["patches_u"] * r["patches_w"]
        t = time_direct(ctx, r, args.steps, max(3, args.warmup), stream, flush, sampler,
                        "the variant untimed, then timed", preload_s=0.4)
        ms, stats = float(np.mean(t["step_ms"])), t["stats"]
        row = {"name": name, "flags": int(r.get("flags", 0)), "ms_per_step": ms,
               "kernel_ms": float(np.mean(t["kern_ms"])),
               "segments_per_s": n_vp * P / (ms / 1e3), "cells_per_s": n_vp / (ms / 1e3),
               "nonzero_cells": int((t["v"] > 0).sum().item()),
               "roofline": alu_roofline(stats, r["dims"], t["kern_ms"], sm_count), "clocks": t["clocks"]}
        if not args.no_cpu_baseline:
            o = oracle_rate(scene, r, max(1.0, args.cpu_seconds / len(variants)), seed=len(results))
            row["cpu_oracle"] = {"segments_per_s": o["cells_per_s"] * P, "cells_per_s": o["cells_per_s"],
                                 "cores": o["cores"], "sample": "%d random viewpoints, %.1f s" % (o["viewpoints"],
                                                                                               o["seconds"])}
        results.append(row)
    sampler.stop()
    print(json.dumps({"mode": "modes", "workload": WORKLOAD_3D, "steps": args.steps,
                      "l2": "512 MB buffer written between timed steps", "results": results}), flush=True)
    ctx.close()


EQUIVISIBLE_WORKLOAD = "2D, 10 m target, 1024 x 1024 cells over 1 km, no obstacles, 16 levels"


def equivisible_request(S=10.0, n=1024, half=500.0, levels=16, samples=64):
    """An empty 2D scene and the request of a segment target of length S at
    the origin facing +y over an n x n grid of 2 half metres a side."""
    import synth

    scene = synth.Scene(2, np.zeros((0, 3), np.int64), np.zeros((0, 3), np.int64))
    req = synth.make_request(2, (0.0, 0.0), synth.AXIS_PX, synth.AXIS_PY, S, samples, (-half, -half),
                             (2 * half / n, 2 * half / n), (n, n), color_levels=levels)
    return scene, req


def grid_centres(req):
    """Cell-centre x and y (metres) of a request's grid, flattened in output order."""
    n = req["grid_nx"]
    xs = (req["grid_origin"][0] + (np.arange(n) + 0.5) * req["grid_step"][0]) / 1024.0
    ys = (req["grid_origin"][1] + (np.arange(req["grid_ny"]) + 0.5) * req["grid_step"][1]) / 1024.0
    X, Y = np.meshgrid(xs, ys)
    return X.ravel(), Y.ravel()


def equivisible_dense(ctx, S=10.0, n=1024, half=500.0, levels=16, samples=64):
    """The dense GPU map of equivisible_request's target, no obstacles.
    Returns (request, device v, colours, cell-centre x, y as numpy)."""
    scene, req = equivisible_request(S, n, half, levels, samples)
    ctx.load_scene(scene)
    ctx.vcm_build(0.0)
    v, c, _, _ = ctx.compute(req)
    X, Y = grid_centres(req)
    return req, v, c.cpu().numpy().astype(np.int64), X, Y


def equivisible_row(c_dense, X, Y, mu, S=10.0, levels=16, d0=1.0):
    """Eq. 6 errors of the paper's partition at angular resolution mu against
    the dense map, with the paper's own measure (Eq. 1 with Eq. 2's
    perceived size) and with the dense map's measure (the exact subtended
    angle), over the grid and within the partition's range d_max."""
    from paper_1310_7297_gb300 import equivisible as E

    t1 = time.perf_counter()
    P = E.Partition(S, mu, d0)
    vp = P.values_at(X, Y)
    cpu_s = time.perf_counter() - t1
    c_paper = E.quantise(vp, levels)
    c_same = E.quantise(P.values_at(X, Y, lambda D, a: E.subtended(S, D, a)), levels)
    inside = np.hypot(X, Y) < P.d_edges[-1]
    return {"mu_deg": mu, "cells": P.n_cells(), "d_max_m": float(P.d_edges[-1]), "cpu_s": cpu_s,
            "eq6_paper_measure": E.eq6_error(c_dense, c_paper),
            "eq6_paper_measure_within_d_max": E.eq6_error(c_dense[inside], c_paper[inside]),
            "eq6_same_measure": E.eq6_error(c_dense, c_same),
            "eq6_same_measure_within_d_max": E.eq6_error(c_dense[inside], c_same[inside]),
            "mean_abs_colour_diff_within_d_max": float(np.mean(np.abs(c_dense[inside] - c_same[inside])))}


def run_equivisible(args):
    """The paper's own equi-visible colouring (distance and angle partition,
    a colour per cell from its centre; CPU) against the dense GPU map of the
    same 2D target, by the error of Eq. 6, for the angular resolutions of
    Table II.  No obstacles: the partition is the paper's step before it
    accounts for them.  Target: a 10 m segment facing +y; grid: 1024 x 1024
    cells over 1 km; 16 colour levels, each map normalised by its own
    maximum; the near point is 1 m."""
    import torch

    from paper_1310_7297_gb300 import Context
    from paper_1310_7297_gb300 import build as B

    B.build()
    ctx = Context(0)
    t0 = time.perf_counter()
    _, _, c_dense, X, Y = equivisible_dense(ctx)
    torch.cuda.synchronize()
    gpu_ms = 1e3 * (time.perf_counter() - t0)
    rows = [equivisible_row(c_dense, X, Y, mu) for mu in (1, 2, 4, 8, 16)]
    print(json.dumps({"mode": "equivisible", "workload": EQUIVISIBLE_WORKLOAD, "dense_gpu_ms": gpu_ms,
                      "rows": rows}), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: skip the 5,000-box, batched and serving sub-records")
    ap.add_argument("--mode", choices=["step", "step3d", "batched", "serve", "gaze", "equivisible", "modes"],
                    default="step",
                    help="step: the headline line on the 100,000-box scene with the sub-records (default); "
                         "step3d: the 5,000-box 3D step alone; batched / serve: the batching and serving runs "
                         "alone (batched adds the autotuner); gaze: recolouring for new gazes; equivisible: the "
                         "paper's equi-visible cells against the dense map (Eq. 6); modes: strict, field of view, "
                         "two-sided and viewer-centric variants of the 3D step")
    ap.add_argument("--grid", type=int, default=2048,
                    help="viewpoint grid side of the headline workload (2048; smaller only to profile a small case)")
    ap.add_argument("--layers", type=int, default=8, help="viewpoint layers of the headline workload (8)")
    ap.add_argument("--preload-s", type=float, default=0.6,
                    help="seconds the step runs untimed before the timed region (for the clock samples)")
    ap.add_argument("--batch-requests", type=int, default=256)
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--serve-count", type=int, default=400)
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--rates", type=float, nargs="+", default=[50, 100, 200, 500, 1000, 2000])
    ap.add_argument("--slots", type=int, default=2)
    ap.add_argument("--max-batch", type=int, default=8)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "step3d":
        run_step3d(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "serve":
        run_serve(args)
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
