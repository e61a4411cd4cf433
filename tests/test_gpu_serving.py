"""Continuous batching through vcm_submit / vcm_poll (GPU).

Requests submitted together are merged by the scheduler into batched
launches on several slots; each result must be the same as the request run
alone (bit for bit: per-viewpoint sums do not depend on batching).  Memory
admission, which counts result buffers and the slots' scratch, holds
requests back until the budget frees up; over-budget requests are refused,
and queued requests can be cancelled.  Failures are made on the host
(vcm_inject): a launch whose spill regions are all held gives up its
bounded device-side wait and reports VCM_E_TIMEOUT; a failed buffer
allocation reports VCM_E_NOMEM; the context keeps working after both.
"""

import numpy as np
import pytest

import synth
from gpu_util import gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene_reqs():
    return synth.workload_batched(seed=13, n_requests=16, n_boxes=4000, min_side=3, max_side=7)


def _ctx(scene, budget=0):
    import __graft_entry__ as g

    g.build()
    from paper_1310_7297_gb300 import Context

    c = Context(0, budget)
    c.load_scene(scene)
    c.vcm_build(50.0)
    return c


def test_mix_equals_alone(scene_reqs):
    scene, reqs = scene_reqs
    ctx = _ctx(scene)
    try:
        alone = [gpu_run(ctx, dict(r, flags=1), bits=True) for r in reqs]
        ctx.vcm_set_slots(3, 5)
        tickets = [ctx.vcm_submit(dict(r, flags=1)) for r in reqs]
        tickets += ctx.vcm_submit_batch([dict(r, flags=1) for r in reqs[:4]])
        for i, t in enumerate(tickets):
            assert ctx.vcm_poll(t, -1) == 0
            v, c, b, st = ctx.vcm_result_get(t)
            ref = alone[i % len(reqs)]
            assert np.array_equal(v.astype(np.float64), ref[0]), i
            assert np.array_equal(c, ref[1]), i
            assert np.array_equal(b, ref[2]), i
            ctx.vcm_result_release(t)
    finally:
        ctx.close()


def _slot_scratch(scene):
    ctx = _ctx(scene)
    try:
        return ctx.vcm_get_memory()["slot_scratch_need"]
    finally:
        ctx.close()


def test_memory_admission_and_rejection(scene_reqs):
    from paper_1310_7297_gb300 import VcmError, n_viewpoints

    scene, reqs = scene_reqs
    biggest = max(n_viewpoints(r) * 5 for r in reqs)
    scratch = _slot_scratch(scene)
    # room for one slot's scratch and about one request at a time
    ctx = _ctx(scene, budget=scratch + biggest + 4096)
    try:
        tickets = [ctx.vcm_submit(r) for r in reqs[:8]]
        for t in tickets:
            assert ctx.vcm_poll(t, -1) == 0
            ctx.vcm_result_release(t)
        r_big = max(reqs, key=n_viewpoints)
        huge = dict(r_big, layer_z=[1741] * 4096)   # 4096 layers: far beyond the budget
        with pytest.raises(VcmError) as e:
            ctx.vcm_submit(huge)
        assert e.value.status == -3   # VCM_E_NOMEM
        m = ctx.vcm_get_memory()
        assert m["results"] == 0 and 0 < m["slot_scratch"] <= m["budget"]
    finally:
        ctx.close()


def test_admission_counts_slot_scratch(scene_reqs):
    """A budget that holds a request's results but not a slot's scratch
    refuses it; one that holds both runs it."""
    from paper_1310_7297_gb300 import VcmError, n_viewpoints

    scene, reqs = scene_reqs
    r = reqs[0]
    need = n_viewpoints(r) * 5 + 1024
    scratch = _slot_scratch(scene)
    assert scratch > 13 << 20   # the work arena alone is 13 MB
    ctx = _ctx(scene, budget=need + scratch - 1)
    try:
        with pytest.raises(VcmError) as e:
            ctx.vcm_submit(r)
        assert e.value.status == -3   # VCM_E_NOMEM
    finally:
        ctx.close()
    ctx = _ctx(scene, budget=need + scratch + 4096)
    try:
        t = ctx.vcm_submit(r)
        assert ctx.vcm_poll(t, -1) == 0
        _, _, _, st = ctx.vcm_result_get(t)
        assert st["group_size"] == 1 and st["device_ms"] > 0 and st["queue_ms"] >= 0
        assert st["latency_ms"] >= st["queue_ms"]
        ctx.vcm_result_release(t)
    finally:
        ctx.close()


def test_bounded_spill_wait_gives_up_with_timeout(scene_reqs):
    """Every spill region held (injected on the host) and 32 staged boxes:
    the blocks of the launch give up their bounded claim after 8 rounds and
    the request reports VCM_E_TIMEOUT; the next launch is complete and equals
    the direct path."""
    from paper_1310_7297_gb300 import VCM_INJECT_SPILL_BUSY, VcmError

    # 800 boxes over 800 m: every tile's candidate list is far longer than 32
    scene, r = synth.workload_3d(seed=7, grid=40, layers=5, patches=(32, 16), n_boxes=800, half_m=400.0,
                                 n_components=6, sigma_m=(30.0, 120.0))
    r = dict(r, flags=1)
    ctx = _ctx(scene)
    try:
        ctx.vcm_set_tune(16, 8, 8, 32)
        alone = gpu_run(ctx, r, bits=True)
        assert alone[3]["boxes_listed"] > 32 * 5 * 3 * 5   # lists average more than 32
        ctx.vcm_inject(VCM_INJECT_SPILL_BUSY, 1)
        t = ctx.vcm_submit(r)
        with pytest.raises(VcmError) as e:
            ctx.vcm_poll(t, -1)
        assert e.value.status == -5   # VCM_E_TIMEOUT
        ctx.vcm_result_release(t)
        t = ctx.vcm_submit(r)
        assert ctx.vcm_poll(t, -1) == 0
        v, c, b, st = ctx.vcm_result_get(t)
        assert st["error"] == 0
        assert np.array_equal(v.astype(np.float64), alone[0]) and np.array_equal(b, alone[2])
        ctx.vcm_result_release(t)
    finally:
        ctx.vcm_set_tune(0)
        ctx.close()


def test_failed_allocation_reports_nomem_and_recovers(scene_reqs):
    from paper_1310_7297_gb300 import VCM_INJECT_ALLOC_FAIL, VCM_INJECT_NONE, VcmError

    scene, reqs = scene_reqs
    ctx = _ctx(scene)
    try:
        ctx.vcm_inject(VCM_INJECT_ALLOC_FAIL, 1)
        t = ctx.vcm_submit(reqs[2])
        with pytest.raises(VcmError) as e:
            ctx.vcm_poll(t, -1)
        assert e.value.status == -3   # VCM_E_NOMEM
        ctx.vcm_result_release(t)
        t = ctx.vcm_submit(reqs[2])
        assert ctx.vcm_poll(t, -1) == 0
        ctx.vcm_result_release(t)
        ctx.vcm_inject(VCM_INJECT_ALLOC_FAIL, 5)
        ctx.vcm_inject(VCM_INJECT_NONE, 0)   # cleared: nothing fails
        t = ctx.vcm_submit(reqs[2])
        assert ctx.vcm_poll(t, -1) == 0
        ctx.vcm_result_release(t)
        with pytest.raises(VcmError):
            ctx.vcm_inject(7, 1)
    finally:
        ctx.close()


def test_cancel_queued_request(scene_reqs):
    from paper_1310_7297_gb300 import VcmError

    scene, reqs = scene_reqs
    ctx = _ctx(scene)
    try:
        ctx.vcm_set_slots(1, 1)
        big = dict(reqs[0], layer_z=[1741 + 10240 * (k % 8) for k in range(64)])
        tickets = [ctx.vcm_submit(big) for _ in range(3)] + [ctx.vcm_submit(reqs[1])]
        ctx.vcm_cancel(tickets[-1])
        with pytest.raises(VcmError) as e:
            ctx.vcm_poll(tickets[-1], 0)
        assert e.value.status == -6   # VCM_E_CANCELLED
        for t in tickets[:-1]:
            assert ctx.vcm_poll(t, -1) == 0
            with pytest.raises(VcmError):
                ctx.vcm_cancel(t)     # already admitted / finished
            ctx.vcm_result_release(t)
        ctx.vcm_result_release(tickets[-1])
    finally:
        ctx.close()


def test_scheduler_spill_path_matches_direct(scene_reqs):
    """Scheduler launches run one block per tile and claim spill regions from a
    per-slot pool; with 32 staged boxes most candidate lists spill."""
    scene, reqs = scene_reqs
    ctx = _ctx(scene)
    try:
        ctx.vcm_set_tune(16, 8, 8, 32)
        alone = [gpu_run(ctx, dict(r, flags=1), bits=True) for r in reqs[:6]]
        for rep in range(2):
            tickets = [ctx.vcm_submit(dict(r, flags=1)) for r in reqs[:6]]
            for i, t in enumerate(tickets):
                assert ctx.vcm_poll(t, -1) == 0
                v, c, b, st = ctx.vcm_result_get(t)
                assert st["error"] == 0 and st["boxes_listed"] > 0
                assert np.array_equal(v.astype(np.float64), alone[i][0])
                assert np.array_equal(b, alone[i][2])
                ctx.vcm_result_release(t)
    finally:
        ctx.vcm_set_tune(0)
        ctx.close()


def test_gaze_change_is_served_from_cached_bits(scene_reqs):
    """Incremental processing in the server (Section IV-C): a request with
    VCM_CACHE_BITS leaves its occlusion bits in the context; later requests
    for the same target and grid with another field of view, gaze, sides,
    strictness or colours are served by recolouring those bits (launch form
    VCM_FORM_RECOLOR, no slab test), and each equals a fresh vcm_compute of
    the same request.  The bits are counted in the memory report, freed by
    vcm_cache_clear, and dropped when the index is rebuilt."""
    from gpu_util import device_edge_cells
    from paper_1310_7297_gb300 import (VCM_CACHE_BITS, VCM_EMIT_BITS, VCM_FORM_RECOLOR, VCM_STRICT, VCM_TWO_SIDED,
                                       n_viewpoints, words)

    scene, reqs = scene_reqs
    ctx = _ctx(scene)
    try:
        r = max(reqs[:8], key=n_viewpoints)
        t = ctx.vcm_submit(dict(r, flags=VCM_CACHE_BITS))
        assert ctx.vcm_poll(t, -1) == 0
        v0, _, _, st0 = ctx.vcm_result_get(t)
        assert st0["launch_form"] != VCM_FORM_RECOLOR and st0["slab_tests"] + st0["corner_tests"] > 0
        ctx.vcm_result_release(t)
        ref0, _, _, _ = gpu_run(ctx, r, bits=False)
        assert np.array_equal(v0.astype(np.float64), ref0)
        m = ctx.vcm_get_memory()
        assert m["cache_entries"] == 1 and m["cached_bits"] == n_viewpoints(r) * words(r) * 4
        cases = [dict(fov_deg=120.0), dict(fov_deg=90.0, gaze=[0.5, 1.0, 0.0]), dict(flags=VCM_TWO_SIDED),
                 dict(flags=VCM_STRICT, fov_deg=150.0), dict(color_levels=5, v_ref=0.3), dict(flags=VCM_EMIT_BITS)]
        for extra in cases:
            q = dict(r, **extra)
            t = ctx.vcm_submit(q)
            assert ctx.vcm_poll(t, -1) == 0
            v, c, b, st = ctx.vcm_result_get(t)
            ctx.vcm_result_release(t)
            assert st["launch_form"] == VCM_FORM_RECOLOR and st["slab_tests"] == 0 and st["error"] == 0, extra
            bits = bool(q.get("flags", 0) & VCM_EMIT_BITS)
            dv, dc, db, dst = gpu_run(ctx, q, bits=bits)
            v = v.astype(np.float64)
            assert np.array_equal(v == 0, dv == 0) and np.allclose(v, dv, rtol=2e-6, atol=0), extra
            L = q["color_levels"]
            edge = device_edge_cells(v, st["v_ref"], L) | device_edge_cells(dv, dst["v_ref"], L)
            assert ((c == dc) | edge).all(), extra
            if bits:
                assert np.array_equal(b, db)
        # another grid is computed, not recoloured
        other = dict(r, grid_nx=r["grid_nx"] - 1)
        t = ctx.vcm_submit(other)
        assert ctx.vcm_poll(t, -1) == 0
        assert ctx.vcm_result_get(t)[3]["launch_form"] != VCM_FORM_RECOLOR
        ctx.vcm_result_release(t)
        ctx.vcm_cache_clear()
        assert ctx.vcm_get_memory()["cache_entries"] == 0
        t = ctx.vcm_submit(dict(r, flags=VCM_CACHE_BITS))
        assert ctx.vcm_poll(t, -1) == 0
        ctx.vcm_result_release(t)
        assert ctx.vcm_get_memory()["cache_entries"] == 1
        ctx.vcm_build(50.0)   # a new index: the cached bits belong to the old one
        m = ctx.vcm_get_memory()
        assert m["cache_entries"] == 0 and m["cached_bits"] == 0
    finally:
        ctx.close()


def test_request_log_and_latency_summary(scene_reqs, tmp_path):
    """Each request whose scheduler launch completes appends one JSON line
    with its timings and device counters, which match what vcm_result_get
    reports; the latency summary covers the completed requests."""
    import json

    scene, reqs = scene_reqs
    ctx = _ctx(scene)
    path = tmp_path / "requests.jsonl"
    try:
        assert ctx.vcm_latency_summary() == (0.0, 0.0, 0)
        ctx.vcm_set_request_log(str(path))
        tickets = [ctx.vcm_submit(r) for r in reqs]
        got = {}
        for t in tickets:
            assert ctx.vcm_poll(t, -1) == 0
            _, _, _, st = ctx.vcm_result_get(t, copy=False)
            got[t] = st
            ctx.vcm_result_release(t)
        ctx.vcm_set_request_log(None)   # closes the file
        lines = [json.loads(x) for x in path.read_text().splitlines()]
        assert sorted(x["ticket"] for x in lines) == sorted(tickets)
        for x in lines:
            st = got[x["ticket"]]
            assert x["status"] == 0
            assert x["segments"] == x["viewpoints"] * x["patches"] == st["segments"]
            for k in ("slab_tests", "corner_tests", "rechecked", "edge_cells", "shortcut_viewpoints",
                      "shared_viewpoints"):
                assert x[k] == st[k], k
            assert abs(x["latency_ms"] - st["latency_ms"]) < 1e-3
            assert abs(x["device_ms"] - st["device_ms"]) < 1e-3
            assert 0.0 <= x["chain_ms"] <= x["device_ms"] + 1e-6
        p50, p99, n = ctx.vcm_latency_summary()
        lat = sorted(got[t]["latency_ms"] for t in tickets)
        assert n == len(tickets)
        assert lat[0] - 1e-6 <= p50 <= p99 <= lat[-1] + 1e-6
    finally:
        ctx.close()

