"""vcm_compute_static: one request without any device allocation.

Some callers cannot call cudaMalloc: code running under an allocator that
owns all device memory (a framework's caching pool) or under a fixed memory
budget.  They pass host boxes and their own device output buffers; the
library keeps its grid index, launch descriptors and counters in a
file-scope device array instead of allocating scratch.  These checks call
it through the C ABI twice in a row (the second call on different inputs,
so it must not depend on what the first left in the array) and compare it
with the context-based vcm_compute.  This file is collected last on purpose.
"""

import numpy as np
import pytest

import synth
from paper_1310_7297_gb300.vcm import STATS_BYTES
from gpu_util import compare_bits, compare_colors, compare_v

pytestmark = pytest.mark.gpu


def _outputs(req, bits):
    import torch

    from paper_1310_7297_gb300 import n_viewpoints, words

    dev = torch.device("cuda", 0)
    n = n_viewpoints(req)
    v = torch.empty(n, dtype=torch.float32, device=dev)
    c = torch.empty(n, dtype=torch.uint8, device=dev)
    b = torch.empty(n * words(req), dtype=torch.int32, device=dev) if bits else None
    s = torch.empty(STATS_BYTES, dtype=torch.uint8, device=dev)
    return v, c, b, s


def _host(v, c, b, n):
    return (v.cpu().numpy().astype(np.float64), c.cpu().numpy(),
            b.cpu().numpy().view(np.uint32).reshape(n, -1) if b is not None else None)


def _static(scene, req, bits):
    import torch

    from paper_1310_7297_gb300 import n_viewpoints, stats_from_tensor, vcm

    r = dict(req, flags=vcm.VCM_EMIT_BITS if bits else 0)
    v, c, b, s = _outputs(r, bits)
    vcm.vcm_compute_static(scene.lo_f32(), scene.hi_f32(), scene.dims, r, v.data_ptr(), c.data_ptr(),
                           b.data_ptr() if b is not None else None, s.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return _host(v, c, b, n_viewpoints(r)) + (stats_from_tensor(s),)


def _context(scene, req, bits):
    import torch

    from paper_1310_7297_gb300 import Context, n_viewpoints, stats_from_tensor

    with Context(0) as ctx:
        ctx.load_scene(scene)
        ctx.vcm_build(0.0)
        v, c, b, s = ctx.compute(req, emit_bits=bits)
        torch.cuda.synchronize()
        return _host(v, c, b, n_viewpoints(req)) + (stats_from_tensor(s),)


def _same(got, ref, levels):
    compare_v(ref[0], got[0], "static vs context")
    compare_colors(ref[0], got[0], got[1], levels, got[3]["v_ref"], ref[3]["v_ref"])
    if ref[2] is not None:
        compare_bits(ref[2], got[2], "static vs context")


def test_static_entry_point_matches_context_path_on_two_calls_in_a_row():
    import __graft_entry__ as g

    g.build()
    s3, r3 = synth.workload_3d(seed=31, grid=40, layers=3, patches=(32, 16), n_boxes=300, half_m=400.0,
                               n_components=5, sigma_m=(60.0, 150.0))
    s2, r2 = synth.workload_2d(seed=32, grid=96, samples=64, n_rects=120)
    ref3 = _context(s3, r3, True)
    ref2 = _context(s2, r2, False)
    assert (ref3[0] > 0).sum() > 100 and (ref2[0] > 0).sum() > 100
    first = _static(s3, r3, True)
    second = _static(s2, r2, False)
    _same(first, ref3, r3["color_levels"])
    _same(second, ref2, r2["color_levels"])
    assert first[3]["v_ref"] == pytest.approx(ref3[3]["v_ref"], rel=1e-5)
    # and again, after the other scene has filled the array
    again = _static(s3, r3, True)
    _same(again, ref3, r3["color_levels"])


def test_static_entry_point_rejects_oversized_inputs():
    """Limits are checked on the host before any device work; the output
    buffers are real and sized for each request all the same."""
    import torch

    from paper_1310_7297_gb300 import VcmError, vcm

    stream = torch.cuda.current_stream().cuda_stream
    s, r = synth.workload_3d(seed=33, grid=8, layers=1, n_boxes=4097, half_m=3000.0, n_components=8,
                             sigma_m=(100.0, 400.0))
    v, c, b, st = _outputs(r, False)
    with pytest.raises(VcmError) as e:
        vcm.vcm_compute_static(s.lo_f32(), s.hi_f32(), 3, r, v.data_ptr(), c.data_ptr(), None, st.data_ptr(), stream)
    assert e.value.status == -1 and "4096" in str(e.value)
    s2, r2 = synth.workload_2d(seed=34, grid=16)
    wide = dict(r2, grid_nx=65536, grid_ny=1, grid_step=[1, 1])   # 65,603 coordinates > 65,536
    v, c, b, st = _outputs(wide, False)
    with pytest.raises(VcmError) as e:
        vcm.vcm_compute_static(s2.lo_f32(), s2.hi_f32(), 2, wide, v.data_ptr(), c.data_ptr(), None, st.data_ptr(),
                               stream)
    assert e.value.status == -1 and "65536" in str(e.value)
    torch.cuda.synchronize()


def test_static_entry_point_near_its_box_limit_and_without_colors():
    """4,000 boxes (box_cap 4,000: 144 KB of shared memory per block and most
    of the array in use) agree with the context path; with d_color = NULL
    the values still agree and nothing else is written."""
    import torch

    from paper_1310_7297_gb300 import n_viewpoints, stats_from_tensor, vcm

    s, r = synth.workload_3d(seed=35, grid=48, layers=2, patches=(16, 8), n_boxes=4000, half_m=2500.0,
                             n_components=8, sigma_m=(200.0, 800.0))
    ref = _context(s, r, True)
    got = _static(s, r, True)
    assert (ref[0] > 0).sum() > 100 and ref[2].any()
    _same(got, ref, r["color_levels"])
    # no colors: the values and counters still come out
    n = n_viewpoints(r)
    v, c, b, st = _outputs(r, False)
    c.fill_(77)
    vcm.vcm_compute_static(s.lo_f32(), s.hi_f32(), 3, r, v.data_ptr(), None, None, st.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    compare_v(ref[0], v.cpu().numpy().astype(np.float64), "static, no colors")
    assert (c.cpu().numpy() == 77).all()
    assert stats_from_tensor(st)["v_ref"] == pytest.approx(ref[3]["v_ref"], rel=1e-5)
    assert n == ref[0].shape[0]


def test_static_entry_point_refuses_a_capturing_stream():
    """Its uploads read host memory that is freed when the call returns, so
    on a stream being captured into a CUDA graph it returns VCM_E_ARG
    before enqueuing anything."""
    import torch

    from paper_1310_7297_gb300 import VcmError, vcm

    s, r = synth.workload_2d(seed=36, grid=16)
    v, c, b, st = _outputs(r, False)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        graph.capture_begin()
        try:
            with pytest.raises(VcmError) as e:
                vcm.vcm_compute_static(s.lo_f32(), s.hi_f32(), 2, r, v.data_ptr(), c.data_ptr(), None,
                                       st.data_ptr(), side.cuda_stream)
        finally:
            graph.capture_end()
    assert e.value.status == -1 and "captur" in str(e.value)
    torch.cuda.synchronize()
