"""The checked build (libvcm_checked.so, kernels compiled with VCM_CHECKED):
its kernels check their indices into spill regions, outputs, lists and
arenas, and a failed check sets the request's vcm_stats.error to
VCM_DEVERR_BOUNDS instead of making the access.  On the small parity cases no
check fires, and the results equal the oracle's as the product library's do.
"""

import numpy as np
import pytest

import synth
from gpu_util import full_parity, gpu_run
from helpers import U, req3, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cctx():
    import __graft_entry__ as g

    g.build()
    from paper_1310_7297_gb300 import Context

    c = Context(0, checked=True)
    yield c
    c.close()


def _load(ctx, sc, cell=0.0):
    ctx.load_scene(sc)
    ctx.vcm_build(cell)


@pytest.mark.parametrize("case", ["2d", "3d", "3d_spill", "fov_two_sided", "viewer", "empty"])
def test_checked_build_matches_the_oracle_with_no_check_firing(cctx, case):
    from paper_1310_7297_gb300 import VCM_TWO_SIDED, VCM_VIEWER

    if case == "2d":
        sc, req = synth.workload_2d(seed=3, grid=64)
    elif case == "empty":
        sc = scene(3, [])
        req = req3((0, 0, 30 * U), pu=8, pw=4, origin=(-50 * U, -50 * U), step=(10 * U, 10 * U), n=(10, 10),
                   layers=(2 * U, 40 * U))
    elif case == "viewer":
        sc, _ = synth.workload_3d(seed=8, grid=32, layers=2, patches=(8, 4), n_boxes=300, half_m=300.0,
                                  n_components=4, sigma_m=(40.0, 100.0))
        req = synth.make_request(3, (12.0, -40.0, 20.0), 0, 2, 2.0, 1, (-300.0, -300.0), (18.75, 18.75), (32, 32),
                                 layers_m=(1.7, 21.7), height_m=1.0, color_levels=16, flags=VCM_VIEWER)
    else:
        sc, req = synth.workload_3d(seed=7, grid=40, layers=3, patches=(32, 16), n_boxes=800, half_m=400.0,
                                    n_components=6, sigma_m=(30.0, 120.0))
        if case == "fov_two_sided":
            req = dict(req, fov_deg=140.0, gaze=[0.3, 1.0, 0.0], flags=VCM_TWO_SIDED)
    _load(cctx, sc)
    if case == "3d_spill":
        cctx.vcm_set_tune(16, 8, 8, 32)   # long candidate lists go through the spill regions
    try:
        gv, gb, st, err, mism = full_parity(cctx, sc, req, bits=True)
        assert st["error"] == 0
    finally:
        cctx.vcm_set_tune(0)


def test_checked_build_batch_scheduler_and_recolor(cctx):
    """The batched launch, a scheduler launch and a recolour in the checked
    build: no check fires and the results equal the direct path's."""
    import torch

    sc, reqs = synth.workload_batched(seed=13, n_requests=6, n_boxes=4000, min_side=3, max_side=6)
    _load(cctx, sc, 50.0)
    alone = [gpu_run(cctx, dict(r, flags=1), bits=True) for r in reqs]
    for a in alone:
        assert a[3]["error"] == 0
    tickets = [cctx.vcm_submit(dict(r, flags=1)) for r in reqs]
    for t, a in zip(tickets, alone):
        assert cctx.vcm_poll(t, -1) == 0
        v, c, b, stt = cctx.vcm_result_get(t)
        assert stt["error"] == 0
        assert np.array_equal(v.astype(np.float64), a[0]) and np.array_equal(b, a[2])
        cctx.vcm_result_release(t)
    r = reqs[0]
    _, _, bits, _ = cctx.compute(r, emit_bits=True)
    v, c, s = cctx.recolor(dict(r, fov_deg=120.0), bits)
    torch.cuda.synchronize()
    from paper_1310_7297_gb300 import stats_from_tensor

    assert stats_from_tensor(s)["error"] == 0
    dv, _, _, _ = gpu_run(cctx, dict(r, fov_deg=120.0), bits=False)
    assert np.allclose(v.cpu().numpy(), dv, rtol=2e-6, atol=0)
