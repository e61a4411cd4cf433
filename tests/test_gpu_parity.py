"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bits must match exactly, v within 1e-5 relative, colors exactly except for
cells within 2e-5 of a bin edge.  Sizes span many tiles with ragged tails;
the full-size 3D workload is checked on sampled viewpoints.
"""

import numpy as np
import pytest

import synth
from paper_1310_7297_gb300.vcm import STATS_BYTES, stats_from_tensor
from gpu_util import compare_bits, compare_colors, compare_v, device_edge_cells, full_parity, gpu_run
from helpers import U, req2, req3, scene
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g

    g.build()
    from paper_1310_7297_gb300 import Context

    c = Context(0)
    yield c
    c.close()


def load(ctx, sc, cell=0.0):
    ctx.load_scene(sc)
    ctx.vcm_build(cell)


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def test_workload_2d_full(ctx):
    sc, req = synth.workload_2d()
    load(ctx, sc)
    gv, gb, st, err, mism = full_parity(ctx, sc, req)
    assert (gv > 0).sum() > 1000
    assert st["rechecked"] >= 0 and st["slab_tests"] > 0


def test_workload_3d_reduced_full(ctx):
    sc, req = synth.workload_3d(seed=7, grid=40, layers=5, patches=(32, 16), n_boxes=800, half_m=400.0,
                                n_components=6, sigma_m=(30.0, 120.0))
    load(ctx, sc, 40.0)
    gv, gb, st, err, mism = full_parity(ctx, sc, req)
    assert (gv > 0).sum() > 500 and gb.any()


@pytest.mark.parametrize("cell", [3.0, 1000.0])
def test_grid_cell_sizes_walk_every_occluder(ctx, cell):
    """The tile kernel walks only the cell rows under the hull's footprint.
    A 3 m grid gives ~270 rows (several 128-row rounds and long diagonal
    spans); a 1 km grid puts the scene in one or two cells.  Results must not
    depend on it."""
    sc, req = synth.workload_3d(seed=7, grid=40, layers=5, patches=(32, 16), n_boxes=800, half_m=400.0,
                                n_components=6, sigma_m=(30.0, 120.0))
    load(ctx, sc, cell)
    gv, gb, st, err, mism = full_parity(ctx, sc, req)
    assert (gv > 0).sum() > 500 and gb.any()
    sc2, req2 = synth.workload_2d()
    load(ctx, sc2, cell)
    full_parity(ctx, sc2, req2)


def test_dense_cells_overflow_the_walk_list(ctx):
    """4,000 boxes of 1-3 m over 120 m with a 1.5 m grid: nearly every cell
    under a tile's footprint holds boxes, so a walk round lists more cells
    than its list holds and the rest take the per-cell path."""
    from synth import make_request

    rng = np.random.default_rng(61)
    n = 4000
    c = rng.integers(-60 * U, 60 * U, size=(n, 3))
    c[:, 2] = 0
    keep = ~((np.abs(c[:, 0]) < 8 * U) & (np.abs(c[:, 1]) < 4 * U))   # off the target
    c = c[keep]
    size = rng.integers(1 * U, 3 * U, size=c.shape)
    lo = c.copy()
    hi = c + size
    hi[:, 2] = rng.integers(1 * U, 9 * U, size=c.shape[0])
    sc = scene(3, list(zip(lo.tolist(), hi.tolist())))
    req = make_request(3, (0.0, 0.0, 6.0), 0, 2, 8.0, 8, (-60.0, -60.0), (5.0, 5.0), (24, 24),
                       layers_m=(1.0, 12.0), axis_w=4, height_m=4.0, patches_w=4, color_levels=8)
    load(ctx, sc, 1.5)
    gv, gb, st, err, mism = full_parity(ctx, sc, req)
    assert (gv > 0).sum() > 20 and gb.any()


def test_workload_3d_full_size_sampled(ctx):
    """512 x 512 x 5 viewpoints, 5,000 boxes, 32 x 16 patches, in the launch
    configuration the benchmark times; the oracle checks 1,200 viewpoints."""
    sc, req = synth.workload_3d()
    load(ctx, sc)
    gv, gc, gb, st = gpu_run(ctx, req, bits=True)
    n = gv.shape[0]
    # every viewpoint written (outputs start as NaN / colour 255), some of
    # them by the chunk pass that the tiles with many open viewpoints feed
    assert np.isfinite(gv).all() and (gc != 255).all()
    assert st["shared_viewpoints"] > 1000
    rng = np.random.default_rng(11)
    nz = np.nonzero(gv > 0)[0]
    idx = np.unique(np.concatenate([rng.choice(n, 600, replace=False), rng.choice(nz, 600, replace=False)]))
    ov, ob = O.run(sc, req, indices=idx, bits=True)
    compare_bits(ob, gb[idx], "full-size sample")
    compare_v(ov, gv[idx], "full-size sample")
    # colors follow the device's own v and v_ref = max v: on the sample they
    # equal the oracle's quantisation of its v by that v_ref, except at
    # counted bin-edge cells, and the count over the whole grid is exact
    L = req["color_levels"]
    assert st["v_ref"] == pytest.approx(float(gv.max()), rel=0, abs=0)
    compare_colors(ov, gv[idx], gc[idx], L, st["v_ref"], st["v_ref"])
    assert st["edge_cells"] == device_edge_cells(gv, st["v_ref"], L).sum()
    assert (gc[gv == 0] == 0).all() and (gc[gv > 0] >= 1).all() and gc.max() == L - 1
    assert st["slab_tests"] > 0


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_empty_scene(ctx):
    sc = scene(3, [])
    r = req3((0, 0, 30 * U), pu=8, pw=4, origin=(-50 * U, -50 * U), step=(10 * U, 10 * U), n=(10, 10),
             layers=(2 * U, 40 * U))
    load(ctx, sc)
    gv, gb, st, err, mism = full_parity(ctx, sc, r)
    assert not gb.any() and (gv > 0).any()


def test_full_wall_and_inside_box(ctx):
    sc = scene(3, [((-2000 * U, 2 * U, -10 * U), (2000 * U, 3 * U, 2000 * U)),
                   ((-40 * U, -40 * U, 0), (-30 * U, -30 * U, 10 * U))])
    r = req3((0, 0, 30 * U), pu=8, pw=4, origin=(-64 * U, -60 * U), step=(16 * U, 16 * U), n=(8, 8),
             layers=(2 * U, 30 * U, 70 * U))
    load(ctx, sc)
    gv, gb, st, err, mism = full_parity(ctx, sc, r)
    assert (gv == 0).all()


@pytest.mark.parametrize("patches", [(1, 1), (7, 3), (8, 4), (16, 8), (40, 5), (48, 20), (64, 32), (33, 1)])
def test_patch_shapes_and_ragged_tiles(ctx, patches):
    sc, _ = synth.workload_3d(seed=3, grid=8, layers=1, n_boxes=400, half_m=250.0, n_components=4,
                              sigma_m=(20.0, 80.0))
    r = req3((0, 0, 30 * U), width=20 * U, height=10 * U, pu=patches[0], pw=patches[1],
             origin=(-240 * U, -240 * U), step=(37 * U, 23 * U), n=(13, 21), layers=(1741, 31 * U, 45 * U))
    load(ctx, sc, 30.0)
    full_parity(ctx, sc, r)


@pytest.mark.parametrize("axes", [(2, 4, 0), (3, 5, 1), (0, 4, 3), (1, 2, 4), (0, 3, 5)])
def test_target_orientations(ctx, axes):
    """u, w and the normal along every axis, both signs (incl. a horizontal
    target facing up or down, seen from layers on both sides)."""
    rng = np.random.default_rng(sum(axes))
    lo = rng.integers(-150 * U, 130 * U, size=(120, 3))
    lo[:, 2] = rng.integers(0, 20 * U, size=120)
    hi = lo + rng.integers(3 * U, 25 * U, size=(120, 3))
    c = np.array([0, 0, 30 * U])
    keep = ~np.all((lo <= c + 12 * U) & (c - 12 * U <= hi), axis=1)
    sc = scene(3, list(zip(lo[keep].tolist(), hi[keep].tolist())))
    r = req3((0, 0, 30 * U), axis_u=axes[0], axis_w=axes[1], normal=axes[2], width=12 * U, height=6 * U,
             pu=12, pw=6, origin=(-160 * U, -160 * U), step=(20 * U, 20 * U), n=(16, 16),
             layers=(2 * U, 30 * U, 60 * U))
    load(ctx, sc, 25.0)
    full_parity(ctx, sc, r)


def test_2d_orientations_and_long_segment(ctx):
    rng = np.random.default_rng(4)
    lo = rng.integers(-300 * U, 280 * U, size=(80, 3))
    lo[:, 2] = 0
    hi = lo + rng.integers(2 * U, 20 * U, size=(80, 3))
    hi[:, 2] = 0
    keep = ~np.all((lo[:, :2] <= 30 * U) & (-30 * U <= hi[:, :2]), axis=1)
    sc = scene(2, list(zip(lo[keep].tolist(), hi[keep].tolist())))
    load(ctx, sc, 20.0)
    for (au, nr, pu) in [(0, 2, 100), (2, 1, 37), (3, 0, 64), (1, 3, 5)]:
        r = req2((0, 0), axis_u=au, normal=nr, width=40 * U, pu=pu, origin=(-300 * U, -300 * U),
                 step=(15 * U, 12 * U), n=(40, 50))
        full_parity(ctx, sc, r)


def test_viewpoints_on_target_plane_and_exact_coincidences(ctx):
    """Viewpoint rows exactly on the target plane (d_n = 0) and viewpoint
    columns equal to patch columns (d_u = 0), with box faces on the same
    lattice lines: the zero-direction and touching cases of the slab test."""
    boxes = []
    for i in range(-6, 7):
        for j in (-3, 2, 5):
            boxes.append(((i * 8 * U, j * 8 * U, 0), (i * 8 * U + 4 * U, j * 8 * U + 4 * U, (i % 4 + 1) * 8 * U)))
    sc = scene(3, boxes)
    # patch columns at x = -15..15 step 2 (odd metres), rows at z = 21..39
    r = req3((0, 0, 30 * U), width=32 * U, height=20 * U, pu=16, pw=10, origin=(-64 * U, -40 * U),
             step=(2 * U, 4 * U), n=(64, 20), layers=(21 * U, 30 * U, 8 * U))
    load(ctx, sc, 16.0)
    gv, gb, st, err, mism = full_parity(ctx, sc, r)
    assert st["rechecked"] > 0   # exact touches land in the band


def test_tie_heavy_integer_scene(ctx):
    """Everything on whole metres: many segments pass exactly through box
    edges and corners, so the float64 re-decision carries the result."""
    rng = np.random.default_rng(9)
    lo = rng.integers(-40, 36, size=(150, 3)) * U
    lo[:, 2] = rng.integers(0, 10, size=150) * U
    hi = lo + rng.integers(1, 6, size=(150, 3)) * U
    keep = ~np.all((lo <= np.array([9, 1, 27]) * U) & (np.array([-9, -1, 13]) * U <= hi), axis=1)
    sc = scene(3, list(zip(lo[keep].tolist(), hi[keep].tolist())))
    r = req3((0, 0, 20 * U), width=16 * U, height=12 * U, pu=8, pw=6, origin=(-40 * U, -40 * U),
             step=(2 * U, 2 * U), n=(40, 40), layers=(0, 5 * U, 20 * U))
    load(ctx, sc, 8.0)
    gv, gb, st, err, mism = full_parity(ctx, sc, r)
    assert st["rechecked"] > 0


def test_large_coordinates_and_thin_boxes(ctx):
    base = 16000 * U
    rng = np.random.default_rng(2)
    lo = rng.integers(base - 300 * U, base - 40 * U, size=(60, 3))
    lo[:, 2] = 0
    ext = rng.integers(0, 15 * U, size=(60, 3))
    ext[::3, 0] = 0   # zero-thickness walls
    hi = np.minimum(lo + ext, 16384 * U)
    sc = scene(3, list(zip(lo.tolist(), hi.tolist())))
    r = req3((base, base, 20 * U), normal=3, width=10 * U, height=6 * U, pu=10, pw=6,
             origin=(base - 320 * U, base - 320 * U), step=(20 * U, 20 * U), n=(16, 16), layers=(1 * U, 18 * U))
    load(ctx, sc, 30.0)
    full_parity(ctx, sc, r)


def test_given_v_ref_and_levels(ctx):
    sc, req = synth.workload_2d(seed=5, grid=48, samples=32, n_rects=60)
    load(ctx, sc)
    for levels, vref in [(2, 0.0), (256, 0.0), (16, 0.05), (8, 100.0)]:
        r = dict(req, color_levels=levels, v_ref=vref)
        gv, gc, gb, st = gpu_run(ctx, r, bits=False)
        ov = O.run(sc, r)
        compare_v(ov, gv)
        compare_colors(ov, gv, gc, levels, st["v_ref"], vref if vref > 0 else None)
        assert st["edge_cells"] == device_edge_cells(gv, st["v_ref"], levels).sum()
        if vref > 0:
            assert st["v_ref"] == pytest.approx(vref, rel=1e-7)


def test_bin_edge_cells_are_counted_exactly(ctx):
    """Colors are exact except at bin-edge cells, which the device counts
    (Def. 1 normalisation into L levels).  With a v_ref chosen so that a
    known cell lands on a bin edge (256 levels), the device's count equals
    the count recomputed from its own float32 v and v_ref, the chosen cell
    is among them, and every color that differs from the oracle's is at a
    counted cell."""
    sc, req = synth.workload_3d(seed=9, grid=64, layers=3, patches=(16, 8), n_boxes=400, half_m=400.0,
                                n_components=5, sigma_m=(40.0, 150.0))
    load(ctx, sc)
    gv, _, _, _ = gpu_run(ctx, req, bits=False)
    nz = np.nonzero(gv > 0)[0]
    assert nz.size > 500
    ov = O.run(sc, req)
    L = 256
    rng = np.random.default_rng(17)
    for k in rng.choice(nz, 4, replace=False):
        m = int(rng.integers(2, L - 2))
        # x_k = (L - 1) v_k / v_ref lands on the edge m, up to float32 rounding
        vref = float(np.float32((L - 1) * np.float32(gv[k]) / m))
        r = dict(req, color_levels=L, v_ref=vref)
        gv2, gc2, _, st = gpu_run(ctx, r, bits=False)
        assert np.array_equal(gv2, gv)   # the values do not depend on v_ref
        edge = device_edge_cells(gv2, st["v_ref"], L)
        assert st["v_ref"] == np.float32(vref)
        assert edge[k], "the constructed cell is not an edge cell"
        assert st["edge_cells"] == int(edge.sum()) >= 1
        mism, n_edge = compare_colors(ov, gv2, gc2, L, st["v_ref"], st["v_ref"])
        assert n_edge == st["edge_cells"]


# ---------------------------------------------------------------------------
# launch shapes, spill, batching, scheduling: identical results
# ---------------------------------------------------------------------------

def _bits_and_v(ctx, req):
    gv, gc, gb, st = gpu_run(ctx, req, bits=True)
    return gv, gc, gb


def test_launch_shapes_and_spill_give_identical_results(ctx):
    sc, req = synth.workload_3d(seed=12, grid=48, layers=2, patches=(16, 8), n_boxes=1500, half_m=300.0,
                                n_components=5, sigma_m=(30.0, 100.0))
    load(ctx, sc, 30.0)
    ref = _bits_and_v(ctx, req)
    try:
        for shape in [(1, 1, 0, 1024), (3, 5, 2, 64), (16, 16, 16, 2048), (8, 8, 1, 32), (4, 4, 4, 48)]:
            ctx.vcm_set_tune(*shape)
            got = _bits_and_v(ctx, req)
            assert np.array_equal(got[0], ref[0]), shape     # bit-identical v
            assert np.array_equal(got[1], ref[1]), shape
            assert np.array_equal(got[2], ref[2]), shape
    finally:
        ctx.vcm_set_tune(0)
    ov, ob = O.run(sc, req, bits=True)
    compare_bits(ob, ref[2])
    compare_v(ov, ref[0])


def test_batch_equals_single_requests(ctx):
    import torch

    from paper_1310_7297_gb300 import n_viewpoints, words

    sc, reqs = synth.workload_batched(seed=8, n_requests=6, n_boxes=3000, min_side=3, max_side=6)
    load(ctx, sc, 50.0)
    singles = [_bits_and_v(ctx, dict(r, flags=1)) for r in reqs]
    dev = torch.device("cuda", 0)
    vs = [torch.full((n_viewpoints(r),), float("nan"), device=dev) for r in reqs]
    cs = [torch.full((n_viewpoints(r),), 255, dtype=torch.uint8, device=dev) for r in reqs]
    bs = [torch.empty(n_viewpoints(r) * words(r), dtype=torch.int32, device=dev) for r in reqs]
    st = torch.empty(STATS_BYTES * len(reqs), dtype=torch.uint8, device=dev)
    ctx.vcm_compute_batch([dict(r, flags=1) for r in reqs], [t.data_ptr() for t in vs], [t.data_ptr() for t in cs],
                          [t.data_ptr() for t in bs], st.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for i, r in enumerate(reqs):
        assert np.array_equal(vs[i].cpu().numpy().astype(np.float64), singles[i][0])
        assert np.array_equal(cs[i].cpu().numpy(), singles[i][1])
        assert np.array_equal(bs[i].cpu().numpy().view(np.uint32).reshape(n_viewpoints(r), -1), singles[i][2])
    # and one of them against the oracle on a sample
    r = reqs[0]
    idx = np.arange(0, n_viewpoints(r), 7)
    ov, ob = O.run(sc, r, indices=idx, bits=True)
    compare_bits(ob, singles[0][2][idx])
    compare_v(ov, singles[0][0][idx])


def test_submit_poll_matches_direct(ctx):
    sc, reqs = synth.workload_batched(seed=9, n_requests=5, n_boxes=2000, min_side=3, max_side=6)
    load(ctx, sc, 50.0)
    tickets = [ctx.vcm_submit(dict(r, flags=1)) for r in reqs]
    for t, r in zip(tickets, reqs):
        assert ctx.vcm_poll(t, -1) == 0
        v, c, b, st = ctx.vcm_result_get(t)
        ref = _bits_and_v(ctx, dict(r, flags=1))
        assert np.array_equal(v.astype(np.float64), ref[0]) and np.array_equal(c, ref[1])
        assert np.array_equal(b, ref[2])
        assert st["latency_ms"] > 0 and st["segments"] == len(v) * r["patches_u"] * r["patches_w"]
        # zero-copy device views of the same result
        dv, dc, db, dst = ctx.vcm_result_device(t)
        assert dv.is_cuda and dv.dtype.is_floating_point and dc.shape == c.shape
        assert np.array_equal(dv.cpu().numpy(), v) and np.array_equal(dc.cpu().numpy(), c)
        assert np.array_equal(db.cpu().numpy().view(np.uint32), b)
        assert dst["segments"] == st["segments"]
        ctx.vcm_result_release(t)


def test_deterministic_repeat(ctx):
    sc, req = synth.workload_2d(seed=3)
    load(ctx, sc)
    a = _bits_and_v(ctx, req)
    b = _bits_and_v(ctx, req)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


# ---------------------------------------------------------------------------
# argument checking through the C ABI
# ---------------------------------------------------------------------------

def test_argument_errors(ctx):
    from paper_1310_7297_gb300 import VcmError

    sc, req = synth.workload_2d(seed=2, grid=16)
    load(ctx, sc)
    ctx.compute(dict(req, center=[1, 0, 0]))     # one lattice unit off centre is fine
    for r, st in [(dict(req, dims=4), -1), (dict(req, normal=0), -1), (dict(req, color_levels=1), -1),
                  (dict(req, grid_step=[0, 8000]), -1), (dict(req, patches_u=0), -1),
                  (dict(req, flags=32), -1), (dict(req, flags=16 | 4), -1)]:
        with pytest.raises(VcmError) as e:
            ctx.compute(r)
        assert e.value.status == st
    with pytest.raises(VcmError) as e:
        ctx.vcm_scene_load_mem(np.array([[0.1, 0.0]], np.float32), np.array([[1.0, 1.0]], np.float32), 2)
    assert e.value.status == -1     # 0.1 m is not on the 2^-10 m lattice
    with pytest.raises(VcmError) as e:
        ctx.vcm_scene_load_mem(np.array([[np.nan, 0.0]], np.float32), np.array([[1.0, 1.0]], np.float32), 2)
    assert e.value.status == -1
    with pytest.raises(VcmError) as e:
        ctx.vcm_scene_load_mem(np.array([[2.0, 0.0]], np.float32), np.array([[1.0, 1.0]], np.float32), 2)
    assert e.value.status == -1     # lo > hi
    # a new scene must be built before use
    ctx.vcm_scene_load_mem(np.array([[2.0, 2.0]], np.float32), np.array([[3.0, 3.0]], np.float32), 2)
    with pytest.raises(VcmError) as e:
        ctx.compute(req)
    assert e.value.status == -7
    with pytest.raises(VcmError) as e:
        ctx.vcm_submit(req)
    assert e.value.status == -7


# ---------------------------------------------------------------------------
# full-size parity for the large and batched workloads (sampled viewpoints)
# ---------------------------------------------------------------------------

def _sampled_bits(ctx, req, idx):
    """Run a request with bits on the device (values prefilled with NaN) and
    bring back only the sampled rows."""
    import torch

    from paper_1310_7297_gb300 import VCM_EMIT_BITS, n_viewpoints, words

    n = n_viewpoints(req)
    req = dict(req, flags=req.get("flags", 0) | VCM_EMIT_BITS)
    v = torch.full((n,), float("nan"), device="cuda")
    c = torch.empty(n, dtype=torch.uint8, device="cuda")
    b = torch.empty(n * words(req), dtype=torch.int32, device="cuda")
    s = torch.empty(STATS_BYTES, dtype=torch.uint8, device="cuda")
    ctx.vcm_compute(req, v.data_ptr(), c.data_ptr(), b.data_ptr(), s.data_ptr(),
                    torch.cuda.current_stream().cuda_stream)
    t = torch.as_tensor(idx, device=v.device)
    bv = v.index_select(0, t).cpu().numpy().astype(np.float64)
    bb = b.view(n, -1).index_select(0, t).cpu().numpy().view(np.uint32)
    bc = c.index_select(0, t).cpu().numpy()
    full_v = v.cpu().numpy().astype(np.float64)
    del b
    torch.cuda.synchronize()
    return bv, bb, bc, full_v, stats_from_tensor(s)


def test_workload_3d_large_full_size_sampled(ctx):
    """100,000 boxes over 10 km, 2048 x 2048 x 8 viewpoints, 64 x 32 patches,
    50 m grid index: bits and v on 400 sampled viewpoints (half of them with
    something visible)."""
    sc, req = synth.workload_3d_large()
    load(ctx, sc, 50.0)
    n = 2048 * 2048 * 8
    rng = np.random.default_rng(21)
    idx0 = np.sort(rng.choice(n, 200, replace=False))
    gv0, gb0, _, v_all, st = _sampled_bits(ctx, req, idx0)
    assert np.isfinite(v_all).all()   # every viewpoint written
    assert st["shared_viewpoints"] > 1000   # the chunk pass ran
    nz = np.nonzero(v_all > 0)[0]
    idx1 = np.sort(rng.choice(nz, min(200, nz.size), replace=False))
    idx = np.unique(np.concatenate([idx0, idx1]))
    gv, gb, gc, v_all, st = _sampled_bits(ctx, req, idx)
    ov, ob = O.run(sc, req, indices=idx, bits=True)
    compare_bits(ob, gb, "large scene sample")
    compare_v(ov, gv, "large scene sample")
    L = req["color_levels"]
    compare_colors(ov, gv, gc, L, st["v_ref"], st["v_ref"])
    assert st["edge_cells"] == device_edge_cells(v_all, st["v_ref"], L).sum()
    assert nz.size > 1000


def test_workload_batched_full_mix_sampled(ctx):
    """The 256-request mix over the shared 50,000-box scene in one persistent
    launch; 8 requests checked against the oracle on sampled viewpoints."""
    import torch

    from paper_1310_7297_gb300 import n_viewpoints, words

    sc, reqs = synth.workload_batched()
    load(ctx, sc, 50.0)
    dev = torch.device("cuda", 0)
    vs = [torch.full((n_viewpoints(r),), float("nan"), device=dev) for r in reqs]
    cs = [torch.full((n_viewpoints(r),), 255, dtype=torch.uint8, device=dev) for r in reqs]
    bs = [torch.empty(n_viewpoints(r) * words(r), dtype=torch.int32, device=dev) for r in reqs]
    st = torch.empty(STATS_BYTES * len(reqs), dtype=torch.uint8, device=dev)
    ctx.vcm_compute_batch([dict(r, flags=1) for r in reqs], [t.data_ptr() for t in vs], [t.data_ptr() for t in cs],
                          [t.data_ptr() for t in bs], st.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    # every viewpoint of every request written
    assert all(bool(torch.isfinite(t).all()) for t in vs) and all(bool((t != 255).all()) for t in cs)
    rng = np.random.default_rng(5)
    for k in rng.choice(len(reqs), 8, replace=False):
        r = reqs[k]
        n = n_viewpoints(r)
        gv = vs[k].cpu().numpy().astype(np.float64)
        nz = np.nonzero(gv > 0)[0]
        idx = np.sort(rng.choice(n, min(n, 60), replace=False))
        if nz.size:
            idx = np.unique(np.concatenate([idx, rng.choice(nz, min(nz.size, 60), replace=False)]))
        gb = bs[k].view(n, -1)[torch.as_tensor(idx, device=dev)].cpu().numpy().view(np.uint32)
        ov, ob = O.run(sc, r, indices=idx, bits=True)
        compare_bits(ob, gb, "batched request %d" % k)
        compare_v(ov, gv[idx], "batched request %d" % k)
        stk = stats_from_tensor(st[k * STATS_BYTES:(k + 1) * STATS_BYTES])
        gc = cs[k].cpu().numpy()
        compare_colors(ov, gv[idx], gc[idx], r["color_levels"], stk["v_ref"], stk["v_ref"])
        assert stk["edge_cells"] == device_edge_cells(gv, stk["v_ref"], r["color_levels"]).sum()


# ---------------------------------------------------------------------------
# strict (completely visible) and viewer-centric modes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["2d", "3d"])
def test_strict_mode(ctx, which):
    from paper_1310_7297_gb300 import VCM_STRICT

    if which == "2d":
        sc, req = synth.workload_2d(seed=6)
    else:
        sc, req = synth.workload_3d(seed=43, grid=40, layers=3, patches=(16, 8), n_boxes=300, half_m=400.0,
                                    n_components=5, sigma_m=(60.0, 150.0))
    load(ctx, sc)
    r = dict(req, flags=VCM_STRICT)
    gv, gb, st, err, mism = full_parity(ctx, sc, r)
    vp = O.run(sc, req)
    assert (gv > 0).sum() > 20 and ((vp > 0) & (gv == 0)).sum() > 20   # some partly visible cells drop out
    # without bits (the any-blocked early exit) the values are the same
    gv2, _, _, _ = gpu_run(ctx, r, bits=False)
    assert np.array_equal(gv2, gv)


@pytest.mark.parametrize("which", ["2d", "3d", "3d_inside"])
def test_viewer_mode(ctx, which):
    from paper_1310_7297_gb300 import VCM_VIEWER
    from synth import make_request

    if which == "2d":
        sc, _ = synth.workload_2d(seed=7)
        r = make_request(2, (37.0, -12.5), 0, 2, 2.0, 1, (-500.0, -500.0), (1000 / 96, 1000 / 96), (96, 96),
                         color_levels=8, flags=VCM_VIEWER)
    else:
        sc, _ = synth.workload_3d(seed=44, grid=8, n_boxes=600, half_m=400.0, n_components=5,
                                  sigma_m=(60.0, 150.0))
        viewer = (12.0, -30.0, 25.0)
        if which == "3d_inside":   # a viewer inside a box sees nothing
            b = sc.lo[0] + (sc.hi[0] - sc.lo[0]) // 2
            viewer = tuple(float(x) / 1024 for x in b)
        r = make_request(3, viewer, 0, 2, 1.0, 1, (-400.0, -400.0), (800 / 64, 800 / 64), (64, 64),
                         layers_m=(1.7, 21.7, 61.7), axis_w=4, height_m=1.0, color_levels=16, flags=VCM_VIEWER)
    load(ctx, sc)
    gv, gb, st, err, mism = full_parity(ctx, sc, r)
    if which == "3d_inside":
        assert (gv == 0).all() and gb.all()
    else:
        assert (gv > 0).sum() > 200 and gb.any()


# ---------------------------------------------------------------------------
# tuning, scene files and profiling hooks through the C ABI
# ---------------------------------------------------------------------------

def test_autotune_keeps_results(ctx):
    sc, reqs = synth.workload_batched(seed=15, n_requests=4, n_boxes=3000, min_side=3, max_side=5)
    load(ctx, sc, 50.0)
    before = [_bits_and_v(ctx, dict(r, flags=1)) for r in reqs]
    shapes = ctx.vcm_autotune(reqs)
    assert len(shapes) == len(reqs) and all(s[0] >= 1 and s[3] >= 32 for s in shapes)
    # a request launched alone takes its class's shape, its tiles shrunk
    # while the launch has few of them
    got = ctx.vcm_get_tune(reqs[0])
    assert got[3] == shapes[0][3] and got[0] <= shapes[0][0] and got[1] <= shapes[0][1]
    after = [_bits_and_v(ctx, dict(r, flags=1)) for r in reqs]
    for a, b in zip(before, after):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_scene_file_round_trip_and_bad_files(ctx, tmp_path):
    from paper_1310_7297_gb300 import VcmError

    sc, req = synth.workload_2d(seed=16)
    load(ctx, sc)
    ref = _bits_and_v(ctx, req)
    path = str(tmp_path / "scene.vcms")
    ctx.vcm_scene_save(path)
    ctx.vcm_scene_load(path)
    ctx.vcm_build(0.0)
    got = _bits_and_v(ctx, req)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    raw = open(path, "rb").read()
    for bad in (b"", b"VCMX" + raw[4:], raw[:-3], raw + b"\0"):
        p = tmp_path / "bad.vcms"
        p.write_bytes(bad)
        with pytest.raises(VcmError) as e:
            ctx.vcm_scene_load(str(p))
        assert e.value.status == -2    # VCM_E_IO
    with pytest.raises(VcmError) as e:
        ctx.vcm_scene_load(str(tmp_path / "missing.vcms"))
    assert e.value.status == -2


def test_timing_events_bracket_the_tile_kernel(ctx):
    import torch

    sc, req = synth.workload_2d(seed=17)
    load(ctx, sc)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    b.record()
    ctx.vcm_set_timing_events(a, b)
    try:
        ctx.compute(req)
        torch.cuda.synchronize()
        assert a.elapsed_time(b) > 0.0
    finally:
        ctx.vcm_set_timing_events(None, None)


# ---------------------------------------------------------------------------
# two-sided targets and the field-of-view cone
# ---------------------------------------------------------------------------

def _reduced(which, seed):
    if which == "2d":
        return synth.workload_2d(seed=seed)
    return synth.workload_3d(seed=seed, grid=40, layers=3, patches=(16, 8), n_boxes=300, half_m=400.0,
                             n_components=5, sigma_m=(60.0, 150.0))


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_two_sided(ctx, which):
    """Both faces count: viewpoints behind the target get values too, and
    those in front keep their one-sided values."""
    from paper_1310_7297_gb300 import VCM_STRICT, VCM_TWO_SIDED

    sc, req = _reduced(which, 51)
    load(ctx, sc)
    r = dict(req, flags=VCM_TWO_SIDED)
    gv, gb, st, err, mism = full_parity(ctx, sc, r)
    one, _, _, _ = gpu_run(ctx, req, bits=False)
    behind = (one == 0) & (gv > 0)
    assert behind.sum() > 50
    front = one > 0
    assert np.allclose(gv[front], one[front], rtol=1e-6, atol=0)
    full_parity(ctx, sc, dict(req, flags=VCM_TWO_SIDED | VCM_STRICT))


@pytest.mark.parametrize("which", ["2d", "3d"])
@pytest.mark.parametrize("case", ["fov120", "fov100_gaze", "two_sided_fov150", "strict_fov130", "fov300"])
def test_field_of_view(ctx, which, case):
    """A cone around the gaze axis masks patches.  The oracle decides it in
    float64; viewpoints with a patch at the cone's edge (within the float32
    error band) may take either decision for it, all others match."""
    from paper_1310_7297_gb300 import VCM_STRICT, VCM_TWO_SIDED

    sc, req = _reduced(which, 52)
    load(ctx, sc)
    r = dict(req)
    if case == "fov120":
        r.update(fov_deg=120.0)
    elif case == "fov100_gaze":
        r.update(fov_deg=100.0, gaze=[-0.6, 1.0, -0.1])
    elif case == "two_sided_fov150":
        r.update(fov_deg=150.0, gaze=[-0.2, 1.0, 0.1], flags=VCM_TWO_SIDED)
    elif case == "strict_fov130":
        r.update(fov_deg=130.0, flags=VCM_STRICT)
    else:
        r.update(fov_deg=300.0, gaze=[0.0, -1.0, 0.0], flags=VCM_TWO_SIDED)
    gv, gb, st, err, mism = full_parity(ctx, sc, r)
    full = O.run(sc, dict(req, flags=r.get("flags", 0)))
    assert (gv > 0).sum() > 20
    if case != "fov300":
        assert (gv < full * (1 - 1e-6)).sum() > 20   # the cone takes some patches away


def test_two_sided_and_fov_argument_errors(ctx):
    from paper_1310_7297_gb300 import VCM_TWO_SIDED, VCM_VIEWER, VcmError
    from synth import make_request

    sc, req = _reduced("2d", 53)
    load(ctx, sc)
    bad = [dict(req, fov_deg=-1.0), dict(req, fov_deg=float("nan")), dict(req, fov_deg=90.0, gaze=[float("inf"), 0, 0])]
    viewer = make_request(2, (37.0, -12.5), 0, 2, 2.0, 1, (-500.0, -500.0), (10.0, 10.0), (8, 8),
                          color_levels=8, flags=VCM_VIEWER)
    bad += [dict(viewer, flags=VCM_VIEWER | VCM_TWO_SIDED), dict(viewer, fov_deg=100.0)]
    for r in bad:
        with pytest.raises(VcmError) as e:
            gpu_run(ctx, r, bits=False)
        assert "VCM_E_ARG" in str(e.value)


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_recolor_from_bits_for_new_gazes(ctx, which):
    """One computation with bits, then new fields of view, gazes, sides and
    strictness from those bits alone: each equals the oracle for that
    request and the direct computation of it."""
    import torch

    from paper_1310_7297_gb300 import VCM_STRICT, VCM_TWO_SIDED

    sc, req = _reduced(which, 54)
    load(ctx, sc)
    _, _, bits, _ = ctx.compute(req, emit_bits=True)
    cases = [dict(), dict(fov_deg=120.0), dict(fov_deg=100.0, gaze=[-0.6, 1.0, -0.1]),
             dict(fov_deg=150.0, gaze=[-0.2, 1.0, 0.1], flags=VCM_TWO_SIDED), dict(fov_deg=90.0, flags=VCM_STRICT),
             dict(flags=VCM_TWO_SIDED | VCM_STRICT), dict(fov_deg=200.0, color_levels=5, v_ref=0.5)]
    for extra in cases:
        r = dict(req, **extra)
        v, c, s = ctx.recolor(r, bits)
        torch.cuda.synchronize()
        gv = v.cpu().numpy().astype(np.float64)
        ov, band = O.run(sc, r, band=True)
        compare_v(ov, gv, str(extra), band)
        st = stats_from_tensor(s)
        compare_colors(ov, gv, c.cpu().numpy(), r["color_levels"], st["v_ref"], r.get("v_ref", 0.0) or None,
                       flex=band[:, 0] > 0)
        dv, _, _, _ = gpu_run(ctx, r, bits=False)
        assert np.allclose(gv, dv, rtol=2e-6, atol=0), extra
        assert (gv > 0).sum() > 20


def test_recolor_argument_errors(ctx):
    from paper_1310_7297_gb300 import VCM_VIEWER, VcmError
    from synth import make_request

    sc, req = _reduced("2d", 55)
    load(ctx, sc)
    _, _, bits, _ = ctx.compute(req, emit_bits=True)
    viewer = make_request(2, (37.0, -12.5), 0, 2, 2.0, 1, (-500.0, -500.0), (10.0, 10.0), (8, 8),
                          color_levels=8, flags=VCM_VIEWER)
    with pytest.raises(VcmError, match="VCM_E_ARG"):
        ctx.recolor(viewer, bits)
    with pytest.raises(VcmError, match="VCM_E_ARG"):
        ctx.vcm_recolor(req, None, 1, None, 1, None)
    with pytest.raises(VcmError, match="VCM_E_ARG"):
        ctx.recolor(dict(req, fov_deg=-5.0), bits)


@pytest.mark.parametrize("case", ["two_sided", "fov_strict", "plain_bits"])
def test_many_patch_requests_take_the_whole_tile_check(ctx, case):
    """Requests of >= 512 patches run the tile kernel's instantiation with
    the whole-tile check (and, when two-sided or coned, the one with both);
    values, bits and colors still match the oracle."""
    from paper_1310_7297_gb300 import VCM_STRICT, VCM_TWO_SIDED

    sc, req = synth.workload_3d(seed=71, grid=24, layers=2, patches=(64, 32), n_boxes=250, half_m=300.0,
                                n_components=4, sigma_m=(40.0, 100.0))
    load(ctx, sc)
    r = dict(req)
    if case == "two_sided":
        r.update(flags=VCM_TWO_SIDED)
    elif case == "fov_strict":
        r.update(flags=VCM_STRICT, fov_deg=140.0, gaze=[-0.3, 1.0, 0.0])
    gv, gb, st, err, mism = full_parity(ctx, sc, r)
    assert gb.any() and (gv > 0).sum() > 10
    assert st["corner_tests"] > 0
