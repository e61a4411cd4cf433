"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the oracle.

* Bits: exact.
* v: within 1e-5 relative.  A viewpoint with patches at the edge of a
  field-of-view cone (the oracle decides the cone in float64; the kernel's
  float32 evaluation may decide a pair differently only where the cone
  margin is within VO_FOV_BAND of the edge) may instead lie anywhere between
  the oracle's value without the edge terms it counted and with the edge
  terms it left out.
* Colors: equal to the oracle's except at cells the device counts as bin-edge
  cells.  The device counts a cell when x = (L-1) v / v_ref, computed in
  float32 from its own v and v_ref, lies within 1e-5 x of an inner bin edge
  (an integer in 1..L-2).  A mismatch needs the device's x and the oracle's
  x on two sides of an edge; they differ by at most (e_v + e_ref + 3u) x,
  with e_v, e_ref <= 12u + 1e-6 the kernel's error bound on v, about
  2.5e-6 x < 1e-5 x, so every mismatch is at a counted cell.  The count
  itself is recomputed here from the device's v and v_ref and must equal
  vcm_stats.edge_cells.
"""

import numpy as np

from oracle import oracle as O

V_RTOL = 1e-5   # relative tolerance on visibility (float32 path vs float64 oracle)
EDGE_RTOL = np.float32(1e-5)   # the device's bin-edge criterion (k_quantise)


def _stats_bytes():
    from paper_1310_7297_gb300 import vcm

    return vcm.STATS_BYTES


def gpu_run(ctx, req, bits=True):
    """One request through vcm_compute into outputs prefilled with
    sentinels (NaN values, colour 255, bit words 0xA5A5A5A5), so that a
    viewpoint the kernels never write fails the comparison."""
    import torch

    from paper_1310_7297_gb300 import VCM_EMIT_BITS, n_viewpoints, stats_from_tensor, words

    dev = torch.device("cuda", ctx.device)
    n = n_viewpoints(req)
    req = dict(req)
    if bits:
        req["flags"] = req.get("flags", 0) | VCM_EMIT_BITS
    v = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
    c = torch.full((n,), 255, dtype=torch.uint8, device=dev)
    b = torch.full((n * words(req),), -1515870811, dtype=torch.int32, device=dev) if bits else None
    s = torch.zeros(_stats_bytes(), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx.vcm_compute(req, v.data_ptr(), c.data_ptr(), b.data_ptr() if b is not None else None, s.data_ptr(),
                    stream.cuda_stream)
    torch.cuda.synchronize()
    v = v.cpu().numpy().astype(np.float64)
    c = c.cpu().numpy()
    if bits:
        b = b.cpu().numpy().view(np.uint32).reshape(n, -1)
    return v, c, b, stats_from_tensor(s)


def compare_v(ov, gv, where="", band=None):
    """v within V_RTOL of the oracle's, and the same zero pattern, except at
    viewpoints with field-of-view band pairs (band[:, 0] > 0), whose value
    must lie in [v - band[:, 1], v + band[:, 2]] (widened by V_RTOL).
    Returns (max relative error off the band, number of band viewpoints)."""
    ov = np.asarray(ov, np.float64)
    gv = np.asarray(gv, np.float64)
    flex = np.zeros(ov.shape, bool) if band is None else np.asarray(band)[:, 0] > 0
    fixed = ~flex
    bad = fixed & ((ov == 0.0) != (gv == 0.0))
    assert not bad.any(), "zero pattern differs %s: %d cells, first %s" % (where, int(bad.sum()),
                                                                         np.nonzero(bad)[0][:5])
    worst = 0.0
    nz = fixed & (ov > 0)
    if nz.any():
        rel = np.abs(gv[nz] - ov[nz]) / ov[nz]
        assert rel.max() <= V_RTOL, "max rel err %.3e %s" % (rel.max(), where)
        worst = float(rel.max())
    if flex.any():
        b = np.asarray(band)[flex]
        lo = (ov[flex] - b[:, 1]) * (1.0 - V_RTOL)
        hi = (ov[flex] + b[:, 2]) * (1.0 + V_RTOL)
        ok = (gv[flex] >= lo - 1e-300) & (gv[flex] <= hi)
        assert ok.all(), "cone-edge viewpoint outside its bracket %s: %s" % (where, np.nonzero(flex)[0][~ok][:5])
    return worst, int(flex.sum())


def compare_bits(ob, gb, where=""):
    ob = np.asarray(ob, np.uint32)
    gb = np.asarray(gb, np.uint32)
    assert ob.shape == gb.shape
    bad = np.nonzero((ob != gb).any(axis=1))[0]
    assert bad.size == 0, "bits differ %s at %d viewpoints, first %s" % (where, bad.size, bad[:5])


def device_edge_cells(gv, v_ref, levels):
    """The cells the device counts as bin-edge cells, recomputed with its
    own float32 operations: x = (L-1) v / v_ref (a multiply and an IEEE
    divide), r = rint(x), edge iff 1 <= r <= L-2 and |x - r| <= 1e-5 x."""
    v = np.asarray(gv, np.float64).astype(np.float32)
    vref = np.float32(v_ref)
    edge = np.zeros(v.shape, bool)
    if not vref > 0:
        return edge
    pos = v > 0
    x = (np.float32(levels - 1) * v[pos]) / vref
    r = np.rint(x)
    edge[pos] = (r >= 1) & (r <= levels - 2) & (np.abs(x - r) <= EDGE_RTOL * x)
    return edge


def compare_colors(ov, gv, gc, levels, dev_v_ref, oracle_v_ref=None, flex=None):
    """Colors equal the oracle's (from its own v and `oracle_v_ref`, by
    default the given v_ref or else its largest v) except at the device's
    bin-edge cells and at cone-edge viewpoints (`flex`).  Returns
    (mismatches, device edge cells)."""
    ov = np.asarray(ov, np.float64)
    if oracle_v_ref is None or not oracle_v_ref > 0:
        oracle_v_ref = float(np.max(ov)) if ov.size else 0.0
    oc = O.quantise(ov, oracle_v_ref, levels)
    edge = device_edge_cells(gv, dev_v_ref, levels)
    mism = oc != np.asarray(gc)
    if flex is not None:
        mism &= ~flex
    stray = mism & ~edge
    assert not stray.any(), "color mismatch at a cell the device does not count as a bin edge: %s" % (
        np.nonzero(stray)[0][:5])
    return int(mism.sum()), int(edge.sum())


def full_parity(ctx, scene, req, bits=True):
    """The whole request on the device against the oracle: bits, v, colors,
    and the device's bin-edge count recomputed from its own output."""
    gv, gc, gb, st = gpu_run(ctx, req, bits)
    if bits:
        ov, ob, band = O.run(scene, req, bits=True, band=True)
        compare_bits(ob, gb)
    else:
        ov, band = O.run(scene, req, band=True)
    err, n_flex = compare_v(ov, gv, band=band)
    given = req.get("v_ref", 0.0)
    mism, n_edge = compare_colors(ov, gv, gc, req["color_levels"], st["v_ref"], given if given > 0 else None,
                                  flex=band[:, 0] > 0)
    assert st["edge_cells"] == n_edge, "device counts %d bin-edge cells, its own v gives %d" % (st["edge_cells"],
                                                                                              n_edge)
    return gv, gb, st, err, mism
