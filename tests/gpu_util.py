"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the oracle (bits exact, v within 1e-5 relative, colors exact
except near bin edges)."""

import numpy as np

from oracle import oracle as O

V_RTOL = 1e-5   # relative tolerance on visibility (float32 path vs float64 oracle)


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


def compare_v(ov, gv, where=""):
    ov = np.asarray(ov, np.float64)
    gv = np.asarray(gv, np.float64)
    assert np.array_equal(ov == 0.0, gv == 0.0), "zero pattern differs %s: %d cells" % (
        where, int(np.sum((ov == 0) != (gv == 0))))
    nz = ov > 0
    if nz.any():
        rel = np.abs(gv[nz] - ov[nz]) / ov[nz]
        assert rel.max() <= V_RTOL, "max rel err %.3e %s" % (rel.max(), where)
        return float(rel.max())
    return 0.0


def compare_bits(ob, gb, where=""):
    ob = np.asarray(ob, np.uint32)
    gb = np.asarray(gb, np.uint32)
    assert ob.shape == gb.shape
    bad = np.nonzero((ob != gb).any(axis=1))[0]
    assert bad.size == 0, "bits differ %s at %d viewpoints, first %s" % (where, bad.size, bad[:5])


def compare_colors(ov, gc, levels, v_ref=None):
    """Colors equal the oracle's, except at cells whose (L-1) v / v_ref lies
    within 2e-5 (relative) of a bin edge.  Returns the number of such
    mismatches."""
    vref = float(v_ref) if v_ref and v_ref > 0 else float(np.max(ov)) if ov.size else 0.0
    oc = O.quantise(ov, vref, levels)
    mism = np.nonzero(oc != gc)[0]
    if mism.size:
        x = (levels - 1) * ov[mism] / vref
        near = np.abs(x - np.rint(x)) <= 2e-5 * x
        assert near.all(), "color mismatch away from a bin edge at %s" % mism[~near][:5]
    return int(mism.size)


def full_parity(ctx, scene, req, bits=True):
    gv, gc, gb, st = gpu_run(ctx, req, bits)
    if bits:
        ov, ob = O.run(scene, req, bits=True)
        compare_bits(ob, gb)
    else:
        ov = O.run(scene, req)
    err = compare_v(ov, gv)
    mism = compare_colors(ov, gc, req["color_levels"], req.get("v_ref", 0.0))
    return gv, gb, st, err, mism
