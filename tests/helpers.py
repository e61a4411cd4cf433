"""Small shared helpers for the tests (request construction in lattice units)."""

import numpy as np

from synth import Scene

U = 1024  # lattice units per metre


def req3(center, axis_u=0, axis_w=4, normal=2, width=20 * U, height=10 * U, pu=4, pw=2,
         origin=(0, 0), step=(U, U), n=(1, 1), layers=(0,), levels=16, v_ref=0.0, flags=0):
    return {
        "dims": 3, "center": list(center), "axis_u": axis_u, "axis_w": axis_w, "normal": normal,
        "width": width, "height": height, "patches_u": pu, "patches_w": pw,
        "grid_origin": list(origin), "grid_step": list(step), "grid_nx": n[0], "grid_ny": n[1],
        "layer_z": list(layers), "color_levels": levels, "v_ref": v_ref, "flags": flags,
    }


def req2(center, axis_u=0, normal=2, width=10 * U, pu=8, origin=(0, 0), step=(U, U), n=(1, 1),
         levels=8, v_ref=0.0, flags=0):
    return {
        "dims": 2, "center": [center[0], center[1], 0], "axis_u": axis_u, "axis_w": 4,
        "normal": normal, "width": width, "height": 0, "patches_u": pu, "patches_w": 1,
        "grid_origin": list(origin), "grid_step": list(step), "grid_nx": n[0], "grid_ny": n[1],
        "layer_z": [0], "color_levels": levels, "v_ref": v_ref, "flags": flags,
    }


def single_viewpoint(req, q):
    """Place a 1x1 grid so that its only viewpoint is exactly q (units)."""
    r = dict(req)
    r["grid_origin"] = [q[0] - 1, q[1] - 1]
    r["grid_step"] = [2, 2]
    r["grid_nx"] = r["grid_ny"] = 1
    if r["dims"] == 3:
        r["layer_z"] = [q[2]]
    return r


def scene(dims, boxes):
    """boxes: list of (lo, hi) triples in units."""
    if not boxes:
        return Scene(dims, np.zeros((0, 3), np.int64), np.zeros((0, 3), np.int64))
    lo = [list(b[0]) + [0] * (3 - len(b[0])) for b in boxes]
    hi = [list(b[1]) + [0] * (3 - len(b[1])) for b in boxes]
    return Scene(dims, lo, hi)


def random_tiny_scene(rng, dims, n_boxes, span):
    """Boxes with coordinates in a small integer range, so that ties
    (touching faces, edges and corners) are frequent."""
    lo, hi = [], []
    for _ in range(n_boxes):
        a = rng.integers(-span, span, size=3)
        e = rng.integers(0, span // 2 + 1, size=3)
        b = a + e
        if dims == 2:
            a[2] = b[2] = 0
        lo.append(a)
        hi.append(b)
    return Scene(dims, np.array(lo, np.int64), np.array(hi, np.int64))
