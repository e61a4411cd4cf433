"""Host side of bench.py (CPU): the variant requests of `--mode modes` are
valid requests whose oracle values order as the definitions fix, and the
oracle timing fills the time it is given."""

import numpy as np

import bench
import synth
from oracle import oracle as O


def _small():
    return synth.workload_3d(seed=7, grid=24, layers=3, patches=(8, 4), n_boxes=300, half_m=300.0)


def test_mode_variants_order_as_defined():
    scene, req = _small()
    var = dict(bench.mode_variants(req))
    assert list(var) == ["plain", "strict", "fov120", "strict_fov120", "two_sided", "viewer"]
    n = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    idx = np.arange(0, n, 3)
    v = {k: O.run(scene, r, indices=idx) for k, r in var.items()}
    for k, x in v.items():
        assert np.isfinite(x).all() and (x >= 0).all(), k
    assert (v["plain"] > 0).sum() > 20
    # strict keeps a viewpoint's value only when every patch is visible
    assert np.all((v["strict"] == 0) | (v["strict"] == v["plain"]))
    # a field of view only removes patches; two sides only add the back
    assert np.all(v["fov120"] <= v["plain"] * (1 + 1e-12))
    assert np.all(v["strict_fov120"] <= v["fov120"] * (1 + 1e-12))
    assert np.all(v["two_sided"] >= v["plain"] * (1 - 1e-12))
    assert (v["two_sided"] > v["plain"]).any()
    # the viewer-centric map: one segment per cell from the viewer
    assert (v["viewer"] > 0).sum() > 20


def test_oracle_rate_fills_its_time():
    # the full 3D workload: a grid too large to exhaust in the time given
    scene, req = synth.workload_3d()
    r = bench.oracle_rate(scene, req, 0.5, seed=3)
    P = req["patches_u"] * req["patches_w"]
    assert r["viewpoints"] >= 64 and r["seconds"] >= 0.3
    assert abs(r["value"] - r["cells_per_s"] * P) <= 1e-6 * r["value"]
    assert r["cores"] >= 1
