"""Seeded input generators: determinism, lattice, sizes, keep-out of the target."""

import numpy as np

import synth
from synth import PCG32


def test_pcg32_reference_stream():
    # pcg32 (XSH-RR) with the SplitMix64 seeding is deterministic per (seed, stream)
    a = [PCG32(42, 1).next_u32() for _ in range(3)]
    b = PCG32(42, 1)
    assert a[0] == b.next_u32()
    c = PCG32(42, 2)
    assert [c.next_u32() for _ in range(4)] != [PCG32(42, 1).next_u32() for _ in range(4)]
    u = PCG32(7)
    xs = [u.uniform() for _ in range(20000)]
    assert 0.0 <= min(xs) and max(xs) < 1.0 and abs(np.mean(xs) - 0.5) < 0.01


def test_workloads_are_deterministic_and_on_lattice():
    s1, r1 = synth.workload_2d()
    s2, r2 = synth.workload_2d()
    assert s1.digest() == s2.digest() and r1 == r2
    assert s1.n == 100 and r1["grid_nx"] == 128 and r1["patches_u"] == 64
    s3, r3 = synth.workload_3d(grid=64, n_boxes=500)
    assert s3.n == 500 and s3.dims == 3
    lim = synth.COORD_LIMIT_UNITS
    for s in (s1, s3):
        assert np.all(s.lo <= s.hi) and np.all(np.abs(s.lo) <= lim) and np.all(np.abs(s.hi) <= lim)
        # float32 copies are exact
        assert np.array_equal(s.lo_f32().astype(np.float64) * 1024, s.lo.astype(np.float64))
    assert r3["layer_z"] == [synth.snap(1.7 + 10 * k) for k in range(5)]


def test_boxes_stay_off_the_target():
    s, r = synth.workload_3d(grid=64, n_boxes=3000, half_m=200.0, n_components=2, sigma_m=(20.0, 40.0))
    c = np.array(r["center"])
    # target x in [-10, 10] m, y = 0, z in [25, 35] m, inflated by 1 m
    U = 1024
    lo_t = c + np.array([-11 * U, -1 * U, -6 * U])
    hi_t = c + np.array([11 * U, 1 * U, 6 * U])
    overlap = np.all((s.lo <= hi_t) & (lo_t <= s.hi), axis=1)
    assert not overlap.any()


def test_batched_mix_shapes():
    s, reqs = synth.workload_batched(n_requests=8, n_boxes=2000)
    assert len(reqs) == 8
    for r in reqs:
        assert 64 <= r["grid_nx"] <= 1024 and 1 <= len(r["layer_z"]) <= 8
        assert (r["patches_u"], r["patches_w"]) in [(8, 4), (16, 8), (32, 16), (64, 32)]
        assert r["normal"] in (0, 1, 2, 3)
    t = synth.poisson_arrivals(1, 100.0, 2000)
    assert np.all(np.diff(t) > 0) and abs(len(t) / t[-1] - 100.0) < 10.0
