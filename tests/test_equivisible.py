"""The paper's equi-visible colouring (the comparison workload of bench.py
--mode equivisible), pinned on CPU against Eq. 1 and Eq. 2 themselves."""

import math

import numpy as np

from paper_1310_7297_gb300 import equivisible as E


def test_distance_edges_drop_the_visual_angle_by_mu():
    S, mu, d0 = 10.0, 4.0, 1.0
    d = E.distance_partition(S, mu, d0)
    v = 2.0 * np.arctan(S / (2.0 * d))                       # Eq. 1
    assert np.allclose(np.diff(v), -math.radians(mu), rtol=0, atol=1e-12)
    assert np.all(np.diff(d) > 0) and d[0] == d0
    assert v[-1] >= math.radians(mu) > v[-1] - math.radians(mu)   # stops at the resolution


def test_angle_edges_give_the_stepped_visual_angles():
    S, mu, dm = 10.0, 2.0, 30.0
    a = E.angle_partition(S, mu, dm)
    assert a[0] == 90.0 and a[-1] == 0.0 and np.all(np.diff(a) < 0)
    v = E.paper_visibility(S, dm, a[:-1])                    # Eq. 1 with Eq. 2's perceived size
    v0 = 2.0 * math.atan(S / (2.0 * dm))
    assert np.allclose(v, v0 - math.radians(mu) * np.arange(len(v)), rtol=0, atol=1e-12)


def test_cells_hold_their_points_and_centres():
    S = 10.0
    P = E.Partition(S, 4.0, 1.0)
    rng = np.random.default_rng(3)
    d = rng.uniform(1.0, P.d_edges[-1] * 0.999, 2000)
    a = rng.uniform(0.5, 89.5, 2000)
    side = rng.choice([-1.0, 1.0], 2000)
    x, y = side * d * np.cos(np.radians(a)), d * np.sin(np.radians(a))
    band, cell = P.cell_of(x, y)
    assert np.all(band >= 0)
    for b, c, dd, aa in zip(band, cell, d, a):
        assert P.d_edges[b] <= dd < P.d_edges[b + 1]
        e = P.a_edges[b]
        assert e[c + 1] <= aa <= e[c]
    # behind the target, nearer than d_0 or beyond the last edge: no cell
    b2, _ = P.cell_of(np.array([0.0, 0.0, 0.0]), np.array([-5.0, 0.5, P.d_edges[-1] * 1.01]))
    assert np.all(b2 == -1)
    # the value of a point is its cell centre's (the visibility seen from there)
    v = P.values_at(x[:5], y[:5])
    for i in range(5):
        dc, ac = P.centres(band[i])
        assert v[i] == E.paper_visibility(S, dc, ac[cell[i]])


def test_eq6_and_quantiser():
    c = np.array([0, 3, 5, 7])
    assert E.eq6_error(c, c) == 0.0
    assert E.eq6_error(c, np.zeros(4)) == 1.0
    assert abs(E.eq6_error([2, 2], [1, 2], area=[3.0, 1.0]) - 3.0 / 8.0) < 1e-15
    v = np.array([0.0, 0.1, 0.5, 1.0])
    assert list(E.quantise(v, 8)) == [0, 1, 4, 7]
