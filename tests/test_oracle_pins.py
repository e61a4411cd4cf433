"""Pins of the CPU oracle against things other than itself (no GPU).

Each group targets a plausible mistake:
  * predicate: exact separating-axis brute force on tie-heavy tiny scenes and
    hand-built touching / grazing / inside cases (a wrong comparison, a
    strict instead of closed interval, a mishandled parallel axis);
  * geometry: patch centres and viewpoints rebuilt with Fractions (a wrong
    index, a transposed u/w, a wrong rounding);
  * measure: the paper's worked example of Eq. 1 and closed-form subtended
    angles and solid angles, with the midpoint rule's O(h^2) convergence (a
    dropped cos, a wrong power of d, a wrong sign of the normal);
  * invariants: a full wall gives zero, adding boxes never clears a bit,
    mirror symmetry, viewpoints behind the target or inside a box give zero;
  * colors: the quantiser's defining properties;
  * blocking is convex in the viewpoint and in the patch (the one-box
    shortcuts of the GPU path rest on it), by the exact predicate;
  * sides and field of view: mirror images through the target plane and
    through x = 0, a cone equal to a cropped target, the paper's FOV region
    bounded by rays from the target ends.
"""

import math
import os

import numpy as np
import pytest

import brute
from helpers import U, random_tiny_scene, req2, req3, scene, single_viewpoint
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = [x.strip() for x in line.split("=", 1)]
            vals[k] = float(v)
    return vals


# ---------------------------------------------------------------------------
# exact predicate
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [2, 3])
def test_predicate_matches_separating_axis_on_tie_heavy_cases(dims):
    rng = np.random.default_rng(100 + dims)
    n_hit = 0
    for _ in range(6000):
        span = int(rng.integers(2, 9))
        q = [int(x) for x in rng.integers(-span, span + 1, size=3)]
        p = [int(x) for x in rng.integers(-span, span + 1, size=3)]
        lo = [int(x) for x in rng.integers(-span, span + 1, size=3)]
        ext = [int(x) for x in rng.integers(0, 2 * span + 1, size=3)]
        if rng.random() < 0.15:
            ext[int(rng.integers(0, 3))] = 0  # zero-thickness box
        hi = [lo[k] + ext[k] for k in range(3)]
        if dims == 2:
            q[2] = p[2] = lo[2] = hi[2] = 0
        want = brute.segment_hits_box_sat(dims, q, p, lo, hi)
        got = O.segment_hits_box(dims, q, p, lo, hi)
        assert bool(got) == want, (q, p, lo, hi)
        n_hit += want
    assert 500 < n_hit < 5500  # both outcomes well represented


def test_predicate_large_coordinates():
    """Values near the 2^24-unit coordinate limit stay exact."""
    rng = np.random.default_rng(7)
    L = 1 << 24
    for _ in range(3000):
        q = [int(x) for x in rng.integers(-L, L + 1, size=3)]
        p = [int(x) for x in rng.integers(-L, L + 1, size=3)]
        # box near the segment's midpoint so hits are common
        m = [(q[k] + p[k]) // 2 for k in range(3)]
        lo = [max(-L, m[k] - int(rng.integers(0, 1 << 20))) for k in range(3)]
        hi = [min(L, m[k] + int(rng.integers(0, 1 << 20))) for k in range(3)]
        assert bool(O.segment_hits_box(3, q, p, lo, hi)) == brute.segment_hits_box_sat(3, q, p, lo, hi)


@pytest.mark.parametrize("case,want", [
    # segment grazing the top face of a box (touching counts, Def. 4)
    (((0, 0, 10), (100, 0, 10), (40, -5, 0), (60, 5, 10)), True),
    # one unit above the face: clear
    (((0, 0, 11), (100, 0, 11), (40, -5, 0), (60, 5, 10)), False),
    # through an edge of the box (diagonal, touching only the edge line)
    (((0, 0, 0), (10, 10, 0), (5, 0, -1), (6, 5, 1)), True),
    # passing one unit outside a corner
    (((0, 1, 0), (10, 11, 0), (5, 0, -1), (6, 5, 1)), False),
    # exactly through a corner point
    (((0, 0, 0), (20, 20, 20), (10, 10, 10), (12, 12, 12)), True),
    # segment ends exactly on the box face (p touches the box)
    (((0, 0, 0), (10, 0, 0), (10, -1, -1), (12, 1, 1)), True),
    # segment stops one unit short of the box
    (((0, 0, 0), (9, 0, 0), (10, -1, -1), (12, 1, 1)), False),
    # viewpoint inside the box
    (((5, 5, 5), (100, 100, 100), (0, 0, 0), (10, 10, 10)), True),
    # viewpoint on a face, segment leaving it
    (((10, 5, 5), (100, 5, 5), (0, 0, 0), (10, 10, 10)), True),
    # parallel to an axis, inside the slab boundary (a_k == 0, d_k == 0)
    (((0, 0, 0), (0, 100, 0), (0, 40, -5), (5, 60, 5)), True),
    # parallel, just outside the slab
    (((-1, 0, 0), (-1, 100, 0), (0, 40, -5), (5, 60, 5)), False),
    # box entirely behind the viewpoint
    (((0, 0, 0), (100, 0, 0), (-20, -1, -1), (-10, 1, 1)), False),
    # zero-thickness wall crossed
    (((0, 0, 0), (100, 0, 0), (50, -5, -5), (50, 5, 5)), True),
])
def test_predicate_hand_built_ties(case, want):
    q, p, lo, hi = case
    assert brute.segment_hits_box_sat(3, q, p, lo, hi) == want
    assert bool(O.segment_hits_box(3, q, p, lo, hi)) == want


# ---------------------------------------------------------------------------
# geometry: patch centres and viewpoints
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("axes", [(0, 4, 2), (1, 4, 3), (2, 5, 0), (4, 0, 3), (3, 4, 1)])
@pytest.mark.parametrize("N", [(1, 1), (3, 5), (4, 2), (7, 3), (64, 32)])
def test_patch_centres_match_fraction_definition(axes, N):
    r = req3((1234, -5679, 30 * U + 3), axis_u=axes[0], axis_w=axes[1], normal=axes[2],
             width=20 * U + 7, height=10 * U + 3, pu=N[0], pw=N[1])
    got = O.patch_centres(r)
    want = np.array(brute.patch_centres(r), np.int64)
    assert np.array_equal(got, want)
    # patch j = iw * pu + iu moves along u first
    au = axes[0] >> 1
    if N[0] > 1:
        step = got[1, au] - got[0, au]
        assert step != 0 and np.sign(step) == (-1 if axes[0] & 1 else 1)


def test_patch_centres_2d():
    r = req2((-3000, 4000), axis_u=3, normal=0, width=10 * U + 1, pu=9)
    assert np.array_equal(O.patch_centres(r), np.array(brute.patch_centres(r), np.int64))


def test_viewpoints_match_fraction_definition_odd_steps():
    r = req3((0, 0, 0), origin=(-1001, 777), step=(33, 17), n=(7, 5), layers=(1741, -3, 22221))
    for idx in range(7 * 5 * 3):
        assert tuple(O.viewpoint(r, idx)) == brute.viewpoint(r, idx)
    # index order is ((layer * ny) + iy) * nx + ix
    assert tuple(O.viewpoint(r, 1)) == brute.viewpoint(r, 1)
    assert O.viewpoint(r, 7)[1] != O.viewpoint(r, 0)[1]
    assert O.viewpoint(r, 35)[2] == -3


# ---------------------------------------------------------------------------
# occlusion bits of whole viewpoints against the brute force
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,seed", [(2, 1), (2, 2), (3, 3), (3, 4), (3, 5)])
def test_bits_match_brute_force_tiny_scenes(dims, seed):
    rng = np.random.default_rng(seed)
    sc = random_tiny_scene(rng, dims, 6, 12)
    if dims == 3:
        r = req3((0, -20, 6), width=16, height=8, pu=4, pw=4, origin=(-13, -7), step=(7, 5),
                 n=(4, 4), layers=(0, 5, 9))
    else:
        r = req2((0, -20), width=16, pu=8, origin=(-13, -7), step=(7, 5), n=(4, 4))
    n = r["grid_nx"] * r["grid_ny"] * len(r["layer_z"])
    v, b = O.run(sc, r, bits=True, threads=2)
    for idx in range(n):
        want = brute.pack_bits(brute.bits(sc, r, idx))
        assert list(b[idx]) == want, idx


# ---------------------------------------------------------------------------
# measure: the paper's worked example and closed forms
# ---------------------------------------------------------------------------

def test_paper_worked_example_visual_angle():
    """Eq. 1 example (Section II-B.1): S = 300 m at D = 400 m head-on gives
    41.11 degrees.  The 2D measure (sum of len cos(theta)/d) is the midpoint
    rule for the subtended angle, so it converges to that value."""
    g = read_golden("paper_visual_angle.txt")
    S, D = int(g["S_m"]), int(g["D_m"])
    errs = []
    for N in (64, 128, 256, 512):
        r = single_viewpoint(req2((0, 0), axis_u=0, normal=2, width=S * U, pu=N), (0, D * U, 0))
        v = O.run(scene(2, []), r)[0]
        exact = 2.0 * math.atan(S / (2.0 * D))
        errs.append(abs(v - exact))
        assert round(math.degrees(v), int(g["printed_decimals"])) == pytest.approx(g["V_deg"], abs=1e-9)
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.5  # midpoint rule: error ~ h^2


def _subtended_2d(q, a, b):
    ax, ay = a[0] - q[0], a[1] - q[1]
    bx, by = b[0] - q[0], b[1] - q[1]
    return math.atan2(abs(ax * by - ay * bx), ax * bx + ay * by)


@pytest.mark.parametrize("q_m", [(37.0, 55.0), (-120.5, 8.25), (3.0, 0.75), (400.0, 1.0)])
def test_2d_sum_converges_to_subtended_angle(q_m):
    W = 10.0
    prev = None
    for N in (64, 128, 256):
        r = single_viewpoint(req2((0, 0), width=int(W * U), pu=N), (int(q_m[0] * U), int(q_m[1] * U), 0))
        v = O.run(scene(2, []), r)[0]
        exact = _subtended_2d(q_m, (-W / 2, 0.0), (W / 2, 0.0))
        err = abs(v - exact)
        assert err < 2e-3 * exact
        if prev is not None and prev > 1e-13:
            assert 3.0 < prev / err < 5.0
        prev = err


def _corner(x, y, d):
    return math.atan(x * y / (d * math.sqrt(x * x + y * y + d * d)))


def _rect_solid_angle(q, c, W, H):
    """Rectangle in the plane y = c_y spanning x in c_x +- W/2, z in c_z +- H/2,
    seen from q: sum of the four corner terms about the foot of the
    perpendicular."""
    d = abs(q[1] - c[1])
    x1, x2 = c[0] - W / 2 - q[0], c[0] + W / 2 - q[0]
    z1, z2 = c[2] - H / 2 - q[2], c[2] + H / 2 - q[2]
    return _corner(x2, z2, d) - _corner(x1, z2, d) - _corner(x2, z1, d) + _corner(x1, z1, d)


def _triangle_solid_angle(q, a, b, c):
    """Van Oosterom and Strackee (1983): tan(Omega/2) = |a.(b x c)| /
    (|a||b||c| + (a.b)|c| + (a.c)|b| + (b.c)|a|)."""
    A = [a[k] - q[k] for k in range(3)]
    B = [b[k] - q[k] for k in range(3)]
    C = [c[k] - q[k] for k in range(3)]
    cross = (B[1] * C[2] - B[2] * C[1], B[2] * C[0] - B[0] * C[2], B[0] * C[1] - B[1] * C[0])
    num = abs(sum(A[k] * cross[k] for k in range(3)))
    la, lb, lc = (math.sqrt(sum(x * x for x in V)) for V in (A, B, C))
    dot = lambda X, Y: sum(X[k] * Y[k] for k in range(3))
    den = la * lb * lc + dot(A, B) * lc + dot(A, C) * lb + dot(B, C) * la
    return 2.0 * math.atan2(num, den)


def test_closed_forms_agree_with_each_other():
    q, c, W, H = (37.0, 55.0, -12.0), (0.0, 0.0, 30.0), 20.0, 10.0
    corners = [(c[0] - W / 2, 0.0, c[2] - H / 2), (c[0] + W / 2, 0.0, c[2] - H / 2),
               (c[0] + W / 2, 0.0, c[2] + H / 2), (c[0] - W / 2, 0.0, c[2] + H / 2)]
    two_tri = (_triangle_solid_angle(q, corners[0], corners[1], corners[2]) +
               _triangle_solid_angle(q, corners[0], corners[2], corners[3]))
    assert _rect_solid_angle(q, c, W, H) == pytest.approx(two_tri, rel=1e-12)
    for d in (5.0, 20.0, 100.0):
        onaxis = 4.0 * math.asin(W * H / math.sqrt((W * W + 4 * d * d) * (H * H + 4 * d * d)))
        assert _rect_solid_angle((0.0, d, 30.0), c, W, H) == pytest.approx(onaxis, rel=1e-12)


@pytest.mark.parametrize("q_m", [(0.0, 5.0, 30.0), (0.0, 20.0, 30.0), (0.0, 100.0, 30.0),
                                 (37.0, 55.0, -12.0), (-8.0, 3.0, 33.5)])
def test_3d_sum_converges_to_rectangle_solid_angle(q_m):
    W, H, c = 20.0, 10.0, (0.0, 0.0, 30.0)
    exact = _rect_solid_angle(q_m, c, W, H)
    prev = None
    for pu, pw in ((32, 16), (64, 32), (128, 64)):
        r = single_viewpoint(req3((0, 0, 30 * U), width=20 * U, height=10 * U, pu=pu, pw=pw),
                             tuple(int(x * U) for x in q_m))
        v = O.run(scene(3, []), r)[0]
        err = abs(v - exact)
        assert err < 2e-3 * exact
        if prev is not None:
            assert 3.0 < prev / err < 5.0
        prev = err


def test_target_orientation_and_normal_sign():
    """Same target described with u/w swapped and the normal flipped: the
    visible measure is the same from the front and zero from behind."""
    q = (37 * U, 55 * U, -12 * U)
    a = single_viewpoint(req3((0, 0, 30 * U), axis_u=0, axis_w=4, normal=2, width=20 * U,
                              height=10 * U, pu=32, pw=16), q)
    b = single_viewpoint(req3((0, 0, 30 * U), axis_u=4, axis_w=0, normal=2, width=10 * U,
                              height=20 * U, pu=16, pw=32), q)
    c = single_viewpoint(req3((0, 0, 30 * U), axis_u=0, axis_w=4, normal=3, width=20 * U,
                              height=10 * U, pu=32, pw=16), q)
    va, vb, vc = (O.run(scene(3, []), r)[0] for r in (a, b, c))
    assert va == pytest.approx(vb, rel=1e-13)
    assert vc == 0.0
    # a 2:1 target is not symmetric in u and w: transposing the sides changes v
    d = single_viewpoint(req3((0, 0, 30 * U), width=10 * U, height=20 * U, pu=32, pw=16), q)
    assert abs(O.run(scene(3, []), d)[0] - va) > 1e-3 * va


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

def test_full_wall_gives_zero():
    r = req3((0, 0, 30 * U), width=20 * U, height=10 * U, pu=8, pw=4, origin=(-64 * U, 5 * U),
             step=(16 * U, 16 * U), n=(8, 4), layers=(2 * U, 30 * U, 70 * U))
    wall = scene(3, [((-2000 * U, 2 * U, -10 * U), (2000 * U, 3 * U, 2000 * U))])
    v, b = O.run(wall, r, bits=True, threads=2)
    assert np.all(v == 0.0)
    assert np.all(b == 0xFFFFFFFF)
    v0 = O.run(scene(3, []), r)
    assert np.all(v0 > 0.0)


def test_viewpoint_inside_box_sees_nothing():
    r = single_viewpoint(req3((0, 0, 30 * U), pu=4, pw=2), (100 * U, 200 * U, 5 * U))
    box = scene(3, [((90 * U, 190 * U, 0), (110 * U, 210 * U, 10 * U))])
    v, b = O.run(box, r, bits=True)
    assert v[0] == 0.0 and b[0, 0] == 0xFF


def test_behind_target_is_zero_but_bits_still_defined():
    r = req3((0, 0, 30 * U), pu=4, pw=2, origin=(-100 * U, -300 * U), step=(25 * U, 25 * U), n=(8, 4),
             layers=(2 * U,))
    sc = scene(3, [((-5 * U, -120 * U, 0), (5 * U, -110 * U, 40 * U))])
    v, b = O.run(sc, r, bits=True, threads=2)
    assert np.all(v == 0.0)           # every viewpoint has y < 0: behind a +y target
    assert b.any() and not b.all()    # occlusion is still evaluated per segment


@pytest.mark.parametrize("seed", [11, 12])
def test_monotone_under_box_insertion(seed):
    import synth
    sc, r = synth.workload_3d(seed=seed, grid=16, layers=2, patches=(8, 4), n_boxes=60, half_m=150.0,
                              n_components=3, sigma_m=(20.0, 60.0))
    v1, b1 = O.run(sc, r, bits=True, threads=4)
    rng = np.random.default_rng(seed)
    extra_lo = rng.integers(-140 * U, 120 * U, size=(25, 3))
    extra_lo[:, 2] = 0
    extra_hi = extra_lo + rng.integers(5 * U, 30 * U, size=(25, 3))
    sc2 = sc.with_boxes(extra_lo, extra_hi)
    v2, b2 = O.run(sc2, r, bits=True, threads=4)
    assert np.all((b1 & ~b2) == 0)     # no bit cleared
    assert np.all(v2 <= v1 + 1e-15 * np.abs(v1))
    assert (b2 != b1).any()


def test_mirror_symmetry():
    """Mirror x -> -x of a scene around a target centred at x = 0 with a grid
    symmetric about x = 0: values mirror exactly, bits mirror patch-wise."""
    rng = np.random.default_rng(5)
    n = 40
    lo = rng.integers(-80 * U, 70 * U, size=(n, 3))
    lo[:, 1] = rng.integers(3 * U, 80 * U, size=n)
    lo[:, 2] = 0
    hi = lo + rng.integers(2 * U, 12 * U, size=(n, 3))
    sc = scene(3, list(zip(lo.tolist(), hi.tolist())))
    mlo, mhi = lo.copy(), hi.copy()
    mlo[:, 0], mhi[:, 0] = -hi[:, 0], -lo[:, 0]
    msc = scene(3, list(zip(mlo.tolist(), mhi.tolist())))
    nx, ny = 10, 6
    r = req3((0, 0, 20 * U), width=12 * U, height=6 * U, pu=6, pw=3, origin=(-nx * 8 * U, 10 * U),
             step=(16 * U, 16 * U), n=(nx, ny), layers=(2 * U, 15 * U))
    v, b = O.run(sc, r, bits=True, threads=4)
    mv, mb = O.run(msc, r, bits=True, threads=4)
    P = 18
    for layer in range(2):
        for iy in range(ny):
            for ix in range(nx):
                i = (layer * ny + iy) * nx + ix
                j = (layer * ny + iy) * nx + (nx - 1 - ix)
                assert v[i] == pytest.approx(mv[j], rel=1e-13, abs=0)
                bi = [(int(b[i, k >> 5]) >> (k & 31)) & 1 for k in range(P)]
                bj = [(int(mb[j, k >> 5]) >> (k & 31)) & 1 for k in range(P)]
                for iw in range(3):
                    for iu in range(6):
                        assert bi[iw * 6 + iu] == bj[iw * 6 + (5 - iu)]
    assert (v > 0).any() and (b != 0).any()


# ---------------------------------------------------------------------------
# colors
# ---------------------------------------------------------------------------

def test_quantiser_properties():
    L = 8
    vref = 2.0
    v = np.array([0.0, 1e-30, vref * 0.5 / (L - 1), vref * 1.5 / (L - 1), vref * 6.5 / (L - 1),
                  vref * (1 - 1e-12), vref, 3 * vref])
    c = O.quantise(v, vref, L)
    assert list(c) == [0, 1, 1, 2, 7, 7, 7, 7]
    # monotone, zero only for zero, top level reached at v_ref, every level used
    rng = np.random.default_rng(3)
    vv = np.sort(rng.uniform(0, vref, 20000))
    cc = O.quantise(vv, vref, L)
    assert np.all(np.diff(cc.astype(int)) >= 0)
    assert set(cc.tolist()) == set(range(1, L))
    assert O.quantise(np.zeros(5), 0.0, L).tolist() == [0] * 5
    assert O.vmax(np.array([0.0, 3.0, 1.0])) == 3.0


# ---------------------------------------------------------------------------
# strict and viewer-centric modes
# ---------------------------------------------------------------------------

STRICT, VIEWER = 2, 4


def test_strict_mode_is_all_or_nothing():
    """Def. 3: the visible region holds the viewpoints that see every patch;
    there the strict value equals the unobstructed one, elsewhere it is 0."""
    import synth

    sc, r = synth.workload_3d(seed=41, grid=20, layers=3, patches=(8, 4), n_boxes=80, half_m=250.0,
                              n_components=4, sigma_m=(40.0, 100.0))
    vp, bp = O.run(sc, r, bits=True, threads=4)
    vs = O.run(sc, dict(r, flags=STRICT), threads=4)
    v0 = O.run(scene(3, []), r, threads=4)
    none_blocked = ~bp.astype(bool).any(axis=1)
    assert np.array_equal(vs[none_blocked], v0[none_blocked])
    assert np.all(vs[~none_blocked] == 0.0)
    assert np.array_equal(vs[none_blocked], vp[none_blocked])
    assert np.all(vs <= vp + 1e-15) and (vs > 0).any() and ((vp > 0) & (vs == 0)).any()


def _viewer_req(dims, viewer, S, origin, step, n, layers=(0,)):
    from helpers import req2, req3

    if dims == 2:
        r = req2((viewer[0], viewer[1]), width=S, origin=origin, step=step, n=n)
    else:
        r = req3(tuple(viewer), width=S, origin=origin, step=step, n=n, layers=layers)
    r["flags"] = VIEWER
    return r


def test_viewer_mode_reproduces_the_paper_example_exactly():
    """Section IV-B with Eq. 1: an object of S = 300 m at D = 400 m from the
    viewer subtends 41.11 degrees (the worked example of Section II-B.1)."""
    g = read_golden("paper_visual_angle.txt")
    S, D = int(g["S_m"]), int(g["D_m"])
    r = _viewer_req(2, (0, 0), S * U, (-1, D * U - 1), (2, 2), (1, 1))
    v = O.run(scene(2, []), r)[0]
    assert v == pytest.approx(2.0 * math.atan(S / (2.0 * D)), rel=1e-14)
    assert round(math.degrees(v), int(g["printed_decimals"])) == pytest.approx(g["V_deg"], abs=1e-9)


def test_viewer_mode_3d_square_solid_angle_and_blocking():
    """3D cells: the solid angle of an S x S square facing the viewer, checked
    against the corner-decomposition closed form; a wall zeroes the cells
    behind it and sets their bits, as the separating-axis brute force says."""
    S = 4 * U
    r = _viewer_req(3, (0, 0, 10 * U), S, (-40 * U, 5 * U), (10 * U, 10 * U), (8, 6), layers=(2 * U, 10 * U))
    v0 = O.run(scene(3, []), r)
    for idx in (0, 7, 20, 47, 60):
        q = O.viewpoint(r, idx) / U
        D = math.dist(q, (0.0, 0.0, 10.0))
        # square of side S at distance D, seen on its axis: rectangle formula
        ref = _rect_solid_angle((0.0, D, 0.0), (0.0, 0.0, 0.0), S / U, S / U)
        assert v0[idx] == pytest.approx(ref, rel=1e-12)
    wall = scene(3, [((-15 * U, 20 * U, 0), (15 * U, 21 * U, 30 * U))])
    v, b = O.run(wall, r, bits=True)
    for idx in range(v.shape[0]):
        q = tuple(int(x) for x in O.viewpoint(r, idx))
        hit = brute.segment_hits_box_sat(3, q, (0, 0, 10 * U), wall.lo[0], wall.hi[0])
        assert bool(b[idx, 0]) == hit
        assert (v[idx] == 0.0) == hit
    assert b.any() and not b.all()


# ---------------------------------------------------------------------------
# two-sided target and field of view
# ---------------------------------------------------------------------------

FLAG_TWO_SIDED = 8


def _mirror_y_scene(lo, hi):
    mlo, mhi = lo.copy(), hi.copy()
    mlo[:, 1], mhi[:, 1] = -hi[:, 1], -lo[:, 1]
    return mlo, mhi


def test_two_sided_front_equals_one_sided_and_back_mirrors_front():
    """A target in the plane y = 0: from the front a two-sided target gives
    exactly the one-sided values; from behind it gives exactly what the
    mirror image (y -> -y, scene mirrored too) gives from the front; on the
    plane it gives 0."""
    rng = np.random.default_rng(21)
    n = 50
    lo = rng.integers(-90 * U, 80 * U, size=(n, 3))
    lo[:, 2] = 0
    hi = lo + rng.integers(2 * U, 14 * U, size=(n, 3))
    keep = ~((lo[:, 0] < 12 * U) & (hi[:, 0] > -12 * U) & (lo[:, 1] < 2 * U) & (hi[:, 1] > -2 * U))
    lo, hi = lo[keep], hi[keep]
    sc = scene(3, list(zip(lo.tolist(), hi.tolist())))
    mlo, mhi = _mirror_y_scene(lo, hi)
    msc = scene(3, list(zip(mlo.tolist(), mhi.tolist())))
    nx, ny = 8, 9
    # rows iy = 0..8 at y = -64, -48, ..., 64 m: row 4 lies in the target plane
    base = dict(width=12 * U, height=6 * U, pu=6, pw=3, origin=(-nx * 8 * U, -72 * U),
                step=(16 * U, 16 * U), n=(nx, ny), layers=(2 * U, 15 * U))
    one = O.run(sc, req3((0, 0, 20 * U), **base))
    two = O.run(sc, req3((0, 0, 20 * U), flags=FLAG_TWO_SIDED, **base))
    two_m = O.run(msc, req3((0, 0, 20 * U), flags=FLAG_TWO_SIDED, **base))
    for layer in range(2):
        for iy in range(ny):
            for ix in range(nx):
                i = (layer * ny + iy) * nx + ix
                j = (layer * ny + (ny - 1 - iy)) * nx + ix
                if iy > 4:
                    assert two[i] == one[i]
                elif iy == 4:
                    assert two[i] == 0.0 and one[i] == 0.0
                else:
                    assert one[i] == 0.0
                    assert two[i] == two_m[j]
    assert (two[: nx * 4] > 0).any() and (two[nx * 5: nx * ny] > 0).any()


def test_two_sided_2d_from_behind_converges_to_subtended_angle():
    q_m = (3.0, -7.0)
    W = 10.0
    prev = None
    for N in (64, 128, 256):
        r = single_viewpoint(req2((0, 0), width=int(W * U), pu=N, flags=FLAG_TWO_SIDED),
                             (int(q_m[0] * U), int(q_m[1] * U), 0))
        v = O.run(scene(2, []), r)[0]
        exact = _subtended_2d(q_m, (-W / 2, 0.0), (W / 2, 0.0))
        err = abs(v - exact)
        assert err < 2e-3 * exact
        if prev is not None:
            assert 3.0 < prev / err < 5.0
        prev = err


def _fov(req, fov, gaze=(0.0, 0.0, 0.0)):
    r = dict(req)
    r["fov_deg"] = fov
    r["gaze"] = list(gaze)
    return r


def test_fov_none_full_and_half_space_equal_no_cone():
    import synth
    sc, r = synth.workload_3d(seed=13, grid=12, layers=2, patches=(8, 4), n_boxes=60, half_m=150.0,
                              n_components=3, sigma_m=(20.0, 60.0))
    v = O.run(sc, r)
    for fov in (0.0, 360.0, 400.0, 180.0):
        assert np.array_equal(O.run(sc, _fov(r, fov)), v)
    # gaze along the normal, given explicitly or scaled, is the default axis
    assert np.array_equal(O.run(sc, _fov(r, 100.0, (0.0, 1.0, 0.0))), O.run(sc, _fov(r, 100.0)))
    assert np.array_equal(O.run(sc, _fov(r, 100.0, (0.0, 3.5, 0.0))), O.run(sc, _fov(r, 100.0)))


def test_fov_equals_cropped_target():
    """Seen from a point on the target's axis, a cone that takes exactly the
    K middle patches (its edge falls between patch directions) gives the
    value of a target cropped to those K patches, which has the same patch
    centres."""
    N, L = 32, 16 * U          # 32 patches of 0.5 m
    D = 20.0
    q = (0, int(D * U), 0)
    for K in (2, 8, 20, 30):
        # the half-angle between patch K/2 - 1/2 and K/2 + 1/2 half-widths off axis
        x_in, x_out = (K / 2 - 0.5) * 0.5, (K / 2 + 0.5) * 0.5
        half = 0.5 * (math.atan2(x_in, D) + math.atan2(x_out, D))
        full = single_viewpoint(req2((0, 0), width=L, pu=N), q)
        crop = single_viewpoint(req2((0, 0), width=K * L // N, pu=K), q)
        v_cone = O.run(scene(2, []), _fov(full, math.degrees(2 * half)))[0]
        v_crop = O.run(scene(2, []), crop)[0]
        assert v_cone == pytest.approx(v_crop, rel=1e-14)


def test_fov_monotone_and_mirror_symmetric():
    rng = np.random.default_rng(8)
    n = 40
    lo = rng.integers(-80 * U, 70 * U, size=(n, 3))
    lo[:, 1] = rng.integers(3 * U, 80 * U, size=n)
    lo[:, 2] = 0
    hi = lo + rng.integers(2 * U, 12 * U, size=(n, 3))
    sc = scene(3, list(zip(lo.tolist(), hi.tolist())))
    mlo, mhi = lo.copy(), hi.copy()
    mlo[:, 0], mhi[:, 0] = -hi[:, 0], -lo[:, 0]
    msc = scene(3, list(zip(mlo.tolist(), mhi.tolist())))
    nx, ny = 10, 6
    r = req3((0, 0, 20 * U), width=12 * U, height=6 * U, pu=6, pw=3, origin=(-nx * 8 * U, 4 * U),
             step=(16 * U, 16 * U), n=(nx, ny), layers=(2 * U, 25 * U))
    prev = None
    for fov in (20.0, 60.0, 120.0, 170.0, 180.0):
        v = O.run(sc, _fov(r, fov))
        if prev is not None:
            assert np.all(v >= prev)
        prev = v
    assert (prev > 0).sum() > (O.run(sc, _fov(r, 20.0)) > 0).sum()
    gaze = (0.4, 1.0, -0.3)
    v = O.run(sc, _fov(r, 90.0, gaze))
    mv = O.run(msc, _fov(r, 90.0, (-gaze[0], gaze[1], gaze[2])))
    for layer in range(2):
        for iy in range(ny):
            for ix in range(nx):
                i = (layer * ny + iy) * nx + ix
                j = (layer * ny + iy) * nx + (nx - 1 - ix)
                assert v[i] == pytest.approx(mv[j], rel=1e-13, abs=0)
    assert (v > 0).any()


def test_fov_region_of_the_paper_is_bounded_by_rays_from_the_target_ends():
    """With a 120 degree field of view the region from which the target is
    seen at all is bounded by rays from its two end points at 60 degrees
    from the normal (Section III-B).  Past the end T_B = (5, 0): a point at
    70 degrees from the normal, seen from T_B, sees nothing; at 50 degrees it
    sees the patches near T_B."""
    r = req2((0, 0), width=10 * U, pu=64)
    for ang, seen in ((70.0, False), (50.0, True)):
        d = 40.0
        q = (5.0 + d * math.sin(math.radians(ang)), d * math.cos(math.radians(ang)))
        rq = single_viewpoint(_fov(r, 120.0), (round(q[0] * U), round(q[1] * U), 0))
        v = O.run(scene(2, []), rq)[0]
        assert (v > 0) == seen
        # and no cone at all sees it either way
        assert O.run(scene(2, []), single_viewpoint(r, (round(q[0] * U), round(q[1] * U), 0)))[0] > 0


def test_fov_with_strict_mode_and_two_sided():
    """Strict with a cone: 0 as soon as any patch is blocked, else the sum
    over the patches in the cone; a two-sided cone is symmetric through the
    target plane."""
    sc = scene(3, [((-30 * U, 20 * U, 0), (-25 * U, 24 * U, 40 * U))])
    base = dict(width=12 * U, height=6 * U, pu=6, pw=3, origin=(-64 * U, -60 * U), step=(16 * U, 15 * U),
                n=(8, 9), layers=(5 * U,))
    part = O.run(sc, _fov(req3((0, 0, 20 * U), **base), 100.0))
    strict, bits = O.run(sc, _fov(req3((0, 0, 20 * U), flags=2 | 1, **base), 100.0), bits=True)
    for i in range(part.shape[0]):
        if bits[i].any():
            assert strict[i] == 0.0
        else:
            assert strict[i] == part[i]
    assert (strict > 0).any() and (bits.any(axis=1) & (part > 0)).any()
    two = O.run(scene(3, []), _fov(req3((0, 0, 20 * U), flags=FLAG_TWO_SIDED, **base), 100.0))
    nx, ny = 8, 9
    ys = [-60 * U + 15 * U * iy + 15 * U // 2 for iy in range(ny)]   # row y, units
    for iy in range(ny):
        for iy2 in range(ny):
            if ys[iy] == -ys[iy2] and ys[iy] != 0:
                for ix in range(nx):
                    assert two[iy * nx + ix] == two[iy2 * nx + ix]


def _angle_to_axis(r, a):
    """Angle between vectors r and a, by atan2 of the cross and dot products
    (an independent route to the cone test's cosine inequality)."""
    cx = r[1] * a[2] - r[2] * a[1]
    cy = r[2] * a[0] - r[0] * a[2]
    cz = r[0] * a[1] - r[1] * a[0]
    return math.atan2(math.sqrt(cx * cx + cy * cy + cz * cz), r[0] * a[0] + r[1] * a[1] + r[2] * a[2])


def test_fov_decision_is_the_angle_to_the_axis():
    """The oracle decides the cone in float64: q is in p's cone iff the angle
    between q - p and the gaze axis is at most half the field of view (for a
    two-sided target, the angle to the axis or to its opposite), and the
    margin it reports has the decision's sign."""
    rng = np.random.default_rng(41)
    base = req3((0, 0, 20 * U), pu=4, pw=2)
    checked = 0
    for _ in range(3000):
        fov = float(rng.uniform(5.0, 355.0))
        g = rng.normal(size=3)
        two = bool(rng.integers(0, 2))
        r = dict(_fov(base, fov, tuple(float(x) for x in g)), flags=FLAG_TWO_SIDED if two else 0)
        q = [int(x) for x in rng.integers(-60 * U, 60 * U, size=3)]
        p = [int(x) for x in rng.integers(-10 * U, 10 * U, size=3)]
        inside, margin = O.fov_test(r, q, p)
        gf = np.asarray(np.float32(g), np.float64)
        a = gf / np.linalg.norm(gf)
        rv = [(q[k] - p[k]) / U for k in range(3)]
        ang = _angle_to_axis(rv, a)
        if two:
            ang = min(ang, math.pi - ang)
        half = math.radians(fov) / 2.0
        if abs(ang - half) < 1e-9:
            continue
        assert inside == (ang <= half), (fov, g, q, p)
        assert (margin >= 0) == inside
        checked += 1
    assert checked > 2900
    assert O.fov_test(base, [0, 0, 0], [1, 1, 1]) == (None, 0.0)


def _f32_cone(q, p, fov, g, two_sided):
    """The float32 evaluation of the cone test that the request header
    defines (one rounding per operation, world order x, y, z)."""
    f = np.float32
    c = f(math.cos(fov * math.pi / 360.0))
    gd = [float(f(x)) for x in g]
    if not any(gd):
        gd = [0.0, 1.0, 0.0]   # the targets here face +y
    n = math.sqrt(sum(x * x for x in gd))
    a = [f(x / n) for x in gd]
    r = [f(f(q[k] / U) - f(p[k] / U)) for k in range(3)]
    d = f(f(f(a[0] * r[0]) + f(a[1] * r[1])) + f(a[2] * r[2]))
    if two_sided:
        d = abs(d)
    rr = f(f(f(r[0] * r[0]) + f(r[1] * r[1])) + f(r[2] * r[2]))
    return bool(d >= f(c * f(np.sqrt(rr))))


def test_fov_band_holds_every_pair_a_float32_evaluation_may_flip():
    """A float32 evaluation of the cone can differ from the float64 decision
    only within VO_FOV_BAND of the edge (the bound derived in the oracle's
    header); on exact ties at 45 degrees (r = (k, k, 0) against the +y axis
    with a 90 degree field of view) the band reports the pair, and the value
    a float32 cone gives lies in the bracket the band states."""
    rng = np.random.default_rng(43)
    base = req3((0, 0, 20 * U), pu=4, pw=2)
    flips = 0
    for _ in range(4000):
        fov = float(rng.choice([60.0, 90.0, 120.0, 150.0, 200.0]))
        g = (0.0, 1.0, 0.0) if rng.random() < 0.5 else tuple(float(x) for x in rng.normal(size=3))
        r = _fov(base, fov, g)
        k = int(rng.integers(1, 40 * U))
        # near-tie pairs: r close to 45 degrees off the +y axis, and random ones
        if rng.random() < 0.5:
            rv = [k + int(rng.integers(-2, 3)), k, int(rng.integers(-2, 3))]
        else:
            rv = [int(x) for x in rng.integers(-40 * U, 40 * U, size=3)]
        p = [int(x) for x in rng.integers(-10 * U, 10 * U, size=3)]
        q = [p[i] + rv[i] for i in range(3)]
        inside, margin = O.fov_test(r, q, p)
        if _f32_cone(q, p, fov, g, False) != inside:
            flips += 1
            assert abs(margin) <= 1e-6, (fov, g, q, p, margin)
    assert flips > 10   # the near ties do flip under float32
    # a 2D target seen from a point from which some patch directions are
    # exactly 45 degrees off the normal: the band reports them
    W, N = 16 * U, 32
    tgt = req2((0, 0), width=W, pu=N)
    pc = O.patch_centres(tgt)
    d = 20 * U
    q = (int(pc[5][0]) + d, d, 0)          # patch 5 at exactly 45 degrees
    r = _fov(single_viewpoint(tgt, q), 90.0)
    v, band = O.run(scene(2, []), r, band=True)
    assert band[0, 0] >= 1
    # the value with the float32 cone decisions is inside the bracket
    v32 = 0.0
    for j in range(N):
        p = pc[j]
        rx, ry = (q[0] - p[0]) / U, (q[1] - p[1]) / U
        if ry > 0 and _f32_cone(q, p, 90.0, (0.0, 0.0, 0.0), False):
            v32 += (W / U / N) * ry / (rx * rx + ry * ry)
    assert v[0] - band[0, 1] - 1e-12 <= v32 <= v[0] + band[0, 2] + 1e-12
    # no cone, or no pair near the edge: an empty band
    _, b0 = O.run(scene(2, []), single_viewpoint(tgt, q), band=True)
    assert not b0.any()


def test_blocking_is_convex_in_viewpoint_and_in_patch():
    """The one-box shortcuts rest on two convexity facts, checked here with
    the exact predicate: for a fixed patch point p, if a box blocks the
    segments from the four corners of a horizontal rectangle of viewpoints,
    it blocks those from every point of the rectangle; and for a fixed
    viewpoint, likewise for the corners of a vertical target rectangle."""
    rng = np.random.default_rng(31)
    tried = hit_v = hit_p = 0
    for _ in range(3000):
        lo = rng.integers(-40 * U, 30 * U, size=3)
        lo[2] = 0
        hi = lo + rng.integers(4 * U, 30 * U, size=3)
        # viewpoint rectangle (z = const) and a patch point p
        x0, y0 = rng.integers(-80 * U, 60 * U, size=2)
        x1, y1 = x0 + int(rng.integers(1, 20 * U)), y0 + int(rng.integers(1, 20 * U))
        z = int(rng.integers(0, 10 * U))
        p = [int(rng.integers(-10 * U, 10 * U)), int(rng.integers(40 * U, 60 * U)), int(rng.integers(20 * U, 40 * U))]
        corners = [[x, y, z] for x in (x0, x1) for y in (y0, y1)]
        tried += 1
        if all(O.segment_hits_box(3, q, p, lo, hi) for q in corners):
            hit_v += 1
            for _ in range(8):
                q = [int(rng.integers(x0, x1 + 1)), int(rng.integers(y0, y1 + 1)), z]
                assert O.segment_hits_box(3, q, p, lo, hi)
        # target rectangle (y = const) seen from a viewpoint q
        q = [int(rng.integers(-80 * U, 60 * U)), int(rng.integers(-80 * U, -50 * U)), int(rng.integers(0, 10 * U))]
        u0, w0 = int(rng.integers(-10 * U, 5 * U)), int(rng.integers(20 * U, 30 * U))
        u1, w1 = u0 + int(rng.integers(1, 10 * U)), w0 + int(rng.integers(1, 10 * U))
        yt = int(rng.integers(40 * U, 60 * U))
        pcs = [[u, yt, w] for u in (u0, u1) for w in (w0, w1)]
        if all(O.segment_hits_box(3, q, pp, lo, hi) for pp in pcs):
            hit_p += 1
            for _ in range(8):
                pp = [int(rng.integers(u0, u1 + 1)), yt, int(rng.integers(w0, w1 + 1))]
                assert O.segment_hits_box(3, q, pp, lo, hi)
    assert hit_v > 30 and hit_p > 30, (hit_v, hit_p)
