"""Exact brute force for tiny scenes, by a route independent of the oracle.

The oracle decides a segment/box hit by intersecting parametric slab
intervals.  Here the same question is answered with the separating-axis test
for a segment against an axis-aligned box (the box's three face normals and
the cross products of the segment direction with the box's edge directions;
Ericson, "Real-Time Collision Detection", 2005, Section 5.3.3), in exact
integers: every quantity is doubled so that midpoints and half-extents stay
integral.  Two closed convex sets that no candidate axis separates strictly
intersect, so touching counts as a hit, as the shadow definition requires
(Def. 4, Section III-B).

Patch centres and viewpoints are rebuilt from their definitions with
``fractions.Fraction`` (cell centres rounded to the 2^-10 m lattice, halves
away from zero).
"""

from fractions import Fraction


def round_half_away(x):
    x = Fraction(x)
    if x >= 0:
        return int((x + Fraction(1, 2)).__floor__())
    return -int((-x + Fraction(1, 2)).__floor__())


def _axis(code):
    return code >> 1, (-1 if code & 1 else 1)


def patch_centres(req):
    au, su = _axis(req["axis_u"])
    aw, sw = _axis(req["axis_w"])
    Nu, Nw = req["patches_u"], (req["patches_w"] if req["dims"] == 3 else 1)
    out = []
    for iw in range(Nw):
        for iu in range(Nu):
            p = list(req["center"][:3])
            if req["dims"] == 2:
                p[2] = 0
            off_u = (Fraction(2 * iu + 1, 2 * Nu) - Fraction(1, 2)) * req["width"]
            p[au] = round_half_away(req["center"][au] + su * off_u)
            if req["dims"] == 3:
                off_w = (Fraction(2 * iw + 1, 2 * Nw) - Fraction(1, 2)) * req["height"]
                p[aw] = round_half_away(req["center"][aw] + sw * off_w)
            out.append(tuple(p))
    return out


def viewpoint(req, index):
    nx, ny = req["grid_nx"], req["grid_ny"]
    ix, iy, layer = index % nx, (index // nx) % ny, index // (nx * ny)
    x = round_half_away(req["grid_origin"][0] + (ix + Fraction(1, 2)) * req["grid_step"][0])
    y = round_half_away(req["grid_origin"][1] + (iy + Fraction(1, 2)) * req["grid_step"][1])
    z = req["layer_z"][layer] if req["dims"] == 3 else 0
    return (x, y, z)


def segment_hits_box_sat(dims, q, p, lo, hi):
    """Exact separating-axis test; True iff the closed segment meets the box."""
    M = [q[k] + p[k] for k in range(dims)]     # 2 x midpoint
    H = [p[k] - q[k] for k in range(dims)]     # 2 x half-vector
    C = [lo[k] + hi[k] for k in range(dims)]   # 2 x box centre
    E = [hi[k] - lo[k] for k in range(dims)]   # 2 x half-extent
    D = [M[k] - C[k] for k in range(dims)]
    for k in range(dims):
        if abs(D[k]) > E[k] + abs(H[k]):
            return False
    if dims == 2:
        N = (-H[1], H[0])
        if abs(D[0] * N[0] + D[1] * N[1]) > E[0] * abs(N[0]) + E[1] * abs(N[1]):
            return False
        return True
    for k in range(3):
        # axis L = e_k x H
        e = [0, 0, 0]
        e[k] = 1
        L = (e[1] * H[2] - e[2] * H[1], e[2] * H[0] - e[0] * H[2], e[0] * H[1] - e[1] * H[0])
        if L == (0, 0, 0):
            continue
        lhs = abs(D[0] * L[0] + D[1] * L[1] + D[2] * L[2])
        rhs = E[0] * abs(L[0]) + E[1] * abs(L[1]) + E[2] * abs(L[2])
        if lhs > rhs:
            return False
    return True


def bits(scene, req, index):
    """Occlusion bits of one viewpoint as a list of 0/1 per patch."""
    q = viewpoint(req, index)
    out = []
    for p in patch_centres(req):
        hit = 0
        for b in range(scene.n):
            if segment_hits_box_sat(scene.dims, q, p, scene.lo[b], scene.hi[b]):
                hit = 1
                break
        out.append(hit)
    return out


def pack_bits(bitlist):
    words = [0] * ((len(bitlist) + 31) // 32)
    for j, b in enumerate(bitlist):
        if b:
            words[j >> 5] |= 1 << (j & 31)
    return words
