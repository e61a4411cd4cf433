"""The paper's own colouring of space into equi-visible cells (Section III-A,
"Distance Based Partition" and "Angle Based Partition"), as a comparison
workload for the dense GPU map: CPU only, 2D, no obstacles (the step before
the paper accounts for them).

* Distance partition: from the near point d_0, the head-on visual angle
  V_0 = 2 atan(S / 2 d_0) (Eq. 1) is lowered by the angular resolution mu at
  each step, and d_i is the distance at which the target subtends
  V_i = V_0 - i mu; it stops once V_i < mu (beyond that the target is not
  distinguishable).
* Angle partition: in the band <d_i, d_i+1> with mid distance d', the visual
  angle seen head-on is lowered by mu per step; S_j = 2 d' tan(V_j / 2) is the
  perceived size giving V_j, and the viewing angle alpha_j at which the
  target looks that large follows from Eq. 2 (perceived size S alpha / 90
  degrees).  The band's cells lie between successive alpha_j, from 90 degrees
  down; it stops once V_j < mu.
* A cell's colour is the visibility at its centre (Section III-A end), by the
  paper's own measure (Eq. 1 with the perceived size of Eq. 2), or by any
  other measure the caller passes.

`eq6_error` is the approximation error of Eq. 6 (Section V): the relative
difference of the area-weighted colour sums of an exact and an approximate
map.
"""

import math

import numpy as np


def distance_partition(S, mu_deg, d0):
    """Band edges d_0 < d_1 < ... (metres): the target of size S subtends
    V_0 - i mu at d_i, V_0 its visual angle at d_0."""
    mu = math.radians(mu_deg)
    v0 = 2.0 * math.atan(S / (2.0 * d0))
    edges = [d0]
    i = 1
    while v0 - i * mu >= mu:
        edges.append(S / (2.0 * math.tan((v0 - i * mu) / 2.0)))
        i += 1
    return np.asarray(edges)


def angle_partition(S, mu_deg, d_mid):
    """Viewing-angle edges (degrees, from 90 down) of one distance band with
    mid distance d_mid: the target seen at alpha_j looks S_j large (Eq. 2),
    with S_j the size that subtends V_j = V_0 - j mu at d_mid (Eq. 1)."""
    mu = math.radians(mu_deg)
    v0 = 2.0 * math.atan(S / (2.0 * d_mid))
    edges = [90.0]
    j = 1
    while v0 - j * mu >= mu:
        s_j = 2.0 * d_mid * math.tan((v0 - j * mu) / 2.0)
        edges.append(90.0 * s_j / S)
        j += 1
    edges.append(0.0)
    return np.asarray(edges)


def paper_visibility(S, D, alpha_deg):
    """Visual angle (radians) of a target of size S at distance D seen at
    viewing angle alpha: Eq. 1 with the perceived size S alpha / 90 of Eq. 2."""
    s = S * np.asarray(alpha_deg) / 90.0
    return 2.0 * np.arctan(s / (2.0 * np.asarray(D)))


class Partition:
    """Equi-visible cells of a 2D segment target of length S centred at the
    origin and facing +y, for angular resolution mu (degrees) and near point
    d0 (metres)."""

    def __init__(self, S, mu_deg, d0):
        self.S = float(S)
        self.d_edges = distance_partition(S, mu_deg, d0)
        mids = 0.5 * (self.d_edges[:-1] + self.d_edges[1:])
        self.a_edges = [angle_partition(S, mu_deg, m) for m in mids]

    def n_cells(self):
        return sum(len(a) - 1 for a in self.a_edges)

    def cell_of(self, x, y):
        """(band, angle cell) of the points (x, y) in front of the target;
        band = -1 outside the partitioned range (nearer than d_0, at or
        beyond the last edge, or not in front)."""
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        d = np.hypot(x, y)
        # viewing angle between the sight line and the target: 90 head-on
        alpha = np.degrees(np.arctan2(y, np.abs(x)))
        band = np.searchsorted(self.d_edges, d, side="right") - 1
        band[(band < 0) | (band >= len(self.d_edges) - 1) | (y <= 0)] = -1
        cell = np.full(d.shape, -1)
        for b in range(len(self.d_edges) - 1):
            sel = band == b
            if not sel.any():
                continue
            edges = self.a_edges[b]   # descending
            # index j with edges[j] >= alpha > edges[j + 1]
            j = np.searchsorted(-edges, -alpha[sel], side="left") - 1
            cell[sel] = np.clip(j, 0, len(edges) - 2)
        return band, cell

    def centres(self, band):
        """Centres (distance, viewing angles in degrees) of a band's cells."""
        d = 0.5 * (self.d_edges[band] + self.d_edges[band + 1])
        e = self.a_edges[band]
        return d, 0.5 * (e[:-1] + e[1:])

    def values_at(self, x, y, measure=None):
        """The partition's value at each point: that of its cell's centre by
        `measure(D, alpha_deg)` (the paper's Eq. 1 x Eq. 2 by default), 0
        outside the partitioned range."""
        if measure is None:
            def measure(D, a):
                return paper_visibility(self.S, D, a)
        band, cell = self.cell_of(x, y)
        out = np.zeros(band.shape)
        for b in range(len(self.d_edges) - 1):
            sel = band == b
            if sel.any():
                d, a = self.centres(b)
                out[sel] = measure(np.full(a.shape, d), a)[cell[sel]]
        return out


def quantise(v, levels, v_ref=None):
    """Colours of values v: 0 for v = 0, else 1 + min(L - 2, floor((L - 1) v / v_ref))."""
    v = np.asarray(v, np.float64)
    vref = float(v_ref) if v_ref else float(v.max()) if v.size else 0.0
    c = np.zeros(v.shape, np.int64)
    if vref > 0:
        nz = v > 0
        c[nz] = 1 + np.minimum(levels - 2, np.floor((levels - 1) * v[nz] / vref)).astype(np.int64)
    return c


def eq6_error(c_exact, c_approx, area=None):
    """Eq. 6: sum_i (c_e,i A_i - c_a,i A_i) / sum_i c_e,i A_i."""
    c_exact = np.asarray(c_exact, np.float64)
    c_approx = np.asarray(c_approx, np.float64)
    a = np.ones(c_exact.shape) if area is None else np.asarray(area, np.float64)
    den = float(np.sum(c_exact * a))
    return float(np.sum((c_exact - c_approx) * a)) / den if den > 0 else 0.0


def subtended(S, D, alpha_deg):
    """Angle (radians) subtended by a segment of length S centred at the
    origin along x, from the point at distance D and viewing angle alpha
    (degrees from the segment's line): the unobstructed limit of the dense
    map's measure, sum of len cos(theta) / d, as the samples get finer."""
    a = np.radians(np.asarray(alpha_deg, np.float64))
    D = np.asarray(D, np.float64)
    px, py = D * np.cos(a), D * np.sin(a)
    return np.abs(np.arctan2(py, px - S / 2.0) - np.arctan2(py, px + S / 2.0))
