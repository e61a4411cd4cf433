"""Seeded synthetic scenes and VCM requests (input generation only).

The paper measures on two city models (British Ordnance Survey, 5,985 objects;
Boston downtown, 130,043 objects; Section V-A) that are not available here.
These generators stand in for them with city-like box fields of the same
scale: uniform rectangles in 2D and Gaussian-mixture clusters of boxes with
lognormal heights in 3D.

Everything is returned on the input lattice: every coordinate is an integer
number of 2^-10 m units with magnitude at most 2^24 units (16,384 m), so that
the same numbers are exact in float32, float64 and int64.  This module draws
inputs only; it computes no viewpoint, patch, occlusion or visibility value.

Axis codes used in requests: 0 = +x, 1 = -x, 2 = +y, 3 = -y, 4 = +z, 5 = -z.
"""

import math

import numpy as np

from .prng import PCG32

LATTICE_PER_M = 1024  # lattice units per metre
COORD_LIMIT_UNITS = 1 << 24  # |coordinate| <= 2^24 units = 16,384 m

AXIS_PX, AXIS_NX, AXIS_PY, AXIS_NY, AXIS_PZ, AXIS_NZ = range(6)


def snap(x_m):
    """Nearest lattice point (in units) to a length in metres."""
    return int(math.floor(x_m * LATTICE_PER_M + 0.5))


def units_to_m(u):
    return np.asarray(u, dtype=np.float64) / LATTICE_PER_M


class Scene:
    """Axis-aligned obstacle boxes in lattice units.

    ``lo`` and ``hi`` are int64 arrays of shape (n, 3); 2D scenes keep z = 0.
    """

    def __init__(self, dims, lo, hi, name=""):
        self.dims = int(dims)
        self.lo = np.ascontiguousarray(lo, dtype=np.int64).reshape(-1, 3)
        self.hi = np.ascontiguousarray(hi, dtype=np.int64).reshape(-1, 3)
        self.name = name
        if self.lo.shape != self.hi.shape:
            raise ValueError("lo/hi shape mismatch")

    @property
    def n(self):
        return self.lo.shape[0]

    def lo_f32(self):
        return (self.lo.astype(np.float64) / LATTICE_PER_M).astype(np.float32)

    def hi_f32(self):
        return (self.hi.astype(np.float64) / LATTICE_PER_M).astype(np.float32)

    def subset(self, idx):
        return Scene(self.dims, self.lo[idx], self.hi[idx], self.name)

    def with_boxes(self, lo, hi):
        lo = np.concatenate([self.lo, np.asarray(lo, np.int64).reshape(-1, 3)])
        hi = np.concatenate([self.hi, np.asarray(hi, np.int64).reshape(-1, 3)])
        return Scene(self.dims, lo, hi, self.name)

    def digest(self):
        import hashlib

        h = hashlib.sha256()
        h.update(self.lo.tobytes())
        h.update(self.hi.tobytes())
        return h.hexdigest()[:16]


def make_request(dims, center_m, axis_u, normal, width_m, patches_u, grid_origin_m,
                 grid_step_m, grid_n, layers_m=(0.0,), axis_w=AXIS_PZ, height_m=0.0,
                 patches_w=1, color_levels=16, v_ref=0.0, flags=0):
    """Build a request dict with every length snapped to the lattice."""
    req = {
        "dims": int(dims),
        "center": [snap(c) for c in center_m] + [0] * (3 - len(center_m)),
        "axis_u": int(axis_u),
        "axis_w": int(axis_w) if dims == 3 else int(AXIS_PZ),
        "normal": int(normal),
        "width": snap(width_m),
        "height": snap(height_m) if dims == 3 else 0,
        "patches_u": int(patches_u),
        "patches_w": int(patches_w) if dims == 3 else 1,
        "grid_origin": [snap(grid_origin_m[0]), snap(grid_origin_m[1])],
        "grid_step": [snap(grid_step_m[0]), snap(grid_step_m[1])],
        "grid_nx": int(grid_n[0]),
        "grid_ny": int(grid_n[1]),
        "layer_z": [snap(z) for z in layers_m] if dims == 3 else [0],
        "color_levels": int(color_levels),
        "v_ref": float(v_ref),
        "flags": int(flags),
    }
    return req


def n_viewpoints(req):
    return req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])


def n_patches(req):
    return req["patches_u"] * req["patches_w"]


def n_segments(req):
    return n_viewpoints(req) * n_patches(req)


def _target_aabb_units(req, inflate_m):
    """Axis-aligned extent of a target rectangle, inflated (units)."""
    c = np.array(req["center"], dtype=np.int64)
    lo = c.copy()
    hi = c.copy()
    half = {req["axis_u"] >> 1: req["width"] // 2 + 1}
    if req["dims"] == 3:
        half[req["axis_w"] >> 1] = req["height"] // 2 + 1
    for ax, h in half.items():
        lo[ax] -= h
        hi[ax] += h
    inf = snap(inflate_m)
    lo -= inf
    hi += inf
    if req["dims"] == 2:
        lo[2] = hi[2] = 0
    return lo, hi


def _overlaps(lo_a, hi_a, lo_b, hi_b, dims):
    return all(lo_a[k] <= hi_b[k] and lo_b[k] <= hi_a[k] for k in range(dims))


# ---------------------------------------------------------------------------
# 2D: uniform rectangles around a segment target
# ---------------------------------------------------------------------------

def scene_2d_uniform(seed, n_rects, half_m, side_m, keep_out_lo, keep_out_hi):
    rng = PCG32(seed, stream=1)
    lo, hi = [], []
    while len(lo) < n_rects:
        cx = rng.uniform(-half_m, half_m)
        cy = rng.uniform(-half_m, half_m)
        sx = rng.uniform(*side_m)
        sy = rng.uniform(*side_m)
        blo = [snap(cx - sx / 2), snap(cy - sy / 2), 0]
        bhi = [snap(cx + sx / 2), snap(cy + sy / 2), 0]
        if _overlaps(blo, bhi, keep_out_lo, keep_out_hi, 2):
            continue
        lo.append(blo)
        hi.append(bhi)
    return Scene(2, lo, hi, name="2d-uniform")


# ---------------------------------------------------------------------------
# 3D: Gaussian-mixture city with lognormal heights
# ---------------------------------------------------------------------------

def scene_3d_mixture(seed, n_boxes, half_m, n_components, sigma_m, foot_m=(10.0, 60.0),
                     height_median_m=20.0, height_sigma=0.6, keep_out=None):
    """Boxes with footprint sides uniform in ``foot_m``, base z = 0, heights
    lognormal(ln median, sigma), centres drawn from an equal-weight isotropic
    Gaussian mixture whose means are uniform over the square scene.  Boxes
    whose footprint leaves the scene, or that touch ``keep_out`` (an inflated
    target extent, (lo, hi) in units), are redrawn."""
    rng = PCG32(seed, stream=2)
    comps = [(rng.uniform(-half_m, half_m), rng.uniform(-half_m, half_m), rng.uniform(*sigma_m))
             for _ in range(n_components)]
    lim = snap(half_m)
    lo = np.empty((n_boxes, 3), np.int64)
    hi = np.empty((n_boxes, 3), np.int64)
    i = 0
    while i < n_boxes:
        mx, my, s = comps[rng.randint(0, n_components - 1)]
        cx = rng.normal(mx, s)
        cy = rng.normal(my, s)
        sx = rng.uniform(*foot_m)
        sy = rng.uniform(*foot_m)
        h = math.exp(math.log(height_median_m) + height_sigma * rng.normal())
        blo = (snap(cx - sx / 2), snap(cy - sy / 2), 0)
        bhi = (snap(cx + sx / 2), snap(cy + sy / 2), max(1, snap(h)))
        if blo[0] < -lim or blo[1] < -lim or bhi[0] > lim or bhi[1] > lim:
            continue
        if keep_out is not None and _overlaps(blo, bhi, keep_out[0], keep_out[1], 3):
            continue
        lo[i] = blo
        hi[i] = bhi
        i += 1
    return Scene(3, lo, hi, name="3d-mixture")


def layers_from(first_m, spacing_m, count):
    return [first_m + spacing_m * k for k in range(count)]


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def workload_2d(seed=1, grid=128, samples=64, n_rects=100):
    """2D plain VCM: a 10 m segment at the centre of a 1 km x 1 km plane,
    uniform rectangles with sides 5-30 m, grid x grid viewpoint cells."""
    req = make_request(2, (0.0, 0.0), AXIS_PX, AXIS_PY, 10.0, samples,
                       (-500.0, -500.0), (1000.0 / grid, 1000.0 / grid), (grid, grid),
                       color_levels=8)
    ko_lo, ko_hi = _target_aabb_units(req, 1.0)
    scene = scene_2d_uniform(seed, n_rects, 500.0, (5.0, 30.0), ko_lo, ko_hi)
    return scene, req


def workload_3d(seed=2, grid=512, layers=5, patches=(32, 16), n_boxes=5000, half_m=1000.0,
                n_components=16, sigma_m=(50.0, 250.0), target_m=(20.0, 10.0),
                target_center_z=30.0, levels=16):
    """3D plain VCM: a vertical W x H target facing +y at the scene centre,
    mixture-clustered boxes, grid x grid viewpoints x layers at 1.7 m + 10 m k."""
    step = 2.0 * half_m / grid
    req = make_request(3, (0.0, 0.0, target_center_z), AXIS_PX, AXIS_PY, target_m[0],
                       patches[0], (-half_m, -half_m), (step, step), (grid, grid),
                       layers_m=layers_from(1.7, 10.0, layers), axis_w=AXIS_PZ,
                       height_m=target_m[1], patches_w=patches[1], color_levels=levels)
    ko = _target_aabb_units(req, 1.0)
    scene = scene_3d_mixture(seed, n_boxes, half_m, n_components, sigma_m, keep_out=ko)
    return scene, req


def workload_3d_large(seed=3, grid=2048, layers=8):
    """3D large scene: 100,000 boxes over 10 km x 10 km, 64-component mixture,
    one 40 m x 20 m target split 64 x 32, grid x grid x layers viewpoints."""
    return workload_3d(seed=seed, grid=grid, layers=layers, patches=(64, 32), n_boxes=100000,
                       half_m=5000.0, n_components=64, sigma_m=(100.0, 600.0),
                       target_m=(40.0, 20.0))


def _random_target_request(rng, scene, half_m, min_side=6, max_side=10, patch_choices=None):
    if patch_choices is None:
        patch_choices = [(8, 4), (16, 8), (32, 16), (64, 32)]
    normals = [AXIS_PX, AXIS_NX, AXIS_PY, AXIS_NY]
    while True:
        w = rng.uniform(2.0, 50.0)
        h = w / 2.0
        cz = rng.uniform(10.0, 60.0)
        nrm = normals[rng.randint(0, 3)]
        cx = rng.uniform(-half_m + 100.0, half_m - 100.0)
        cy = rng.uniform(-half_m + 100.0, half_m - 100.0)
        # the in-plane horizontal axis is the other horizontal axis
        axis_u = AXIS_PY if (nrm >> 1) == 0 else AXIS_PX
        n_side = int(round(2.0 ** rng.uniform(min_side, max_side)))
        n_layers = rng.randint(1, 8)
        pu, pw = patch_choices[rng.randint(0, len(patch_choices) - 1)]
        step = 2000.0 / n_side
        step_u = max(1, snap(step))
        side_units = step_u * n_side
        ox = min(max(snap(cx) - side_units // 2, -snap(half_m)), snap(half_m) - side_units)
        oy = min(max(snap(cy) - side_units // 2, -snap(half_m)), snap(half_m) - side_units)
        req = make_request(3, (cx, cy, cz), axis_u, nrm, w, pu, (ox / LATTICE_PER_M, oy / LATTICE_PER_M),
                           (step_u / LATTICE_PER_M, step_u / LATTICE_PER_M), (n_side, n_side),
                           layers_m=layers_from(1.7, 10.0, n_layers), axis_w=AXIS_PZ,
                           height_m=h, patches_w=pw, color_levels=16)
        ko_lo, ko_hi = _target_aabb_units(req, 1.0)
        hit = np.all((scene.lo <= ko_hi[None, :]) & (ko_lo[None, :] <= scene.hi), axis=1)
        if not hit.any():
            return req


def workload_batched(seed=4, n_requests=256, n_boxes=50000, min_side=6, max_side=10,
                     patch_choices=None):
    """Batched uneven VCMs: a shared mixture scene over 10 km x 10 km and
    ``n_requests`` targets with widths 2-50 m (height = width / 2), centre
    heights 10-60 m, normals in {+-x, +-y}, 2 km viewpoint squares with
    log-uniform sides 2^6..2^10 cells, 1-8 layers and 8x4..64x32 patches."""
    scene = scene_3d_mixture(seed, n_boxes, 5000.0, 64, (100.0, 600.0))
    rng = PCG32(seed, stream=3)
    reqs = [_random_target_request(rng, scene, 5000.0, min_side, max_side, patch_choices)
            for _ in range(n_requests)]
    return scene, reqs


def poisson_arrivals(seed, rate_per_s, count):
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = PCG32(seed, stream=4)
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(rate_per_s)
        out.append(t)
    return out


def serving_requests(scene, seed=5, count=64, min_side=6, max_side=10, patch_choices=None):
    """Requests drawn from the batched mix, placed against ``scene``."""
    rng = PCG32(seed, stream=5)
    return [_random_target_request(rng, scene, 5000.0, min_side, max_side, patch_choices)
            for _ in range(count)]
