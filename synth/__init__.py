"""Seeded synthetic inputs (scenes, requests, arrival times) shared by the
oracle-side tests and the GPU path.  Input generation only: no visibility
arithmetic lives here."""

from .prng import PCG32, splitmix64  # noqa: F401
from .scenes import (  # noqa: F401
    AXIS_NX, AXIS_NY, AXIS_NZ, AXIS_PX, AXIS_PY, AXIS_PZ, COORD_LIMIT_UNITS, LATTICE_PER_M,
    Scene, layers_from, make_request, n_patches, n_segments, n_viewpoints, poisson_arrivals,
    scene_2d_uniform, scene_3d_mixture, serving_requests, snap, units_to_m, workload_2d,
    workload_3d, workload_3d_large, workload_batched,
)
