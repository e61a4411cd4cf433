"""GB300-native visibility color maps (target-centric VCM, Def. 1 of
"Scalable Visibility Color Map Construction in Spatial Databases").

The compute path is libvcm.so (hand-written sm_103a CUDA behind the C ABI in
include/vcm.h); ``vcm`` is its thin ctypes binding.  Build it with
``paper_1310_7297_gb300.build.build()``.
"""

from .vcm import (  # noqa: F401
    VCM_CACHE_BITS, VCM_DEVERR_BOUNDS, VCM_DEVERR_NONE, VCM_DEVERR_SPILL_WAIT, VCM_EMIT_BITS, VCM_FORM_ONE_TILE,
    VCM_FORM_PERSISTENT, VCM_FORM_RECOLOR, VCM_INJECT_ALLOC_FAIL, VCM_INJECT_NONE, VCM_INJECT_SPILL_BUSY, VCM_STRICT,
    VCM_TWO_SIDED, VCM_VIEWER, Context, VcmError, lib, make_request, n_viewpoints, stats_from_tensor, words,
)
