"""Python binding of libvcm (include/vcm.h): ctypes marshalling only.

Every step of the visibility color map runs inside libvcm's CUDA kernels;
this module converts arguments and raises ``VcmError`` on a non-OK status.
PyTorch supplies device memory and streams for the direct device path
(``vcm_compute``).  There is no CPU fallback: if the shared library is
missing, importing it raises.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvcm.so")
# the same library with the kernels' bounds checks compiled in (VCM_CHECKED)
CHECKED_LIB_PATH = os.path.join(_HERE, "_build", "libvcm_checked.so")

VCM_OK, VCM_PENDING = 0, 1
VCM_E_ARG, VCM_E_IO, VCM_E_NOMEM, VCM_E_CUDA = -1, -2, -3, -4
VCM_E_TIMEOUT, VCM_E_CANCELLED, VCM_E_STATE = -5, -6, -7
VCM_EMIT_BITS, VCM_STRICT, VCM_VIEWER, VCM_TWO_SIDED, VCM_CACHE_BITS = 1, 2, 4, 8, 16
VCM_DEVERR_NONE, VCM_DEVERR_BOUNDS, VCM_DEVERR_SPILL_WAIT = 0, 1, 2
VCM_FORM_PERSISTENT, VCM_FORM_ONE_TILE, VCM_FORM_RECOLOR = 0, 1, 2
VCM_INJECT_NONE, VCM_INJECT_SPILL_BUSY, VCM_INJECT_ALLOC_FAIL = 0, 1, 2
STATUS_NAMES = {0: "VCM_OK", 1: "VCM_PENDING", -1: "VCM_E_ARG", -2: "VCM_E_IO", -3: "VCM_E_NOMEM",
                -4: "VCM_E_CUDA", -5: "VCM_E_TIMEOUT", -6: "VCM_E_CANCELLED", -7: "VCM_E_STATE"}
UNITS_PER_M = 1024

# every symbol declared in include/vcm.h
EXPORTS = ["vcm_ctx_create", "vcm_ctx_destroy", "vcm_last_error", "vcm_scene_load_mem", "vcm_scene_load",
           "vcm_scene_save", "vcm_build", "vcm_compute", "vcm_submit", "vcm_submit_batch", "vcm_poll",
           "vcm_result_get", "vcm_result_release", "vcm_cancel", "vcm_set_slots", "vcm_compute_batch",
           "vcm_autotune", "vcm_set_tune", "vcm_get_tune", "vcm_set_timing_events", "vcm_compute_static",
           "vcm_recolor", "vcm_get_memory", "vcm_inject", "vcm_cache_clear", "vcm_set_request_log",
           "vcm_latency_summary"]


class _DeviceArray:
    """A device buffer described by __cuda_array_interface__ (version 3)."""

    def __init__(self, addr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (addr, False),
                                         "version": 3, "strides": None, "stream": None}


class VcmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class vcm_request(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32), ("center", ctypes.c_float * 3), ("axis_u", ctypes.c_int32),
                ("axis_w", ctypes.c_int32), ("normal", ctypes.c_int32), ("width", ctypes.c_float),
                ("height", ctypes.c_float), ("patches_u", ctypes.c_uint32), ("patches_w", ctypes.c_uint32),
                ("grid_origin", ctypes.c_float * 2), ("grid_step", ctypes.c_float * 2),
                ("grid_nx", ctypes.c_uint32), ("grid_ny", ctypes.c_uint32), ("n_layers", ctypes.c_uint32),
                ("layer_z", ctypes.POINTER(ctypes.c_float)), ("color_levels", ctypes.c_uint32),
                ("v_ref", ctypes.c_float), ("flags", ctypes.c_uint32), ("fov_deg", ctypes.c_float),
                ("gaze", ctypes.c_float * 3)]


class vcm_stats(ctypes.Structure):
    _fields_ = [("v_ref", ctypes.c_float), ("vmax_bits", ctypes.c_uint32), ("edge_cells", ctypes.c_uint32),
                ("error", ctypes.c_uint32), ("slab_tests", ctypes.c_ulonglong),
                ("rechecked", ctypes.c_ulonglong), ("segments", ctypes.c_ulonglong),
                ("boxes_listed", ctypes.c_ulonglong), ("corner_tests", ctypes.c_ulonglong),
                ("shortcut_viewpoints", ctypes.c_ulonglong), ("shared_viewpoints", ctypes.c_ulonglong)]


class vcm_result(ctypes.Structure):
    _fields_ = [("v", ctypes.POINTER(ctypes.c_float)), ("color", ctypes.POINTER(ctypes.c_uint8)),
                ("bits", ctypes.POINTER(ctypes.c_uint32)), ("d_v", ctypes.c_void_p),
                ("d_color", ctypes.c_void_p), ("d_bits", ctypes.c_void_p), ("n_viewpoints", ctypes.c_uint64),
                ("words_per_viewpoint", ctypes.c_uint32), ("stats", vcm_stats), ("latency_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("device_ms", ctypes.c_double), ("group_size", ctypes.c_uint32),
                ("launch_form", ctypes.c_uint32), ("launch_ms", ctypes.c_double),
                ("chain_ms", ctypes.c_double)]


class vcm_memory(ctypes.Structure):
    _fields_ = [("budget", ctypes.c_uint64), ("results", ctypes.c_uint64), ("slot_scratch", ctypes.c_uint64),
                ("slot_scratch_need", ctypes.c_uint64), ("cached_bits", ctypes.c_uint64),
                ("cache_entries", ctypes.c_uint32)]


class vcm_tune(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_uint32), ("tile_y", ctypes.c_uint32), ("patch_k", ctypes.c_uint32),
                ("box_cap", ctypes.c_uint32)]


STATS_BYTES = ctypes.sizeof(vcm_stats)

_lib = None
_lib_checked = None


def lib(checked=False):
    """The loaded libvcm.so (or libvcm_checked.so); raises if it has not
    been built."""
    global _lib, _lib_checked
    if checked:
        if _lib_checked is None:
            _lib_checked = _load(CHECKED_LIB_PATH)
        return _lib_checked
    if _lib is None:
        _lib = _load(LIB_PATH)
    return _lib


def _load(path):
    if not os.path.exists(path):
        raise RuntimeError("%s is not built; run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    P, VP, S = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int
    L.vcm_ctx_create.argtypes = [ctypes.c_int, ctypes.c_size_t, P(VP)]
    L.vcm_ctx_destroy.argtypes = [VP]
    L.vcm_ctx_destroy.restype = None
    L.vcm_last_error.argtypes = [VP]
    L.vcm_last_error.restype = ctypes.c_char_p
    L.vcm_scene_load_mem.argtypes = [VP, P(ctypes.c_float), P(ctypes.c_float), ctypes.c_uint32, ctypes.c_int32]
    L.vcm_scene_load.argtypes = [VP, ctypes.c_char_p]
    L.vcm_scene_save.argtypes = [VP, ctypes.c_char_p]
    L.vcm_build.argtypes = [VP, ctypes.c_float]
    L.vcm_compute.argtypes = [VP, P(vcm_request), VP, VP, VP, VP, VP]
    L.vcm_recolor.argtypes = [VP, P(vcm_request), VP, VP, VP, VP, VP]
    L.vcm_compute_batch.argtypes = [VP, P(vcm_request), ctypes.c_uint32, P(VP), P(VP), P(VP), VP, VP]
    L.vcm_submit.argtypes = [VP, P(vcm_request), P(ctypes.c_uint64)]
    L.vcm_submit_batch.argtypes = [VP, P(vcm_request), ctypes.c_uint32, P(ctypes.c_uint64)]
    L.vcm_poll.argtypes = [VP, ctypes.c_uint64, ctypes.c_int32]
    L.vcm_result_get.argtypes = [VP, ctypes.c_uint64, P(vcm_result)]
    L.vcm_result_release.argtypes = [VP, ctypes.c_uint64]
    L.vcm_cancel.argtypes = [VP, ctypes.c_uint64]
    L.vcm_set_slots.argtypes = [VP, ctypes.c_uint32, ctypes.c_uint32]
    L.vcm_autotune.argtypes = [VP, P(vcm_request), ctypes.c_uint32, P(vcm_tune)]
    L.vcm_set_tune.argtypes = [VP, P(vcm_tune)]
    L.vcm_get_tune.argtypes = [VP, P(vcm_request), P(vcm_tune)]
    L.vcm_set_timing_events.argtypes = [VP, VP, VP]
    L.vcm_compute_static.argtypes = [P(ctypes.c_float), P(ctypes.c_float), ctypes.c_uint32, ctypes.c_int32,
                                     P(vcm_request), VP, VP, VP, VP, VP]
    L.vcm_get_memory.argtypes = [VP, P(vcm_memory)]
    L.vcm_inject.argtypes = [VP, ctypes.c_uint32, ctypes.c_uint32]
    L.vcm_cache_clear.argtypes = [VP]
    for name in EXPORTS:
        if name not in ("vcm_ctx_destroy", "vcm_last_error"):
            getattr(L, name).restype = S
    return L


def _check(status, ctx=None, L=None):
    if status != VCM_OK:
        raise VcmError(status, (L or lib()).vcm_last_error(ctx).decode(errors="replace"))
    return status


def make_request(d):
    """vcm_request from a request dict in lattice units (as made by ``synth``).
    Returns (struct, keepalive) - keep the second alive while the struct is used."""
    r = vcm_request()
    u = float(UNITS_PER_M)
    r.dims = d["dims"]
    for k in range(3):
        r.center[k] = d["center"][k] / u
    r.axis_u, r.axis_w, r.normal = d["axis_u"], d["axis_w"], d["normal"]
    r.width, r.height = d["width"] / u, d["height"] / u
    r.patches_u, r.patches_w = d["patches_u"], d["patches_w"]
    for k in range(2):
        r.grid_origin[k] = d["grid_origin"][k] / u
        r.grid_step[k] = d["grid_step"][k] / u
    r.grid_nx, r.grid_ny = d["grid_nx"], d["grid_ny"]
    z = np.ascontiguousarray(np.asarray(d["layer_z"], np.float64) / u, dtype=np.float32)
    r.n_layers = len(z)
    r.layer_z = z.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    r.color_levels = d["color_levels"]
    r.v_ref = d.get("v_ref", 0.0)
    r.flags = d.get("flags", 0)
    r.fov_deg = d.get("fov_deg", 0.0)
    g = d.get("gaze", (0.0, 0.0, 0.0))
    for k in range(3):
        r.gaze[k] = g[k]
    return r, z


def n_viewpoints(d):
    return d["grid_nx"] * d["grid_ny"] * (len(d["layer_z"]) if d["dims"] == 3 else 1)


def words(d):
    if d.get("flags", 0) & VCM_VIEWER:
        return 1   # one bit per cell
    return (d["patches_u"] * (d["patches_w"] if d["dims"] == 3 else 1) + 31) // 32


class Context:
    """Owns one vcm_ctx; methods mirror the C entry points."""

    def __init__(self, device=0, mem_budget_bytes=0, checked=False):
        """checked: use libvcm_checked.so, whose kernels check their indices
        (a failed check sets vcm_stats.error to VCM_DEVERR_BOUNDS)."""
        self.L = lib(checked)
        h = ctypes.c_void_p()
        _check(self.L.vcm_ctx_create(device, mem_budget_bytes, ctypes.byref(h)), None, self.L)
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            self.L.vcm_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, status):
        return _check(status, self.h, self.L)

    # scene ------------------------------------------------------------------
    def vcm_scene_load_mem(self, lo, hi, dims):
        lo = np.ascontiguousarray(lo, dtype=np.float32)[:, :dims].copy()
        hi = np.ascontiguousarray(hi, dtype=np.float32)[:, :dims].copy()
        fp = ctypes.POINTER(ctypes.c_float)
        return self._ck(self.L.vcm_scene_load_mem(self.h, lo.ctypes.data_as(fp), hi.ctypes.data_as(fp),
                                                  lo.shape[0], dims))

    def load_scene(self, scene):
        """Upload a ``synth.Scene`` (lattice units)."""
        return self.vcm_scene_load_mem(scene.lo_f32(), scene.hi_f32(), scene.dims)

    def vcm_scene_load(self, path):
        return self._ck(self.L.vcm_scene_load(self.h, path.encode()))

    def vcm_scene_save(self, path):
        return self._ck(self.L.vcm_scene_save(self.h, path.encode()))

    def vcm_build(self, grid_cell_m=0.0):
        return self._ck(self.L.vcm_build(self.h, float(grid_cell_m)))

    # direct device path -----------------------------------------------------
    def vcm_compute(self, req, d_v, d_color, d_bits, d_stats, stream):
        r, keep = make_request(req)
        st = self.L.vcm_compute(self.h, ctypes.byref(r), d_v, d_color, d_bits, d_stats, stream)
        del keep
        return self._ck(st)

    def vcm_compute_batch(self, reqs, d_v, d_color, d_bits, d_stats, stream):
        n = len(reqs)
        arr = (vcm_request * n)()
        keep = []
        for i, d in enumerate(reqs):
            r, z = make_request(d)
            arr[i] = r
            keep.append(z)
        VPA = ctypes.c_void_p * n
        st = self.L.vcm_compute_batch(self.h, arr, n, VPA(*d_v), VPA(*d_color), VPA(*d_bits), d_stats, stream)
        return self._ck(st)

    def compute(self, req, emit_bits=False, stream=None):
        """Run one request on the current torch stream into new torch tensors.
        Returns (v, color, bits or None, stats) as device tensors (stats as a
        uint8 tensor of one vcm_stats)."""
        import torch

        dev = torch.device("cuda", self.device)
        n = n_viewpoints(req)
        req = dict(req)
        if emit_bits:
            req["flags"] = req.get("flags", 0) | VCM_EMIT_BITS
        v = torch.empty(n, dtype=torch.float32, device=dev)
        c = torch.empty(n, dtype=torch.uint8, device=dev)
        b = torch.empty(n * words(req), dtype=torch.int32, device=dev) if emit_bits else None
        s = torch.empty(STATS_BYTES, dtype=torch.uint8, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.vcm_compute(req, v.data_ptr(), c.data_ptr(), b.data_ptr() if b is not None else None,
                         s.data_ptr(), stream.cuda_stream)
        return v, c, b, s

    def vcm_recolor(self, req, d_bits, d_v, d_color, d_stats, stream):
        r, keep = make_request(req)
        st = self.L.vcm_recolor(self.h, ctypes.byref(r), d_bits, d_v, d_color, d_stats, stream)
        return self._ck(st)

    def recolor(self, req, bits, stream=None):
        """Values and colors of `req` from occlusion bits made earlier (a
        device tensor from compute(..., emit_bits=True) of the same target
        and grid), on the current torch stream.  Returns (v, color, stats)."""
        import torch

        dev = torch.device("cuda", self.device)
        n = n_viewpoints(req)
        v = torch.empty(n, dtype=torch.float32, device=dev)
        c = torch.empty(n, dtype=torch.uint8, device=dev)
        s = torch.empty(STATS_BYTES, dtype=torch.uint8, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.vcm_recolor(req, bits.data_ptr(), v.data_ptr(), c.data_ptr(), s.data_ptr(), stream.cuda_stream)
        return v, c, s

    # asynchronous requests ---------------------------------------------------
    def vcm_submit(self, req):
        r, keep = make_request(req)
        t = ctypes.c_uint64()
        self._ck(self.L.vcm_submit(self.h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def vcm_submit_batch(self, reqs):
        n = len(reqs)
        arr = (vcm_request * n)()
        keep = []
        for i, d in enumerate(reqs):
            r, z = make_request(d)
            arr[i] = r
            keep.append(z)
        ts = (ctypes.c_uint64 * n)()
        self._ck(self.L.vcm_submit_batch(self.h, arr, n, ts))
        return list(ts)

    def vcm_poll(self, ticket, wait_ms=-1):
        st = self.L.vcm_poll(self.h, ticket, wait_ms)
        if st == VCM_PENDING:
            return VCM_PENDING
        return self._ck(st)

    def vcm_result_get(self, ticket, copy=True):
        """Result as numpy arrays (copies unless copy=False) and a stats dict."""
        res = vcm_result()
        self._ck(self.L.vcm_result_get(self.h, ticket, ctypes.byref(res)))
        n = res.n_viewpoints
        v = np.ctypeslib.as_array(res.v, shape=(n,))
        c = np.ctypeslib.as_array(res.color, shape=(n,))
        b = None
        if res.bits:
            b = np.ctypeslib.as_array(res.bits, shape=(n, res.words_per_viewpoint))
        if copy:
            v, c = v.copy(), c.copy()
            b = b.copy() if b is not None else None
        st = {k: getattr(res.stats, k) for k, _ in vcm_stats._fields_}
        for k in ("latency_ms", "queue_ms", "device_ms", "group_size", "launch_form", "launch_ms", "chain_ms"):
            st[k] = getattr(res, k)
        return v, c, b, st

    def vcm_result_device(self, ticket):
        """Zero-copy torch views (v, color, bits or None, stats dict) of a
        finished ticket's device buffers, which the context owns: valid until
        vcm_result_release(ticket).  Exported through
        __cuda_array_interface__ (no stream: the result is complete)."""
        import torch

        res = vcm_result()
        self._ck(self.L.vcm_result_get(self.h, ticket, ctypes.byref(res)))
        n = res.n_viewpoints
        dev = torch.device("cuda", self.device)

        def view(addr, shape, typestr):
            return torch.as_tensor(_DeviceArray(int(addr), shape, typestr), device=dev)

        v = view(res.d_v, (n,), "<f4")
        c = view(res.d_color, (n,), "|u1")
        # bit words as int32 (the same 32 bits; torch's uint32 support is partial)
        b = view(res.d_bits, (n, res.words_per_viewpoint), "<i4") if res.d_bits else None
        st = {k: getattr(res.stats, k) for k, _ in vcm_stats._fields_}
        for k in ("latency_ms", "queue_ms", "device_ms", "group_size", "launch_form", "launch_ms", "chain_ms"):
            st[k] = getattr(res, k)
        return v, c, b, st

    def vcm_result_release(self, ticket):
        return self._ck(self.L.vcm_result_release(self.h, ticket))

    def vcm_cancel(self, ticket):
        return self._ck(self.L.vcm_cancel(self.h, ticket))

    def vcm_set_slots(self, slots, max_batch):
        return self._ck(self.L.vcm_set_slots(self.h, slots, max_batch))

    def vcm_get_memory(self):
        m = vcm_memory()
        self._ck(self.L.vcm_get_memory(self.h, ctypes.byref(m)))
        return {k: getattr(m, k) for k, _ in vcm_memory._fields_}

    def vcm_inject(self, kind, count):
        return self._ck(self.L.vcm_inject(self.h, kind, count))

    def vcm_cache_clear(self):
        return self._ck(self.L.vcm_cache_clear(self.h))

    def vcm_set_request_log(self, path):
        """Append one JSON metric line per completed request to `path` (None closes it)."""
        arg = None if path is None else os.fsencode(path)
        return self._ck(self.L.vcm_set_request_log(self.h, ctypes.c_char_p(arg)))

    def vcm_latency_summary(self):
        """(p50_ms, p99_ms, completed) over the scheduler's recent requests."""
        p50, p99, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
        self._ck(self.L.vcm_latency_summary(self.h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(n)))
        return p50.value, p99.value, n.value

    # tuning -------------------------------------------------------------------
    def vcm_autotune(self, samples):
        n = len(samples)
        arr = (vcm_request * n)()
        keep = []
        for i, d in enumerate(samples):
            r, z = make_request(d)
            arr[i] = r
            keep.append(z)
        out = (vcm_tune * n)()
        self._ck(self.L.vcm_autotune(self.h, arr, n, out))
        return [(t.tile_x, t.tile_y, t.patch_k, t.box_cap) for t in out]

    def vcm_set_tune(self, tile_x=0, tile_y=0, patch_k=0, box_cap=0):
        t = vcm_tune(tile_x, tile_y, patch_k, box_cap)
        return self._ck(self.L.vcm_set_tune(self.h, ctypes.byref(t)))

    def vcm_set_timing_events(self, before, after):
        """torch.cuda.Event pair (or None, None) recorded around the tile kernel."""
        b = before.cuda_event if before is not None else None
        a = after.cuda_event if after is not None else None
        return self._ck(self.L.vcm_set_timing_events(self.h, b, a))

    def vcm_get_tune(self, req):
        r, keep = make_request(req)
        t = vcm_tune()
        self._ck(self.L.vcm_get_tune(self.h, ctypes.byref(r), ctypes.byref(t)))
        return (t.tile_x, t.tile_y, t.patch_k, t.box_cap)


def vcm_compute_static(lo, hi, dims, req, d_v, d_color, d_bits, d_stats, stream, checked=False):
    """Module-level wrapper of the C entry point that allocates no device
    memory (no context): host boxes lo/hi (n x dims), device outputs."""
    lo = np.ascontiguousarray(np.asarray(lo, np.float32)[:, :dims])
    hi = np.ascontiguousarray(np.asarray(hi, np.float32)[:, :dims])
    r, keep = make_request(req)
    fp = ctypes.POINTER(ctypes.c_float)
    L = lib(checked)
    st = L.vcm_compute_static(lo.ctypes.data_as(fp), hi.ctypes.data_as(fp), lo.shape[0], dims, ctypes.byref(r),
                              d_v, d_color, d_bits, d_stats, stream)
    del keep
    return _check(st, None, L)


def stats_from_tensor(s):
    """Decode a device stats tensor (uint8, one vcm_stats) into a dict."""
    raw = bytes(s.cpu().numpy().tobytes())
    st = vcm_stats.from_buffer_copy(raw)
    return {k: getattr(st, k) for k, _ in vcm_stats._fields_}
