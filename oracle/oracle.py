"""ctypes front end of the CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It compiles ``vcm_oracle.c`` with gcc
into ``oracle/_build`` and converts the seeded inputs of ``synth`` into the
oracle's plain C structs.
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vcm_oracle.c")
_HDR = os.path.join(_HERE, "vcm_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libvcm_oracle.so")

_i64p = ctypes.POINTER(ctypes.c_int64)


class VoScene(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32), ("n_boxes", ctypes.c_int64),
                ("lo", _i64p), ("hi", _i64p)]


class VoRequest(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32), ("center", ctypes.c_int64 * 3),
                ("axis_u", ctypes.c_int32), ("axis_w", ctypes.c_int32), ("normal", ctypes.c_int32),
                ("width", ctypes.c_int64), ("height", ctypes.c_int64),
                ("patches_u", ctypes.c_int32), ("patches_w", ctypes.c_int32),
                ("grid_origin", ctypes.c_int64 * 2), ("grid_step", ctypes.c_int64 * 2),
                ("grid_nx", ctypes.c_int32), ("grid_ny", ctypes.c_int32),
                ("n_layers", ctypes.c_int32), ("layer_z", _i64p), ("mode", ctypes.c_int32),
                ("two_sided", ctypes.c_int32), ("fov_deg", ctypes.c_float), ("gaze", ctypes.c_float * 3)]

MODE_PARTIAL, MODE_STRICT, MODE_VIEWER = 0, 1, 2
FLAG_STRICT, FLAG_VIEWER, FLAG_TWO_SIDED = 2, 4, 8   # request flag bits that select the modes


def build(force=False):
    """Compile the oracle shared library if it is missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
               "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.vo_check.argtypes = [ctypes.POINTER(VoScene), ctypes.POINTER(VoRequest)]
        L.vo_patch_centres.argtypes = [ctypes.POINTER(VoRequest), _i64p]
        L.vo_patch_measure.argtypes = [ctypes.POINTER(VoRequest)]
        L.vo_patch_measure.restype = ctypes.c_double
        L.vo_viewpoint.argtypes = [ctypes.POINTER(VoRequest), ctypes.c_int64, _i64p]
        L.vo_segment_hits_box.argtypes = [ctypes.c_int, _i64p, _i64p, _i64p, _i64p]
        L.vo_visibility.argtypes = [ctypes.POINTER(VoScene), ctypes.POINTER(VoRequest),
                                    ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32)]
        L.vo_visibility.restype = ctypes.c_double
        L.vo_run.argtypes = [ctypes.POINTER(VoScene), ctypes.POINTER(VoRequest), _i64p,
                             ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
        L.vo_run_ex.argtypes = [ctypes.POINTER(VoScene), ctypes.POINTER(VoRequest), _i64p,
                                ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.vo_fov_test.argtypes = [ctypes.POINTER(VoRequest), _i64p, _i64p, ctypes.POINTER(ctypes.c_double)]
        L.vo_max.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int64]
        L.vo_max.restype = ctypes.c_double
        L.vo_quantise.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                  ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8)]
        _lib = L
    return _lib


def _p64(a):
    return a.ctypes.data_as(_i64p)


class _Pack:
    """Keeps the numpy buffers behind a struct alive."""

    def __init__(self, scene, req):
        self.req_layers = np.ascontiguousarray(req["layer_z"], dtype=np.int64)
        self.r = VoRequest()
        r = self.r
        r.dims = req["dims"]
        for k in range(3):
            r.center[k] = int(req["center"][k])
        r.axis_u, r.axis_w, r.normal = req["axis_u"], req["axis_w"], req["normal"]
        r.width, r.height = int(req["width"]), int(req["height"])
        r.patches_u, r.patches_w = req["patches_u"], req["patches_w"]
        for k in range(2):
            r.grid_origin[k] = int(req["grid_origin"][k])
            r.grid_step[k] = int(req["grid_step"][k])
        r.grid_nx, r.grid_ny = req["grid_nx"], req["grid_ny"]
        r.n_layers = len(req["layer_z"])
        r.layer_z = _p64(self.req_layers)
        fl = int(req.get("flags", 0))
        r.mode = MODE_VIEWER if fl & FLAG_VIEWER else (MODE_STRICT if fl & FLAG_STRICT else MODE_PARTIAL)
        r.two_sided = 1 if fl & FLAG_TWO_SIDED else 0
        r.fov_deg = float(req.get("fov_deg", 0.0))
        g = req.get("gaze", (0.0, 0.0, 0.0))
        for k in range(3):
            r.gaze[k] = float(g[k])
        self.s = None
        if scene is not None:
            self.lo = np.ascontiguousarray(scene.lo, dtype=np.int64)
            self.hi = np.ascontiguousarray(scene.hi, dtype=np.int64)
            self.s = VoScene(scene.dims, scene.n, _p64(self.lo), _p64(self.hi))


def check(scene, req):
    pk = _Pack(scene, req)
    return lib().vo_check(ctypes.byref(pk.s) if pk.s else None, ctypes.byref(pk.r))


def patch_centres(req):
    pk = _Pack(None, req)
    P = req["patches_u"] * req["patches_w"]
    out = np.zeros((P, 3), np.int64)
    if lib().vo_patch_centres(ctypes.byref(pk.r), _p64(out)) != 0:
        raise ValueError("patch centre outside the coordinate limit")
    return out


def patch_measure(req):
    pk = _Pack(None, req)
    return lib().vo_patch_measure(ctypes.byref(pk.r))


def viewpoint(req, index):
    pk = _Pack(None, req)
    out = np.zeros(3, np.int64)
    if lib().vo_viewpoint(ctypes.byref(pk.r), int(index), _p64(out)) != 0:
        raise ValueError("viewpoint outside the coordinate limit")
    return out


def segment_hits_box(dims, q, p, lo, hi):
    arrs = [np.ascontiguousarray(list(x) + [0] * (3 - len(x)), dtype=np.int64) for x in (q, p, lo, hi)]
    return lib().vo_segment_hits_box(int(dims), *[_p64(a) for a in arrs])


def default_threads():
    return max(1, os.cpu_count() or 1)


def run(scene, req, indices=None, bits=False, threads=None, band=False):
    """Visibility (float64) of the given viewpoint indices (all by default),
    and optionally the occlusion bits as uint32 [n, ceil(P/32)] and the
    field-of-view band as float64 [n, 3] (pairs within the band of the
    cone's edge, the terms of those counted, the terms of those left out).
    Returns v, or a tuple (v, bits) / (v, band) / (v, bits, band)."""
    pk = _Pack(scene, req)
    nvp = req["grid_nx"] * req["grid_ny"] * len(req["layer_z"])
    if indices is None:
        indices = np.arange(nvp, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.int64)
    n = indices.shape[0]
    P = 1 if int(req.get("flags", 0)) & FLAG_VIEWER else req["patches_u"] * req["patches_w"]
    words = (P + 31) // 32
    v = np.zeros(n, np.float64)
    b = np.zeros((n, words), np.uint32) if bits else None
    bd = np.zeros((n, 3), np.float64) if band else None
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib().vo_run_ex(ctypes.byref(pk.s), ctypes.byref(pk.r), _p64(indices), n, v.ctypes.data_as(dp),
                         b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)) if bits else None,
                         bd.ctypes.data_as(dp) if band else None, int(threads or default_threads()))
    if rc != 0:
        raise ValueError("oracle rejected the request")
    out = (v,) + ((b,) if bits else ()) + ((bd,) if band else ())
    return out[0] if len(out) == 1 else out


def fov_test(req, q, p):
    """Cone decision for the pair (q, p) in units: (inside, relative margin),
    or (None, 0.0) when the request has no cone."""
    pk = _Pack(None, req)
    qa = np.ascontiguousarray(list(q) + [0] * (3 - len(q)), dtype=np.int64)
    pa = np.ascontiguousarray(list(p) + [0] * (3 - len(p)), dtype=np.int64)
    m = ctypes.c_double(0.0)
    r = lib().vo_fov_test(ctypes.byref(pk.r), _p64(qa), _p64(pa), ctypes.byref(m))
    return (None, 0.0) if r < 0 else (bool(r), m.value)


def vmax(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().vo_max(v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), v.shape[0])


def quantise(v, v_ref, levels):
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(v.shape[0], np.uint8)
    rc = lib().vo_quantise(v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), v.shape[0],
                           float(v_ref), int(levels), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    if rc != 0:
        raise ValueError("bad color level count")
    return out
