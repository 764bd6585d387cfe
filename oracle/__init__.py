"""CPU oracle for fragment-history volumes (arXiv 2211.15460).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline use it to check the CUDA path. The library never imports it.

`fhv_oracle.c` is a plain, sequential C restatement of the method (see its
header for the steps and the readings it fixes). This module compiles it with
gcc (float contraction off, so every float32 operation is rounded on its own)
and wraps it with ctypes over numpy arrays. Scenes and cameras are duck-typed:
any object with the attributes of `paper_2211_15460_gb300.scenes.Scene` /
`Camera` works; nothing from the CUDA package is imported here.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FHV_ORACLE_SRC lets the mutation tests build a deliberately broken copy of
# the oracle in a scratch directory; the default is the source next to this file.
_SRC = os.environ.get("FHV_ORACLE_SRC", os.path.join(_HERE, "fhv_oracle.c"))
_OUT = os.path.join(os.path.dirname(_SRC) if "FHV_ORACLE_SRC" in os.environ else _HERE, "_build",
                    "libfhv_oracle.so")
_lock = threading.Lock()
_lib = None

RECORD_DTYPE = np.dtype([("key", "<u8"), ("tri", "<u4"), ("nrm", "<u4")])
VIEW, NORMAL, AXIS3 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no float contraction)."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


class _Scene(C.Structure):
    _fields_ = [("idx", C.c_void_p), ("pos", C.c_void_p), ("nrm", C.c_void_p), ("tri_material", C.c_void_p),
                ("n_tri", C.c_uint32), ("n_vtx", C.c_uint32), ("cube_min", C.c_float * 3), ("cube_side", C.c_float)]


class _Camera(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("right", C.c_float * 3), ("up", C.c_float * 3), ("fwd", C.c_float * 3),
                ("pitch", C.c_float), ("width", C.c_int32), ("height", C.c_int32), ("z0", C.c_float),
                ("z1", C.c_float)]


def lib():
    """The oracle's C library, compiled on first use."""
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.orc_morton63.restype = C.c_uint64
            L.orc_morton63.argtypes = [C.c_uint32] * 3
            L.orc_oct_encode.restype = C.c_uint32
            L.orc_oct_encode.argtypes = [C.c_float] * 3
            L.orc_oct_decode.restype = None
            L.orc_oct_decode.argtypes = [C.c_uint32, P]
            L.orc_fragments.restype = C.c_uint64
            L.orc_fragments.argtypes = [P, C.c_int, P, C.c_float, P, P, P, C.c_uint64]
            L.orc_ppfl.restype = C.c_uint64
            L.orc_ppfl.argtypes = [P, P, P, P, P, C.c_uint64]
            L.orc_pofl.restype = C.c_uint64
            L.orc_pofl.argtypes = [P, C.c_int, P, C.c_float, C.c_int, P, P, P, P, C.c_uint64]
            L.orc_pofa_sort.restype = None
            L.orc_pofa_sort.argtypes = [P, C.c_uint64, P]
            L.orc_octant_range.restype = None
            L.orc_octant_range.argtypes = [P, C.c_uint64, C.c_int, C.c_uint64, P, P]
            L.orc_pofa.restype = None
            L.orc_pofa.argtypes = [P, C.c_uint64, C.c_int, P, P, P]
            L.orc_splat_visibility.restype = None
            L.orc_splat_visibility.argtypes = [P, C.c_uint64, P, P, C.c_int, P]
            L.orc_shade.restype = None
            L.orc_shade.argtypes = [P, P, P, P, P, C.c_int, P, P]
            L.orc_raycast.restype = None
            L.orc_raycast.argtypes = [P, C.c_uint64, P, P, P, P, C.c_int, P, P, P]
            L.orc_level_base.restype = C.c_uint64
            L.orc_level_base.argtypes = [C.c_int]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _Pinned:
    """Keeps the numpy arrays behind a ctypes scene alive."""

    def __init__(self, scene):
        self.idx = np.ascontiguousarray(scene.idx, np.uint32)
        self.pos = np.ascontiguousarray(scene.pos, np.float32)
        self.nrm = np.ascontiguousarray(scene.nrm, np.float32)
        self.mat = np.ascontiguousarray(scene.tri_material, np.uint32)
        s = _Scene()
        s.idx, s.pos, s.nrm, s.tri_material = (self.idx.ctypes.data, self.pos.ctypes.data, self.nrm.ctypes.data,
                                               self.mat.ctypes.data)
        s.n_tri = self.idx.size // 3
        s.n_vtx = self.pos.size // 3
        s.cube_min[:] = [float(v) for v in np.asarray(scene.cube_min, np.float32)]
        s.cube_side = float(np.float32(scene.cube_side))
        self.s = s


def _camera(cam) -> _Camera:
    c = _Camera()
    if cam is None:
        return c
    c.origin[:] = [float(v) for v in np.asarray(cam.origin, np.float32)]
    c.right[:] = [float(v) for v in np.asarray(cam.right, np.float32)]
    c.up[:] = [float(v) for v in np.asarray(cam.up, np.float32)]
    c.fwd[:] = [float(v) for v in np.asarray(cam.fwd, np.float32)]
    c.pitch = float(np.float32(cam.pitch))
    c.width, c.height = int(cam.width), int(cam.height)
    c.z0, c.z1 = float(np.float32(cam.z0)), float(np.float32(cam.z1))
    return c


# ------------------------------------------------------------------ primitives

def morton63(x: int, y: int, z: int) -> int:
    """Morton code of a quantised position (Section 3.1, Fig. 5): bit k of x, y, z at bits 3k+2, 3k+1, 3k."""
    return int(lib().orc_morton63(x, y, z))


def oct_encode(n) -> int:
    """Octahedral snorm16 code of a unit normal (Cigolle et al. 2014), the normal field of the 16-byte record."""
    n = np.asarray(n, np.float32)
    return int(lib().orc_oct_encode(float(n[0]), float(n[1]), float(n[2])))


def oct_decode(code: int) -> np.ndarray:
    """Inverse of oct_encode, in double, normalised."""
    out = np.zeros(3, np.float64)
    lib().orc_oct_decode(code, _ptr(out))
    return out


def level_base(level: int) -> int:
    """First octant of `level` in the concatenated per-level arrays, root first (Section 3.1, Fig. 6)."""
    return int(lib().orc_level_base(level))


def n_octants(depth: int) -> int:
    """Octants of levels 0..depth."""
    return level_base(depth + 1)


def decode_position(keys: np.ndarray) -> np.ndarray:
    """Quantised (x, y, z) from Morton codes (plain bit loop)."""
    keys = np.asarray(keys, np.uint64)
    q = np.zeros((keys.size, 3), np.int64)
    for b in range(21):
        for c, off in enumerate((2, 1, 0)):
            q[:, c] |= ((keys >> np.uint64(3 * b + off)) & np.uint64(1)).astype(np.int64) << b
    return q


# ------------------------------------------------------------------ method

def fragments(scene, mode: int, camera=None, pitch: float = 0.0):
    """All fragments in (triangle, row, column) order, with sample coords."""
    ps = _Pinned(scene)
    cam = _camera(camera)
    n = int(lib().orc_fragments(C.byref(ps.s), mode, C.byref(cam), float(np.float32(pitch)), None, None, None, 0))
    rec = np.zeros(n, RECORD_DTYPE)
    si = np.zeros(n, np.int64)
    sj = np.zeros(n, np.int64)
    lib().orc_fragments(C.byref(ps.s), mode, C.byref(cam), float(np.float32(pitch)), _ptr(rec), _ptr(si), _ptr(sj), n)
    return rec, si, sj


def fragment_count(scene, mode: int, camera=None, pitch: float = 0.0) -> int:
    """Number of fragments `fragments` would return, without storing them."""
    ps = _Pinned(scene)
    cam = _camera(camera)
    return int(lib().orc_fragments(C.byref(ps.s), mode, C.byref(cam), float(np.float32(pitch)), None, None, None, 0))


def ppfl(scene, camera, capacity: int):
    """FHV_PPFL: returns (count, head[W*H], records[capacity], next[capacity])."""
    ps = _Pinned(scene)
    cam = _camera(camera)
    head = np.empty(camera.width * camera.height, np.int32)
    rec = np.zeros(capacity, RECORD_DTYPE)
    nxt = np.full(capacity, -1, np.int32)
    cnt = int(lib().orc_ppfl(C.byref(ps.s), C.byref(cam), _ptr(head), _ptr(rec), _ptr(nxt), capacity))
    return cnt, head, rec, nxt


def pofl(scene, mode: int, camera, pitch: float, depth: int, capacity: int):
    """FHV_POFL: returns (count, leaf_head[8^d], levels[sum_{l<d} 8^l], records, next)."""
    ps = _Pinned(scene)
    cam = _camera(camera)
    leaf = np.empty(1 << (3 * depth), np.int32)
    levels = np.zeros(max(level_base(depth), 1), np.uint32)
    rec = np.zeros(capacity, RECORD_DTYPE)
    nxt = np.full(capacity, -1, np.int32)
    cnt = int(lib().orc_pofl(C.byref(ps.s), mode, C.byref(cam), float(np.float32(pitch)), depth, _ptr(leaf),
                             _ptr(levels), _ptr(rec), _ptr(nxt), capacity))
    return cnt, leaf, levels[: level_base(depth)], rec, nxt


def pofa_sort(records: np.ndarray) -> np.ndarray:
    """FHV_POFA order (Sections 3.1, 3.2; Fig. 6): records sorted by (Morton key, triangle, normal), so
    every octant's records are contiguous in Morton order."""
    rec = np.ascontiguousarray(records, RECORD_DTYPE)
    out = np.zeros_like(rec)
    lib().orc_pofa_sort(_ptr(rec), rec.size, _ptr(out))
    return out


def octant_range(sorted_records: np.ndarray, level: int, octant: int):
    """(off, cnt) of one octant of `level` in sorted records: the records whose level prefix is below
    it, and those with it (Section 3.1, Fig. 6)."""
    off = np.zeros(1, np.uint32)
    cnt = np.zeros(1, np.uint32)
    lib().orc_octant_range(_ptr(sorted_records), sorted_records.size, level, octant, _ptr(off), _ptr(cnt))
    return int(off[0]), int(cnt[0])


def pofa(records: np.ndarray, depth: int):
    """FHV_POFA: (sorted records, off[all levels], cnt[all levels])."""
    rec = np.ascontiguousarray(records, RECORD_DTYPE)
    out = np.zeros_like(rec)
    m = n_octants(depth)
    off = np.zeros(m, np.uint32)
    cnt = np.zeros(m, np.uint32)
    lib().orc_pofa(_ptr(rec), rec.size, depth, _ptr(out), _ptr(off), _ptr(cnt))
    return out, off, cnt


def splat_visibility(records: np.ndarray, scene, camera, k: int = 1) -> np.ndarray:
    """Splat visibility (Section 3.3): per pixel the minimum (24-bit depth << 40 | index) over the
    fragments whose k x k footprint covers it; all ones where nothing does."""
    rec = np.ascontiguousarray(records, RECORD_DTYPE)
    ps = _Pinned(scene)
    cam = _camera(camera)
    vis = np.empty(camera.width * camera.height, np.uint64)
    lib().orc_splat_visibility(_ptr(rec), rec.size, C.byref(ps.s), C.byref(cam), k, _ptr(vis))
    return vis


def shade(vis: np.ndarray, records: np.ndarray, scene, albedo, lights, camera) -> np.ndarray:
    """Shading of the visible fragments (Section 3.3, local illumination as in Section 5): albedo times
    the sum over lights of intensity * max(0, n . l); RGBA, background 0."""
    rec = np.ascontiguousarray(records, RECORD_DTYPE)
    ps = _Pinned(scene)
    cam = _camera(camera)
    alb = np.ascontiguousarray(albedo, np.float32)
    lig = np.ascontiguousarray(lights, np.float32).reshape(-1, 8)
    vis = np.ascontiguousarray(vis, np.uint64)
    rgba = np.empty((camera.width * camera.height, 4), np.float32)
    lib().orc_shade(_ptr(vis), _ptr(rec), C.byref(ps.s), _ptr(alb), _ptr(lig), lig.shape[0], C.byref(cam), _ptr(rgba))
    return rgba


def render(records, scene, camera, lights, k: int = 1):
    """A novel view: splat_visibility, then shade (Section 3.3)."""
    vis = splat_visibility(records, scene, camera, k)
    return vis, shade(vis, records, scene, scene.albedo, lights, camera)


def raycast(records, scene, camera, lights, alpha=None):
    """Ray casting: (vis, rgba). alpha: per-material opacity (None: opaque)."""
    rec = np.ascontiguousarray(records, RECORD_DTYPE)
    ps = _Pinned(scene)
    cam = _camera(camera)
    alb = np.ascontiguousarray(scene.albedo, np.float32)
    al = None if alpha is None else np.ascontiguousarray(alpha, np.float32)
    lig = np.ascontiguousarray(lights, np.float32).reshape(-1, 8)
    vis = np.empty(camera.width * camera.height, np.uint64)
    rgba = np.empty((camera.width * camera.height, 4), np.float32)
    lib().orc_raycast(_ptr(rec), rec.size, C.byref(ps.s), _ptr(alb), None if al is None else _ptr(al), _ptr(lig),
                      lig.shape[0], C.byref(cam), _ptr(vis), _ptr(rgba))
    return vis, rgba

