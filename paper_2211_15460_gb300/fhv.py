"""Python binding of libfhv.so (include/fhv.h): argument marshalling only.

Every function here has the name of a C entry point and forwards to it;
device memory is owned by PyTorch tensors on the current CUDA device and the
stream is PyTorch's current stream unless one is given. All computation runs
in the library's CUDA kernels: if the library cannot be loaded this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

FHV_OK, FHV_ERR_INVALID_ARG, FHV_ERR_OVERFLOW, FHV_ERR_CUDA, FHV_ERR_TIMEOUT, FHV_ERR_UNSUPPORTED = range(6)
FHV_DEV_TIMEOUT, FHV_DEV_HUGE_TRIANGLE, FHV_DEV_RANGE, FHV_DEV_BAD_VIEW = 0x1, 0x2, 0x4, 0x8
FHV_DEV_INDEX_OVERFLOW = 0x10
FHV_CAPTURE_VIEW, FHV_CAPTURE_NORMAL, FHV_CAPTURE_AXIS3 = 0, 1, 2
FHV_LAYOUT_PPFL, FHV_LAYOUT_POFL, FHV_LAYOUT_POFA, FHV_LAYOUT_POFA_DIRECT, FHV_LAYOUT_POFA_SPARSE = 0, 1, 2, 3, 4
FHV_RENDER_WS_BYTES = 256
FHV_RAYCAST_WS_BYTES = 256 + 256 * 262144
RECORD_DTYPE = np.dtype([("key", "<u8"), ("tri", "<u4"), ("nrm", "<u4")])
OCTANT_DTYPE = np.dtype([("octant", "<u8"), ("off", "<u4"), ("cnt", "<u4")])

# every entry point declared in include/fhv.h
EXPORTS = ("fhv_level_offset", "fhv_memory_model", "fhv_query_sizes", "fhv_capture_ppfl", "fhv_build_pofl",
           "fhv_compact_pofa", "fhv_render_view", "fhv_get_count", "fhv_read_status", "fhv_status_str",
           "fhv_set_kernel_events", "fhv_kernel_events_recorded", "fhv_compact_pofa_static",
           "fhv_batch_workspace_size", "fhv_render_views", "fhv_raycast_pofa", "fhv_conv3x3_bf16",
           "fhv_conv3x3_wgrad_bf16", "fhv_conv3x3_flip_bf16", "fhv_splat_features", "fhv_gapfill_loss",
           "fhv_adam_bf16", "fhv_gapfill_compose", "fhv_atomic_probe", "fhv_build_pofl_reuse",
           "fhv_splat_visibility", "fhv_shade_owned", "fhv_pofa_leaf_index", "fhv_wait_probe",
           "fhv_build_pofa_direct", "fhv_read_static_status", "fhv_capture_fragments",
           "fhv_launch_count", "fhv_compact_pofa_sparse", "fhv_pofa_save", "fhv_pofa_load_header",
           "fhv_pofa_load")
FHV_STATIC_MAX_RECORDS = 1 << 20
FHV_WAIT_PROBE_WS_BYTES = 256 + 16


def FHV_LEAF_INDEX_WS_BYTES(n_max: int) -> int:
    """Workspace bytes of fhv_pofa_leaf_index for up to n_max records (the header macro)."""
    return 16 + 12 * ((int(n_max) + 4095) // 4096)


class FhvError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_str(status)} ({status})")
        self.status = status


class fhv_scene(C.Structure):
    _fields_ = [("idx", C.c_void_p), ("pos", C.c_void_p), ("nrm", C.c_void_p), ("tri_material", C.c_void_p),
                ("n_tri", C.c_uint32), ("n_vtx", C.c_uint32), ("cube_min", C.c_float * 3), ("cube_side", C.c_float),
                ("tri_base", C.c_uint32)]


class fhv_ortho_camera(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("right", C.c_float * 3), ("up", C.c_float * 3), ("fwd", C.c_float * 3),
                ("pitch", C.c_float), ("width", C.c_int32), ("height", C.c_int32), ("z0", C.c_float),
                ("z1", C.c_float)]


class fhv_frag_buf(C.Structure):
    _fields_ = [("rec", C.c_void_p), ("next", C.c_void_p), ("capacity", C.c_uint64), ("d_count", C.c_void_p)]


class fhv_splat_source(C.Structure):
    _fields_ = [("d_frag", C.c_void_p), ("n_max", C.c_uint64), ("d_n", C.c_void_p), ("tri_material", C.c_void_p),
                ("albedo", C.c_void_p), ("cube_min", C.c_float * 3), ("cube_side", C.c_float)]


class fhv_view(C.Structure):
    _fields_ = [("cam", fhv_ortho_camera), ("source", C.c_uint32), ("d_vis", C.c_void_p), ("d_rgba", C.c_void_p)]


class fhv_batch_config(C.Structure):
    _fields_ = [("views_per_item", C.c_uint32), ("frags_per_item", C.c_uint32), ("pixels_per_item", C.c_uint32),
                ("ctas_per_sm", C.c_uint32), ("splat_mode", C.c_uint32)]


class fhv_pofa_header(C.Structure):
    _fields_ = [("depth", C.c_int32), ("index_kind", C.c_int32), ("n_records", C.c_uint64),
                ("n_index_entries", C.c_uint64), ("reserved", C.c_uint64 * 5)]


class fhv_sizes(C.Structure):
    _fields_ = [("workspace_bytes", C.c_uint64), ("index_bytes", C.c_uint64), ("fragment_bytes", C.c_uint64),
                ("n_index_entries", C.c_uint64)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    """Path of the in-tree libfhv.so this module loads."""
    return _build.LIB


def lib():
    """Load libfhv.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libfhv.so is missing; build it with paper_2211_15460_gb300._build")
            L = C.CDLL(path)
            P, S = C.c_void_p, C.c_int
            L.fhv_level_offset.restype = C.c_uint64
            L.fhv_level_offset.argtypes = [C.c_int]
            L.fhv_memory_model.restype = S
            L.fhv_memory_model.argtypes = [S, C.c_uint64, C.c_int, C.c_double, C.c_uint64, C.c_uint32, C.c_uint32, P]
            L.fhv_query_sizes.restype = S
            L.fhv_query_sizes.argtypes = [S, C.c_uint32, C.c_int32, C.c_int32, C.c_int, C.c_uint64, P]
            L.fhv_capture_ppfl.restype = S
            L.fhv_capture_ppfl.argtypes = [P, P, P, P, P, C.c_size_t, P]
            L.fhv_build_pofl.restype = S
            L.fhv_build_pofl.argtypes = [P, S, P, C.c_float, C.c_int, P, P, P, P, C.c_size_t, P]
            L.fhv_launch_count.restype = C.c_uint64
            L.fhv_launch_count.argtypes = []
            L.fhv_pofa_save.restype = S
            L.fhv_pofa_save.argtypes = [C.c_char_p, C.c_int, P, C.c_uint64, P, P, P, P]
            L.fhv_pofa_load_header.restype = S
            L.fhv_pofa_load_header.argtypes = [C.c_char_p, P]
            L.fhv_pofa_load.restype = S
            L.fhv_pofa_load.argtypes = [C.c_char_p, P, C.c_uint64, P, P, P, C.c_uint64, P]
            L.fhv_compact_pofa_sparse.restype = S
            L.fhv_compact_pofa_sparse.argtypes = [P, C.c_uint64, P, C.c_int, P, P, C.c_uint64, P, P, C.c_size_t, P]
            L.fhv_capture_fragments.restype = S
            L.fhv_capture_fragments.argtypes = [P, S, P, C.c_float, P, P, C.c_size_t, P]
            L.fhv_compact_pofa.restype = S
            L.fhv_compact_pofa.argtypes = [P, C.c_uint64, P, C.c_int, P, P, P, P, C.c_size_t, P]
            L.fhv_build_pofa_direct.restype = S
            L.fhv_build_pofa_direct.argtypes = [P, S, P, C.c_float, C.c_int, P, C.c_uint64, P, P, P, P, C.c_size_t,
                                                P]
            L.fhv_build_pofl_reuse.restype = S
            L.fhv_build_pofl_reuse.argtypes = [P, S, P, C.c_float, C.c_int, P, P, P, P, C.c_size_t, P]
            L.fhv_render_view.restype = S
            L.fhv_render_view.argtypes = [P, C.c_uint64, P, P, P, P, C.c_int, P, C.c_int, P, P, P, C.c_size_t, P]
            L.fhv_wait_probe.restype = S
            L.fhv_wait_probe.argtypes = [C.c_int, P, C.c_size_t, P]
            L.fhv_pofa_leaf_index.restype = S
            L.fhv_pofa_leaf_index.argtypes = [P, C.c_uint64, P, C.c_int, P, P, P, P, P, C.c_size_t, P]
            L.fhv_splat_visibility.restype = S
            L.fhv_splat_visibility.argtypes = [P, C.c_uint64, P, C.c_uint64, P, P, C.c_int, P, P, C.c_size_t, P]
            L.fhv_shade_owned.restype = S
            L.fhv_shade_owned.argtypes = [P, C.c_uint64, P, C.c_uint64, P, P, P, C.c_int, P, P, P, P, C.c_size_t, P]
            L.fhv_get_count.restype = S
            L.fhv_get_count.argtypes = [P, P, P]
            L.fhv_read_status.restype = S
            L.fhv_read_status.argtypes = [P, P, P]
            L.fhv_status_str.restype = C.c_char_p
            L.fhv_status_str.argtypes = [S]
            L.fhv_set_kernel_events.restype = S
            L.fhv_set_kernel_events.argtypes = [C.c_char_p, P, P, S]
            L.fhv_kernel_events_recorded.restype = S
            L.fhv_kernel_events_recorded.argtypes = []
            L.fhv_batch_workspace_size.restype = S
            L.fhv_batch_workspace_size.argtypes = [C.c_int, P]
            L.fhv_render_views.restype = S
            L.fhv_render_views.argtypes = [P, C.c_int, P, C.c_int, P, C.c_int, C.c_int, P, P, C.c_size_t, P]
            L.fhv_compact_pofa_static.restype = S
            L.fhv_compact_pofa_static.argtypes = [P, C.c_uint64, P, C.c_int, P, P, P, P]
            L.fhv_read_static_status.restype = S
            L.fhv_read_static_status.argtypes = [P, P]
            L.fhv_conv3x3_bf16.restype = S
            L.fhv_conv3x3_bf16.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P, P, C.c_int, C.c_int, P, P, P, P]
            L.fhv_conv3x3_wgrad_bf16.restype = S
            L.fhv_conv3x3_wgrad_bf16.argtypes = [P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, P]
            L.fhv_conv3x3_flip_bf16.restype = S
            L.fhv_conv3x3_flip_bf16.argtypes = [P, C.c_int, C.c_int, P, P]
            L.fhv_splat_features.restype = S
            L.fhv_splat_features.argtypes = [P, P, P, P, P, P]
            L.fhv_gapfill_loss.restype = S
            L.fhv_gapfill_loss.argtypes = [P, P, P, C.c_uint64, C.c_float, P, P, P]
            L.fhv_gapfill_compose.restype = S
            L.fhv_gapfill_compose.argtypes = [P, P, C.c_uint64, P, P]
            L.fhv_adam_bf16.restype = S
            L.fhv_adam_bf16.argtypes = [P, P, P, P, C.c_uint64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, P,
                                        P]
            L.fhv_atomic_probe.restype = S
            L.fhv_atomic_probe.argtypes = [P, C.c_uint64, C.c_int, C.c_int, P, P]
            L.fhv_raycast_pofa.restype = S
            L.fhv_raycast_pofa.argtypes = [P, C.c_uint64, P, P, C.c_int, P, P, P, C.c_float, P, C.c_int, P, P, P, P,
                                           C.c_size_t, P]
            _lib = L
    return _lib


def status_str(status: int) -> str:
    """Name of an fhv_status code."""
    return lib().fhv_status_str(int(status)).decode()


def _check(status: int, where: str) -> int:
    if status != FHV_OK:
        raise FhvError(status, where)
    return status


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream if hasattr(s, "cuda_stream") else int(s))


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


# ----------------------------------------------------------------- structs

class DeviceScene:
    """A scene's arrays in device memory plus its fhv_scene struct."""

    def __init__(self, scene, device="cuda", non_blocking=False):
        import torch

        self.idx = torch.from_numpy(np.ascontiguousarray(scene.idx, np.uint32).view(np.int32)).to(device, non_blocking=non_blocking)
        self.pos = torch.from_numpy(np.ascontiguousarray(scene.pos, np.float32)).to(device, non_blocking=non_blocking)
        self.nrm = torch.from_numpy(np.ascontiguousarray(scene.nrm, np.float32)).to(device, non_blocking=non_blocking)
        self.tri_material = torch.from_numpy(np.ascontiguousarray(scene.tri_material, np.uint32).view(np.int32)).to(
            device, non_blocking=non_blocking)
        self.albedo = torch.from_numpy(np.ascontiguousarray(scene.albedo, np.float32)).to(device, non_blocking=non_blocking)
        self.n_tri = int(scene.n_tri)
        self.n_vtx = int(scene.n_vtx)
        self.cube_min = [float(v) for v in np.asarray(scene.cube_min, np.float32)]
        self.cube_side = float(np.float32(scene.cube_side))

    def struct(self) -> fhv_scene:
        s = fhv_scene()
        s.idx, s.pos, s.nrm, s.tri_material = (_ptr(self.idx), _ptr(self.pos), _ptr(self.nrm),
                                               _ptr(self.tri_material))
        s.n_tri, s.n_vtx = self.n_tri, self.n_vtx
        s.cube_min[:] = self.cube_min
        s.cube_side = self.cube_side
        s.tri_base = 0
        return s

    def slice(self, t0: int, t1: int) -> "SceneSlice":
        """Triangles [t0, t1) of this scene, captured with this scene's triangle ids."""
        return SceneSlice(self, t0, t1)


class SceneSlice:
    """Triangles [t0, t1) of a DeviceScene as an fhv_scene: index and
    material pointers advanced to triangle t0, the whole scene's vertices
    and cube, tri_base = t0 (records carry the whole scene's triangle ids)."""

    def __init__(self, scene: DeviceScene, t0: int, t1: int):
        if not 0 <= t0 <= t1 <= scene.n_tri:
            raise ValueError(f"triangle range [{t0}, {t1}) outside [0, {scene.n_tri}]")
        self.scene, self.t0, self.t1 = scene, int(t0), int(t1)
        self.albedo = scene.albedo

    def struct(self) -> fhv_scene:
        s = self.scene.struct()
        if self.t1 > self.t0:
            s.idx = _ptr(self.scene.idx) + 12 * self.t0
            s.tri_material = _ptr(self.scene.tri_material) + 4 * self.t0
        s.n_tri = self.t1 - self.t0
        s.tri_base = self.t0
        return s


def camera_struct(cam) -> fhv_ortho_camera:
    """An fhv_ortho_camera filled from a scenes.Camera (float32 fields)."""
    c = fhv_ortho_camera()
    c.origin[:] = [float(v) for v in np.asarray(cam.origin, np.float32)]
    c.right[:] = [float(v) for v in np.asarray(cam.right, np.float32)]
    c.up[:] = [float(v) for v in np.asarray(cam.up, np.float32)]
    c.fwd[:] = [float(v) for v in np.asarray(cam.fwd, np.float32)]
    c.pitch = float(np.float32(cam.pitch))
    c.width, c.height = int(cam.width), int(cam.height)
    c.z0, c.z1 = float(np.float32(cam.z0)), float(np.float32(cam.z1))
    return c


class FragBuf:
    """Global fragment list: 16-byte records, next links (unless `links` is
    False: records-only captures need none) and the counter."""

    def __init__(self, capacity: int, device="cuda", links: bool = True):
        import torch

        self.capacity = int(capacity)
        self.rec = torch.empty(max(self.capacity, 1) * 2, dtype=torch.int64, device=device)
        self.next = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=device) if links else None
        self.count = torch.zeros(2, dtype=torch.int64, device=device)

    def struct(self) -> fhv_frag_buf:
        f = fhv_frag_buf()
        f.rec, f.capacity, f.d_count = _ptr(self.rec), self.capacity, _ptr(self.count)
        f.next = _ptr(self.next) if self.next is not None else None
        return f

    def records_numpy(self, n: int) -> np.ndarray:
        return self.rec[: 2 * n].cpu().numpy().view(RECORD_DTYPE)


def records_to_numpy(t, n: int) -> np.ndarray:
    """View the first n records of an int64 [2 * capacity] tensor."""
    return t[: 2 * n].cpu().numpy().view(RECORD_DTYPE)


def workspace(nbytes: int, device="cuda"):
    """A device workspace of at least `nbytes` (and at least the 256-byte header), uint8."""
    import torch

    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ------------------------------------------------------------- entry points

def fhv_level_offset(level: int) -> int:
    """Index of level `level`'s first octant in the concatenated per-level arrays (root first)."""
    return int(lib().fhv_level_offset(level))


def fhv_memory_model(layout: int, n_pixels: int, depth: int, avg_depth_complexity: float, n_fragments: int,
                     list_record_bytes: int, array_record_bytes: int) -> int:
    """Bytes of a PPFL / POFL / POFA by the sizing formulas that reproduce Table 4."""
    out = C.c_uint64(0)
    _check(lib().fhv_memory_model(layout, n_pixels, depth, avg_depth_complexity, n_fragments, list_record_bytes,
                                  array_record_bytes, C.byref(out)), "fhv_memory_model")
    return int(out.value)


def fhv_query_sizes(layout: int, n_tri: int, width: int, height: int, depth: int, n_fragments: int) -> fhv_sizes:
    """Workspace, index and fragment sizes of a layout (fhv_sizes)."""
    out = fhv_sizes()
    _check(lib().fhv_query_sizes(layout, n_tri, width, height, depth, n_fragments, C.byref(out)), "fhv_query_sizes")
    return out


def fhv_capture_ppfl(scene: DeviceScene, cam, head, frags: FragBuf, ws, stream=None) -> int:
    """FHV_PPFL capture (Section 3.2): every fragment of the scene seen by `cam` into per-pixel lists
    (head: int32 [W * H])."""
    s, c, f = scene.struct(), camera_struct(cam), frags.struct()
    return _check(lib().fhv_capture_ppfl(C.byref(s), C.byref(c), _ptr(head), C.byref(f), _ptr(ws), ws.numel(),
                                         _stream(stream)), "fhv_capture_ppfl")


def fhv_build_pofl(scene: DeviceScene, mode: int, cam, pitch: float, depth: int, leaf_head, levels, frags: FragBuf,
                   ws, stream=None) -> int:
    """FHV_POFL build (Section 3.2): every fragment into the list of its leaf octant (leaf_head: int32
    [8^depth]) with child-occupancy masks of levels 0..depth-1 in `levels`."""
    s, f = scene.struct(), frags.struct()
    c = camera_struct(cam) if cam is not None else None
    return _check(lib().fhv_build_pofl(C.byref(s), mode, C.byref(c) if c is not None else None,
                                       float(np.float32(pitch)), depth, _ptr(leaf_head), _ptr(levels), C.byref(f),
                                       _ptr(ws), ws.numel(), _stream(stream)), "fhv_build_pofl")


def fhv_capture_fragments(scene: DeviceScene, mode: int, cam, pitch: float, frags: FragBuf, ws, stream=None) -> int:
    """Fragment capture into the global fragment list only (Sections 3.1, 3.2): records in rasteriser
    order, no lists; the input of fhv_compact_pofa."""
    s, f = scene.struct(), frags.struct()
    c = camera_struct(cam) if cam is not None else None
    return _check(lib().fhv_capture_fragments(C.byref(s), mode, C.byref(c) if c is not None else None,
                                              float(np.float32(pitch)), C.byref(f), _ptr(ws), ws.numel(),
                                              _stream(stream)), "fhv_capture_fragments")


def fhv_build_pofl_reuse(scene: DeviceScene, mode: int, cam, pitch: float, depth: int, leaf_head, levels,
                         frags: FragBuf, ws, stream=None) -> int:
    """fhv_build_pofl into lists that hold the previous build's result
    (resets only the heads that build wrote)."""
    s, f = scene.struct(), frags.struct()
    c = camera_struct(cam) if cam is not None else None
    return _check(lib().fhv_build_pofl_reuse(C.byref(s), mode, C.byref(c) if c is not None else None,
                                             float(np.float32(pitch)), depth, _ptr(leaf_head), _ptr(levels),
                                             C.byref(f), _ptr(ws), ws.numel(), _stream(stream)),
                  "fhv_build_pofl_reuse")


def fhv_build_pofa_direct(scene: DeviceScene, mode: int, cam, pitch: float, depth: int, pofa, capacity: int, count,
                          off, cnt, ws, stream=None) -> int:
    """The POFA rasterised straight into octant ranges (count, scan, scatter;
    no lists). `count` receives the fragment count even past `capacity`."""
    s = scene.struct()
    c = camera_struct(cam) if cam is not None else None
    return _check(lib().fhv_build_pofa_direct(C.byref(s), mode, C.byref(c) if c is not None else None,
                                              float(np.float32(pitch)), depth, _ptr(pofa) or None, capacity,
                                              _ptr(count), _ptr(off), _ptr(cnt), _ptr(ws), ws.numel(),
                                              _stream(stream)), "fhv_build_pofa_direct")


def fhv_compact_pofa(rec_in, n_max: int, d_n, depth: int, pofa, off, cnt, ws, stream=None) -> int:
    """FHV_POFA compaction (Sections 3.1, 3.2): records sorted into per-octant ranges, with (off, cnt) of
    every octant of every level (int32 [fhv_level_offset(depth + 1)] each)."""
    return _check(lib().fhv_compact_pofa(_ptr(rec_in), n_max, _ptr(d_n) or None, depth, _ptr(pofa), _ptr(off),
                                         _ptr(cnt), _ptr(ws), ws.numel(), _stream(stream)), "fhv_compact_pofa")


def fhv_compact_pofa_sparse(rec_in, n_max: int, d_n, depth: int, pofa, index, index_capacity: int, level_base,
                            ws, stream=None) -> int:
    """FHV_POFA compaction with a sparse octree index (Sections 3.1, 3.2): the same records as
    fhv_compact_pofa; `index` (int64 [2 * index_capacity], OCTANT_DTYPE entries) gets every occupied
    octant of every level, level l at [level_base[l], level_base[l + 1]) (level_base: int64 [depth + 2])."""
    return _check(lib().fhv_compact_pofa_sparse(_ptr(rec_in), n_max, _ptr(d_n) or None, depth, _ptr(pofa),
                                                _ptr(index) or None, index_capacity, _ptr(level_base), _ptr(ws),
                                                ws.numel(), _stream(stream)), "fhv_compact_pofa_sparse")


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def fhv_pofa_save(path: str, depth: int, pofa, off=None, cnt=None, index=None, level_base=None) -> None:
    """Write a POFA from host numpy arrays (records RECORD_DTYPE; the dense off/cnt uint32 arrays, or the
    sparse index OCTANT_DTYPE entries with its uint64 level bases) to `path`."""
    pofa = np.ascontiguousarray(pofa, RECORD_DTYPE)
    args = [np.ascontiguousarray(a, t) if a is not None else None
            for a, t in ((off, np.uint32), (cnt, np.uint32), (index, OCTANT_DTYPE), (level_base, np.uint64))]
    _check(lib().fhv_pofa_save(path.encode(), depth, _np_ptr(pofa), pofa.size, *[_np_ptr(a) for a in args]),
           "fhv_pofa_save")


def fhv_pofa_load_header(path: str) -> fhv_pofa_header:
    """The header of a saved POFA."""
    h = fhv_pofa_header()
    _check(lib().fhv_pofa_load_header(path.encode(), C.byref(h)), "fhv_pofa_load_header")
    return h


def fhv_pofa_load(path: str):
    """A saved POFA as host numpy arrays: (depth, records, index) with index = (off, cnt) for the complete
    octree or (entries, level_base) for a sparse index."""
    h = fhv_pofa_load_header(path)
    rec = np.zeros(max(h.n_records, 1), RECORD_DTYPE)
    if h.index_kind == 0:
        off = np.zeros(h.n_index_entries, np.uint32)
        cnt = np.zeros(h.n_index_entries, np.uint32)
        _check(lib().fhv_pofa_load(path.encode(), _np_ptr(rec), h.n_records, _np_ptr(off), _np_ptr(cnt), None, 0,
                                   None), "fhv_pofa_load")
        return h.depth, rec[: h.n_records], (off, cnt)
    ent = np.zeros(max(h.n_index_entries, 1), OCTANT_DTYPE)
    base = np.zeros(h.depth + 2, np.uint64)
    _check(lib().fhv_pofa_load(path.encode(), _np_ptr(rec), h.n_records, None, None, _np_ptr(ent),
                               h.n_index_entries, _np_ptr(base)), "fhv_pofa_load")
    return h.depth, rec[: h.n_records], (ent[: h.n_index_entries], base)


def sparse_levels(index, level_base, depth: int):
    """Host view of a sparse index: a list over levels 0..depth of OCTANT_DTYPE arrays."""
    lb = level_base[: depth + 2].cpu().numpy().astype(np.int64)
    entries = index[: 2 * int(lb[-1])].cpu().numpy().view(OCTANT_DTYPE).reshape(-1)
    return [entries[lb[l]: lb[l + 1]] for l in range(depth + 1)]


def fhv_compact_pofa_static(rec_in, n_max: int, d_n, depth: int, pofa, off, cnt, stream=None) -> int:
    """fhv_compact_pofa without a caller workspace (library-held scratch)."""
    return _check(lib().fhv_compact_pofa_static(_ptr(rec_in), n_max, _ptr(d_n) or None, depth, _ptr(pofa), _ptr(off),
                                                _ptr(cnt), _stream(stream)), "fhv_compact_pofa_static")


def fhv_render_view(frag, n_max: int, d_n, scene: DeviceScene, albedo, lights, n_lights: int, cam, footprint_k: int,
                    vis, rgba, ws, stream=None) -> int:
    """One novel view by splatting (Section 3.3): exact visibility keys (int64 [W * H]) and shaded RGBA
    (float32 [W * H * 4])."""
    s, c = scene.struct(), camera_struct(cam)
    return _check(lib().fhv_render_view(_ptr(frag), n_max, _ptr(d_n) or None, C.byref(s), _ptr(albedo), _ptr(lights),
                                        n_lights, C.byref(c), footprint_k, _ptr(vis), _ptr(rgba), _ptr(ws), ws.numel(),
                                        _stream(stream)), "fhv_render_view")


def fhv_wait_probe(kind: int, ws, stream=None) -> int:
    """A bounded device wait on a condition nothing satisfies; the workspace status reports FHV_DEV_TIMEOUT."""
    return _check(lib().fhv_wait_probe(kind, _ptr(ws), ws.numel(), _stream(stream)), "fhv_wait_probe")


def fhv_pofa_leaf_index(pofa, n_max: int, d_n, depth: int, leaf, off, cnt, m, ws, stream=None) -> int:
    """Sparse leaf index of a POFA: occupied leaves, their offsets and counts; m (device) = how many."""
    return _check(lib().fhv_pofa_leaf_index(_ptr(pofa), n_max, _ptr(d_n) or None, depth, _ptr(leaf), _ptr(off),
                                            _ptr(cnt), _ptr(m), _ptr(ws), ws.numel(), _stream(stream)),
                  "fhv_pofa_leaf_index")


def fhv_splat_visibility(frag, n_max: int, d_n, index_base: int, scene: DeviceScene, cam, footprint_k: int, vis, ws,
                         stream=None) -> int:
    """The splat step of fhv_render_view for records numbered from index_base."""
    s, c = scene.struct(), camera_struct(cam)
    return _check(lib().fhv_splat_visibility(_ptr(frag), n_max, _ptr(d_n) or None, index_base, C.byref(s), C.byref(c),
                                             footprint_k, _ptr(vis), _ptr(ws), ws.numel(), _stream(stream)),
                  "fhv_splat_visibility")


def fhv_shade_owned(frag, n_max: int, d_n, index_base: int, scene: DeviceScene, albedo, lights, n_lights: int, cam, vis,
                    rgba, ws, stream=None) -> int:
    """Shades the pixels whose winner is one of the records [index_base, index_base + n); zeros elsewhere."""
    s, c = scene.struct(), camera_struct(cam)
    return _check(lib().fhv_shade_owned(_ptr(frag), n_max, _ptr(d_n) or None, index_base, C.byref(s), _ptr(albedo),
                                        _ptr(lights), n_lights, C.byref(c), _ptr(vis), _ptr(rgba), _ptr(ws),
                                        ws.numel(), _stream(stream)), "fhv_shade_owned")


def fhv_raycast_pofa(pofa, n_max: int, off, cnt, depth: int, scene: DeviceScene, albedo, alpha, t_stop: float,
                     lights, n_lights: int, cam, vis, rgba, ws, stream=None) -> int:
    """Ray casting through a POFA; alpha None = opaque (R), else R/T."""
    s, c = scene.struct(), camera_struct(cam)
    return _check(lib().fhv_raycast_pofa(_ptr(pofa), n_max, _ptr(off), _ptr(cnt), depth, C.byref(s), _ptr(albedo),
                                         _ptr(alpha) or None, t_stop, _ptr(lights), n_lights, C.byref(c), _ptr(vis),
                                         _ptr(rgba), _ptr(ws), ws.numel(), _stream(stream)), "fhv_raycast_pofa")


def fhv_conv3x3_bf16(x, n, h, w, cin, weight, bias, cout, relu, mask, y, ws, stream=None) -> int:
    """Gap-filler 3x3 convolution on the tensor cores: y = act(conv3x3(x, weight) + bias), NHWC BF16, then
    zeroed channelwise where `mask` <= 0 (bias, ReLU and mask optional)."""
    return _check(lib().fhv_conv3x3_bf16(_ptr(x), n, h, w, cin, _ptr(weight), _ptr(bias) or None, cout, int(relu),
                                         _ptr(mask) or None, _ptr(y), _ptr(ws), _stream(stream)), "fhv_conv3x3_bf16")


def fhv_conv3x3_wgrad_bf16(x, dy, n, h, w, cin, cout, dweight, dbias, ws, stream=None) -> int:
    """Weight (and bias) gradient of fhv_conv3x3_bf16, accumulated into FP32 `dweight` / `dbias`."""
    return _check(lib().fhv_conv3x3_wgrad_bf16(_ptr(x), _ptr(dy), n, h, w, cin, cout, _ptr(dweight),
                                               _ptr(dbias) or None, _ptr(ws), _stream(stream)),
                  "fhv_conv3x3_wgrad_bf16")


def fhv_conv3x3_flip_bf16(weight, cin, cout, flipped, stream=None) -> int:
    """Weights rotated by 180 degrees with cin and cout swapped (the input-gradient convolution)."""
    return _check(lib().fhv_conv3x3_flip_bf16(_ptr(weight), cin, cout, _ptr(flipped), _stream(stream)),
                  "fhv_conv3x3_flip_bf16")


def fhv_splat_features(vis, rgba, frag, cam, feat, stream=None) -> int:
    """The gap-filler's input features of a splatted view (colour, depth, coverage, normal)."""
    c = camera_struct(cam)
    return _check(lib().fhv_splat_features(_ptr(vis), _ptr(rgba), _ptr(frag), C.byref(c), _ptr(feat),
                                           _stream(stream)), "fhv_splat_features")


def fhv_gapfill_loss(out, base, target, pixels, grad_scale, loss_sum, grad, stream=None) -> int:
    """Sum of squared RGB errors of out + base against the target, added to `loss_sum`; `grad` gets
    grad_scale * (out + base - target)."""
    return _check(lib().fhv_gapfill_loss(_ptr(out), _ptr(base) or None, _ptr(target), pixels, grad_scale,
                                         _ptr(loss_sum) or None, _ptr(grad) or None, _stream(stream)),
                  "fhv_gapfill_loss")


def fhv_gapfill_compose(out, base, pixels, rgba, stream=None) -> int:
    """The filled image: base + out, written as RGBA."""
    return _check(lib().fhv_gapfill_compose(_ptr(out), _ptr(base) or None, pixels, _ptr(rgba), _stream(stream)),
                  "fhv_gapfill_compose")


def fhv_adam_bf16(param, grad, m, v, n, lr, beta1, beta2, eps, step, out_bf16, stream=None) -> int:
    """One bias-corrected Adam step on FP32 parameters; clears `grad` and writes the optional BF16 copy."""
    return _check(lib().fhv_adam_bf16(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), n, lr, beta1, beta2, eps, step,
                                      _ptr(out_bf16) or None, _stream(stream)), "fhv_adam_bf16")


def fhv_atomic_probe(buf, n_words: int, ops_per_thread: int, returning, stream=None) -> int:
    """Launches the L2 microbenchmark (returning: 0 reductions, 1 returning atomics, 2 volatile reads);
    returns the operations it performs."""
    total = C.c_uint64(0)
    _check(lib().fhv_atomic_probe(_ptr(buf), n_words, ops_per_thread, int(returning), C.byref(total),
                                  _stream(stream)), "fhv_atomic_probe")
    return int(total.value)


def fhv_get_count(frags: FragBuf, stream=None):
    """(status, count): status is FHV_ERR_OVERFLOW when count > capacity."""
    f = frags.struct()
    out = C.c_uint64(0)
    st = lib().fhv_get_count(C.byref(f), C.byref(out), _stream(stream))
    if st not in (FHV_OK, FHV_ERR_OVERFLOW):
        raise FhvError(st, "fhv_get_count")
    return st, int(out.value)


def fhv_read_static_status(stream=None):
    """Synchronises `stream` and returns (status, FHV_DEV_* bits) of the last fhv_compact_pofa_static call."""
    out = C.c_uint32(0)
    st = lib().fhv_read_static_status(C.byref(out), _stream(stream))
    if st not in (FHV_OK, FHV_ERR_TIMEOUT):
        raise FhvError(st, "fhv_read_static_status")
    return st, int(out.value)


def fhv_read_status(ws, stream=None):
    """Synchronises `stream` and returns (status, FHV_DEV_* bits) of the last call that used `ws`."""
    out = C.c_uint32(0)
    st = lib().fhv_read_status(_ptr(ws), C.byref(out), _stream(stream))
    if st not in (FHV_OK, FHV_ERR_TIMEOUT):
        raise FhvError(st, "fhv_read_status")
    return st, int(out.value)


def fhv_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().fhv_launch_count())


def fhv_set_kernel_events(kernel, starts, stops) -> int:
    """Record torch.cuda.Event pairs around the first len(starts) launches of
    `kernel` (None clears). The events are recorded once here so that their
    CUDA handles exist."""
    if kernel is None or not starts:
        return _check(lib().fhv_set_kernel_events(None, None, None, 0), "fhv_set_kernel_events")
    for e in list(starts) + list(stops):
        e.record()
    n = len(starts)
    arr_s = (C.c_void_p * n)(*[e.cuda_event for e in starts])
    arr_e = (C.c_void_p * n)(*[e.cuda_event for e in stops])
    return _check(lib().fhv_set_kernel_events(kernel.encode(), arr_s, arr_e, n), "fhv_set_kernel_events")


def fhv_kernel_events_recorded() -> int:
    """How many event pairs fhv_set_kernel_events has recorded so far."""
    return int(lib().fhv_kernel_events_recorded())


def device_structs(structs, device="cuda"):
    """Copy an array of ctypes structures into a 16-byte aligned device buffer."""
    import torch

    raw = b"".join(bytes(x) for x in structs) or bytes(16)
    host = torch.frombuffer(bytearray(raw), dtype=torch.uint8)
    return host.to(device)


def fhv_batch_workspace_size(n_views: int) -> int:
    """Workspace bytes of fhv_render_views for `n_views` views."""
    out = C.c_size_t(0)
    _check(lib().fhv_batch_workspace_size(n_views, C.byref(out)), "fhv_batch_workspace_size")
    return int(out.value)


def fhv_render_views(d_sources, n_sources: int, d_views, n_views: int, lights, n_lights: int, footprint_k: int,
                     cfg: "fhv_batch_config", ws, stream=None) -> int:
    """Many views of many sources in one call (batched splat and shade), one visibility and image per
    view."""
    return _check(lib().fhv_render_views(_ptr(d_sources), n_sources, _ptr(d_views), n_views, _ptr(lights), n_lights,
                                         footprint_k, C.byref(cfg) if cfg is not None else None, _ptr(ws), ws.numel(),
                                         _stream(stream)), "fhv_render_views")
