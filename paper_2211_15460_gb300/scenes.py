"""Seeded synthetic scenes, cameras and lights for fragment-history volumes.

This module only generates inputs: triangle meshes, materials, lights and
orthographic cameras. It holds none of the method's arithmetic (no
quantisation, rasterisation, Morton coding, sorting or shading) and imports
neither the CUDA binding nor the CPU oracle, so both sides can be fed from it.

The paper's own scenes (1,532 and 23.5 M triangles, Section 4, Figure 10) are
not available; these seeded scenes stand in for them with the shapes the
benchmark configurations name: UV-spheres, value-noise heightfields and boxes.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", 2014) used as a counter-based generator:
draw j of a stream with seed s is mix(s + (j + 1) * 0x9E3779B97F4A7C15).
Uniform floats take the top 24 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """splitmix64 stream; every call consumes the next `n` counters."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        """The next n outputs of the stream."""
        j = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix(self.seed + j * _GAMMA)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """float64 values in [lo, hi) built from the top 24 bits of each draw."""
        u = (self.u64(n) >> np.uint64(40)).astype(np.float64) / float(1 << 24)
        return lo + (hi - lo) * u


@dataclass
class Scene:
    """Indexed triangle mesh with per-vertex normals and per-triangle materials.

    pos, nrm: float32 [V, 3]; idx: uint32 [T, 3]; tri_material: uint32 [T];
    albedo: float32 [M, 3]. cube_min / cube_side describe the axis-aligned
    quantisation cube that encloses the scene (AABB minimum; largest extent
    enlarged by 2^-10 so every vertex lies strictly inside).
    """

    pos: np.ndarray
    nrm: np.ndarray
    idx: np.ndarray
    tri_material: np.ndarray
    albedo: np.ndarray
    cube_min: np.ndarray = field(default=None)
    cube_side: np.float32 = field(default=None)

    def __post_init__(self):
        self.pos = np.ascontiguousarray(self.pos, dtype=np.float32).reshape(-1, 3)
        self.nrm = np.ascontiguousarray(self.nrm, dtype=np.float32).reshape(-1, 3)
        self.idx = np.ascontiguousarray(self.idx, dtype=np.uint32).reshape(-1, 3)
        self.tri_material = np.ascontiguousarray(self.tri_material, dtype=np.uint32).reshape(-1)
        self.albedo = np.ascontiguousarray(self.albedo, dtype=np.float32).reshape(-1, 3)
        if self.cube_min is None:
            self.cube_min, self.cube_side = bounding_cube(self.pos)
        self.cube_min = np.ascontiguousarray(self.cube_min, dtype=np.float32).reshape(3)
        self.cube_side = np.float32(self.cube_side)

    @property
    def n_tri(self) -> int:
        """Number of triangles."""
        return int(self.idx.shape[0])

    @property
    def n_vtx(self) -> int:
        """Number of vertices."""
        return int(self.pos.shape[0])

    @property
    def center(self) -> np.ndarray:
        """Centre of the quantisation cube (float64)."""
        return self.cube_min.astype(np.float64) + 0.5 * float(self.cube_side)


def bounding_cube(pos: np.ndarray):
    """Quantisation cube of the positions: AABB minimum and largest extent enlarged by 2^-10."""
    if pos.shape[0] == 0:
        return np.zeros(3, np.float32), np.float32(1.0)
    lo = pos.min(axis=0).astype(np.float32)
    hi = pos.max(axis=0).astype(np.float32)
    ext = float(np.max(hi.astype(np.float64) - lo.astype(np.float64)))
    if ext <= 0.0:
        ext = 1.0
    return lo, np.float32(ext * (1.0 + 2.0 ** -10))


def concat(parts, albedo) -> Scene:
    """Concatenate (pos, nrm, idx, material) parts into one scene."""
    pos, nrm, idx, mat = [], [], [], []
    base = 0
    for p, n, i, m in parts:
        pos.append(p)
        nrm.append(n)
        idx.append(i.astype(np.int64) + base)
        mat.append(np.full(i.shape[0], m, np.uint32) if np.isscalar(m) else m)
        base += p.shape[0]
    return Scene(
        pos=np.concatenate(pos) if pos else np.zeros((0, 3)),
        nrm=np.concatenate(nrm) if nrm else np.zeros((0, 3)),
        idx=np.concatenate(idx) if idx else np.zeros((0, 3)),
        tri_material=np.concatenate(mat) if mat else np.zeros(0),
        albedo=albedo,
    )


# --------------------------------------------------------------------------- meshes

def uv_sphere(center, radius, segments=32, rings=16):
    """Closed UV-sphere with shared vertices: 2*segments*(rings-1) triangles."""
    c = np.asarray(center, np.float64)
    th = np.pi * np.arange(1, rings) / rings  # interior ring latitudes
    ph = 2.0 * np.pi * np.arange(segments) / segments
    st, ct = np.sin(th)[:, None], np.cos(th)[:, None]
    ring_dirs = np.stack(
        [st * np.cos(ph)[None, :], np.broadcast_to(ct, (rings - 1, segments)), st * np.sin(ph)[None, :]],
        axis=-1,
    ).reshape(-1, 3)
    dirs = np.concatenate([[[0.0, 1.0, 0.0]], ring_dirs, [[0.0, -1.0, 0.0]]])
    pos = c + radius * dirs
    top, bot = 0, 1 + (rings - 1) * segments

    def v(r, s):  # r in [0, rings-2]
        return 1 + r * segments + (s % segments)

    tris = []
    for s in range(segments):
        tris.append((top, v(0, s + 1), v(0, s)))
    for r in range(rings - 2):
        for s in range(segments):
            a, b = v(r, s), v(r, s + 1)
            cc, d = v(r + 1, s), v(r + 1, s + 1)
            tris.append((a, b, d))
            tris.append((a, d, cc))
    for s in range(segments):
        tris.append((bot, v(rings - 2, s), v(rings - 2, s + 1)))
    return pos, dirs.copy(), np.asarray(tris, np.int64)


def box(center, sides):
    """Axis-aligned box: 24 vertices (flat normals), 12 outward triangles."""
    c = np.asarray(center, np.float64)
    h = 0.5 * np.asarray(sides, np.float64)
    pos, nrm, tris = [], [], []
    for axis in range(3):
        for sgn in (1.0, -1.0):
            n = np.zeros(3)
            n[axis] = sgn
            u = np.zeros(3)
            u[(axis + 1) % 3] = 1.0
            w = np.cross(n, u)
            base = len(pos)
            for a, b in ((-1, -1), (1, -1), (1, 1), (-1, 1)):
                pos.append(c + h * (n + a * u + b * w))
                nrm.append(n)
            tris.append((base, base + 1, base + 2))
            tris.append((base, base + 2, base + 3))
    return np.asarray(pos), np.asarray(nrm), np.asarray(tris, np.int64)


def boxes(centers, sides):
    """Many axis-aligned boxes at once; box b is exactly `box(centers[b], sides[b])`."""
    c = np.asarray(centers, np.float64).reshape(-1, 1, 3)
    h = 0.5 * np.asarray(sides, np.float64).reshape(-1, 1, 3)
    nb = c.shape[0]
    frame_n, corner_off, tris = [], [], []
    for axis in range(3):
        for sgn in (1.0, -1.0):
            n = np.zeros(3)
            n[axis] = sgn
            u = np.zeros(3)
            u[(axis + 1) % 3] = 1.0
            w = np.cross(n, u)
            base = len(frame_n)
            for a, b in ((-1, -1), (1, -1), (1, 1), (-1, 1)):
                frame_n.append(n)
                corner_off.append(n + a * u + b * w)
            tris.append((base, base + 1, base + 2))
            tris.append((base, base + 2, base + 3))
    off = np.asarray(corner_off)[None, :, :]  # [1, 24, 3]
    pos = (c + h * off).reshape(-1, 3)
    nrm = np.broadcast_to(np.asarray(frame_n)[None], (nb, 24, 3)).reshape(-1, 3)
    idx = (np.asarray(tris, np.int64)[None, :, :] + 24 * np.arange(nb)[:, None, None]).reshape(-1, 3)
    return pos, nrm, idx


def _smooth(t):
    return t * t * (3.0 - 2.0 * t)


def _dsmooth(t):
    return 6.0 * t * (1.0 - t)


def heightfield(rng: Rng, n: int, amplitude=0.2, lattice=16):
    """n x n vertex grid over [0,1]^2 (x, z) with y = amplitude * value noise.

    Value noise: hashed U[0,1] values on a (lattice+1)^2 grid, smoothstep
    bilinear interpolation. Normals from the analytic gradient.
    """
    vals = rng.uniform((lattice + 1) * (lattice + 1)).reshape(lattice + 1, lattice + 1)
    g = np.linspace(0.0, 1.0, n)
    X, Z = np.meshgrid(g, g, indexing="xy")
    fx, fz = X * lattice, Z * lattice
    ix = np.minimum(fx.astype(np.int64), lattice - 1)
    iz = np.minimum(fz.astype(np.int64), lattice - 1)
    tx, tz = fx - ix, fz - iz
    sx, sz = _smooth(tx), _smooth(tz)
    v00, v10 = vals[iz, ix], vals[iz, ix + 1]
    v01, v11 = vals[iz + 1, ix], vals[iz + 1, ix + 1]
    a = v00 + (v10 - v00) * sx
    b = v01 + (v11 - v01) * sx
    H = amplitude * (a + (b - a) * sz)
    dsx = _dsmooth(tx) * lattice
    dsz = _dsmooth(tz) * lattice
    dHdx = amplitude * ((v10 - v00) * (1 - sz) + (v11 - v01) * sz) * dsx
    dHdz = amplitude * (b - a) * dsz
    pos = np.stack([X, H, Z], axis=-1).reshape(-1, 3)
    nrm = np.stack([-dHdx, np.ones_like(H), -dHdz], axis=-1).reshape(-1, 3)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r = np.arange(n - 1)
    i00 = (r[:, None] * n + r[None, :]).reshape(-1)
    i10, i01, i11 = i00 + 1, i00 + n, i00 + n + 1
    # upward-facing (counter-clockwise seen from +y)
    t1 = np.stack([i00, i01, i11], axis=1)
    t2 = np.stack([i00, i11, i10], axis=1)
    tris = np.stack([t1, t2], axis=1).reshape(-1, 3)
    return pos, nrm, tris


# --------------------------------------------------------------------------- cameras / lights

@dataclass
class Camera:
    """Orthographic camera: image-plane centre `origin`, unit `right`, `up`,
    `fwd` (viewing direction), world size of one pixel `pitch`, and the depth
    range [z0, z1] (along fwd, relative to origin) for the 24-bit depth code."""

    origin: np.ndarray
    right: np.ndarray
    up: np.ndarray
    fwd: np.ndarray
    pitch: float
    width: int
    height: int
    z0: float
    z1: float

    def __post_init__(self):
        for k in ("origin", "right", "up", "fwd"):
            setattr(self, k, np.ascontiguousarray(getattr(self, k), dtype=np.float32).reshape(3))
        self.pitch = np.float32(self.pitch)
        self.z0 = np.float32(self.z0)
        self.z1 = np.float32(self.z1)
        self.width = int(self.width)
        self.height = int(self.height)


def orbit_camera(scene: Scene, width: int, height: int, azimuth_deg=0.0, elevation_deg=30.0, orbit_deg=0.0):
    """Camera at the cube centre looking at it from (azimuth + orbit, elevation).

    The pitch frames the cube's bounding sphere in min(width, height) pixels;
    the depth range is the sphere's. Orbiting rotates the view about world +y
    through the cube centre.
    """
    c = scene.center
    R = 0.5 * math.sqrt(3.0) * float(scene.cube_side)
    az = math.radians(azimuth_deg + orbit_deg)
    el = math.radians(elevation_deg)
    eye_dir = np.array([math.cos(el) * math.sin(az), math.sin(el), math.cos(el) * math.cos(az)])
    fwd = -eye_dir
    right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    up /= np.linalg.norm(up)
    return Camera(c, right, up, fwd, 2.0 * R / min(width, height), width, height, -R, R)


def directional_light(direction, intensity=(1.0, 1.0, 1.0)):
    """A light record {0, unit direction towards the light, intensity, 0}."""
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    return np.array([0.0, *d, *intensity, 0.0], np.float32)


def point_light(position, intensity=(1.0, 1.0, 1.0)):
    """A light record {1, position, intensity, 0}."""
    return np.array([1.0, *position, *intensity, 0.0], np.float32)


# --------------------------------------------------------------------------- workloads

def spheres_scene(seed=1, n_spheres=8, segments=32, rings=16, radius_scale=1.0):
    """Seeded UV-spheres: centres U[0,1]^3, radii U[0.05,0.2] x radius_scale,
    albedo U[0.2,1]^3."""
    rng = Rng(seed)
    centres = rng.uniform(3 * n_spheres).reshape(n_spheres, 3)
    radii = rng.uniform(n_spheres, 0.05, 0.2) * radius_scale
    albedo = rng.uniform(3 * n_spheres, 0.2, 1.0).reshape(n_spheres, 3)
    if n_spheres <= 64:
        parts = []
        for s in range(n_spheres):
            p, n, t = uv_sphere(centres[s], radii[s], segments, rings)
            parts.append((p, n, t, s))
        return concat(parts, albedo)
    proto_p, proto_n, proto_t = uv_sphere((0.0, 0.0, 0.0), 1.0, segments, rings)
    nv, nt = proto_p.shape[0], proto_t.shape[0]
    dirs = proto_p  # unit sphere: positions are the directions
    pos = (centres[:, None, :] + radii[:, None, None] * dirs[None]).reshape(-1, 3)
    nrm = np.broadcast_to(proto_n[None], (n_spheres, nv, 3)).reshape(-1, 3)
    idx = (proto_t[None] + nv * np.arange(n_spheres)[:, None, None]).reshape(-1, 3)
    mat = np.repeat(np.arange(n_spheres, dtype=np.uint32), nt)
    return Scene(pos=pos, nrm=nrm, idx=idx, tri_material=mat, albedo=albedo)


def terrain_scene(seed=2, grid=708, n_boxes=200, amplitude=0.2, lattice=16):
    """Heightfield (grid^2 vertices, value noise) plus seeded boxes.

    Boxes: centre U[0,1] x U[0,0.2] x U[0,1] (y up), sides U[0.01,0.08] per
    axis. Material 0 is the terrain, material 1+b is box b.
    """
    rng = Rng(seed)
    p, n, t = heightfield(rng, grid, amplitude, lattice)
    parts = [(p, n, t, 0)]
    cx = rng.uniform(n_boxes)
    cz = rng.uniform(n_boxes)
    cy = rng.uniform(n_boxes, 0.0, 0.2)
    sides = rng.uniform(3 * n_boxes, 0.01, 0.08).reshape(n_boxes, 3)
    bp, bn, bt = boxes(np.stack([cx, cy, cz], axis=1), sides)
    parts.append((bp, bn, bt, np.repeat(1 + np.arange(n_boxes, dtype=np.uint32), 12)))
    albedo = np.concatenate([[[0.55, 0.6, 0.45]], rng.uniform(3 * n_boxes, 0.2, 1.0).reshape(n_boxes, 3)])
    return concat(parts, albedo)


def instanced_spheres_heightfield(seed=5, n_spheres=2000, grid=2048, segments=64, rings=32):
    """Stress scene: instanced UV-spheres scattered over a heightfield."""
    rng = Rng(seed)
    p, n, t = heightfield(rng, grid, 0.2, 16)
    parts = [(p, n, t, 0)]
    proto_p, proto_n, proto_t = uv_sphere((0.0, 0.0, 0.0), 1.0, segments, rings)
    cen = np.stack([rng.uniform(n_spheres), rng.uniform(n_spheres, 0.2, 0.4), rng.uniform(n_spheres)], axis=1)
    rad = rng.uniform(n_spheres, 0.004, 0.02)
    nv = proto_p.shape[0]
    parts.append(((cen[:, None, :] + rad[:, None, None] * proto_p[None]).reshape(-1, 3),
                  np.broadcast_to(proto_n[None], (n_spheres, nv, 3)).reshape(-1, 3),
                  (proto_t[None] + nv * np.arange(n_spheres)[:, None, None]).reshape(-1, 3),
                  np.repeat(1 + (np.arange(n_spheres) % 64).astype(np.uint32), proto_t.shape[0])))
    albedo = np.concatenate([[[0.55, 0.6, 0.45]], rng.uniform(3 * 64, 0.2, 1.0).reshape(64, 3)])
    return concat(parts, albedo)


def boxes_scene(seed=4, n_boxes=1000):
    """Seeded boxes in the unit cube: centre U[0,1]^3, sides U[0.005,0.05]."""
    rng = Rng(seed)
    c = rng.uniform(3 * n_boxes).reshape(n_boxes, 3)
    sides = rng.uniform(3 * n_boxes, 0.005, 0.05).reshape(n_boxes, 3)
    bp, bn, bt = boxes(c, sides)
    mat = np.repeat((np.arange(n_boxes) % 32).astype(np.uint32), 12)
    return concat([(bp, bn, bt, mat)], rng.uniform(3 * 32, 0.2, 1.0).reshape(32, 3))


@dataclass
class Workload:
    """One plain-FHV configuration: scene, capture camera, octree depth,
    novel views, lights and splat footprint."""

    name: str
    scene: Scene
    capture: Camera
    depth: int
    views: list
    lights: np.ndarray
    footprint_k: int = 1
    normal_pitch: float = None

    def __post_init__(self):
        if self.normal_pitch is None:
            self.normal_pitch = float(self.capture.pitch)
        self.lights = np.ascontiguousarray(self.lights, np.float32).reshape(-1, 8)


def workload_spheres_256(seed=1):
    """8 UV-spheres (32x16, 7,680 triangles), 256^2 capture, depth 6, one
    novel view at a 30 degree orbit, one directional light."""
    sc = spheres_scene(seed)
    cap = orbit_camera(sc, 256, 256)
    views = [orbit_camera(sc, 256, 256, orbit_deg=30.0)]
    lights = directional_light((1.0, 1.0, 1.0))[None]
    return Workload("spheres8_256_d6", sc, cap, 6, views, lights)


# Axis captures of the stress scene take cube_side / STRESS_RESOLUTION as
# their pitch: the square resolution that gives about 5e8 fragments (measured
# by counting the scene's fragments at two coarse pitches and scaling by the
# area: 5.0e8 at 7616, i.e. 564,481 at 256 x (7616 / 256)^2).
STRESS_RESOLUTION = 7616


def workload_stress(seed=5):
    """Stress configuration: 16,316,418 triangles (2000 instanced 64x32
    UV-spheres on a 2048^2 heightfield), captured along the three axes (the
    fragments of the six axis-aligned views, each once) into one POFA at
    depth 11 with pitch cube_side / 7616 (about 5e8 fragments), 16 novel
    views at 3840x2160 orbiting in 22.5 degree steps, 8 point lights."""
    sc = instanced_spheres_heightfield(seed)
    cap = orbit_camera(sc, 3840, 2160)  # the axis capture does not use a camera
    views = [orbit_camera(sc, 3840, 2160, orbit_deg=22.5 * i) for i in range(16)]
    rng = Rng(seed * 1000 + 7)
    lx, lz = rng.uniform(8), rng.uniform(8)
    ly = rng.uniform(8, 0.5, 1.0)
    lights = np.stack([point_light((lx[i], ly[i], lz[i]), (0.125, 0.125, 0.125)) for i in range(8)])
    return Workload("stress16M_axis3_d11_4k", sc, cap, 11, views, lights,
                    normal_pitch=float(sc.cube_side) / STRESS_RESOLUTION)


def workload_stress_small(seed=5):
    """The stress configuration scaled down for profiles and quick checks:
    3,085,058 triangles (250 instanced UV-spheres on a 1024^2 heightfield),
    three-axis capture at pitch cube_side / 3808 (about 5.3e7 fragments),
    POFA at depth 9, 16 views at 1920x1080 (about 26 fragments per pixel
    and view, the stress step's kind of overdraw), 8 point lights."""
    sc = instanced_spheres_heightfield(seed, n_spheres=250, grid=1024)
    cap = orbit_camera(sc, 1920, 1080)
    views = [orbit_camera(sc, 1920, 1080, orbit_deg=22.5 * i) for i in range(16)]
    rng = Rng(seed * 1000 + 7)
    lx, lz = rng.uniform(8), rng.uniform(8)
    ly = rng.uniform(8, 0.5, 1.0)
    lights = np.stack([point_light((lx[i], ly[i], lz[i]), (0.125, 0.125, 0.125)) for i in range(8)])
    return Workload("stress3M_axis3_d9_1080p", sc, cap, 9, views, lights,
                    normal_pitch=float(sc.cube_side) / (STRESS_RESOLUTION // 2))


def workload_terrain_1080p(seed=2, grid=708, n_boxes=200):
    """1,002,098-triangle terrain (708^2 heightfield + 200 boxes), 1920x1080
    capture, depth 10, novel views at 0/30/60 degrees, 8 point lights."""
    sc = terrain_scene(seed, grid, n_boxes)
    cap = orbit_camera(sc, 1920, 1080)
    views = [orbit_camera(sc, 1920, 1080, orbit_deg=a) for a in (0.0, 30.0, 60.0)]
    rng = Rng(seed * 1000 + 7)
    lx, lz = rng.uniform(8), rng.uniform(8)
    ly = rng.uniform(8, 0.5, 1.0)
    lights = np.stack([point_light((lx[i], ly[i], lz[i]), (0.125, 0.125, 0.125)) for i in range(8)])
    return Workload("terrain1M_1080p_d10", sc, cap, 10, views, lights)
