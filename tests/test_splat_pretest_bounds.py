"""The batched splat's per-chunk depth pre-test (splat mode 5) must be
conservative: it projects the eight corners of a chunk's bounding box with
the splat's own float32 steps and claims that every position inside the box
lands within 2 pixels of the corners' pixel range and gets a depth code no
lower than the corners' smallest minus M = 2^-18 ext qscale + 8 (ext the
largest |dx| + |dy| + |dz| over the corners), while ext / pitch and the
corners' pixel coordinates stay below 2^19. A chunk is skipped for a view
only under that claim, so a wrong bound would drop a winning fragment.

These checks replay the projection's float32 steps on the CPU (every
operation rounded to nearest on its own, as the kernels and the oracle do)
for random boxes, views and points inside the boxes, corners included, and
require every point to satisfy the bounds; a box 16 cells short of its
records breaks them (the checks bite)."""
import math

import numpy as np

f32 = np.float32


def view(rng, side, width, height):
    """An orthographic view as the splat derives it: origin, axes, 1 / pitch,
    half sizes, z0 and the depth scale 2^24 / (z1 - z0), all float32."""
    az, el = rng.uniform(0, 2 * math.pi), rng.uniform(-1.2, 1.2)
    eye = np.array([math.cos(el) * math.sin(az), math.sin(el), math.cos(el) * math.cos(az)])
    fwd = -eye
    right = np.cross(fwd, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    R = 0.5 * math.sqrt(3.0) * side
    centre = rng.uniform(-side, side, 3)
    pitch = 2.0 * R / min(width, height) * rng.uniform(0.05, 1.5)
    z0, z1 = -R * rng.uniform(0.8, 1.5), R * rng.uniform(0.8, 1.5)
    return {"o": centre.astype(f32), "r": right.astype(f32), "u": up.astype(f32), "f": fwd.astype(f32),
            "inv_pitch": f32(1.0) / f32(pitch), "hw": f32(0.5) * f32(width), "hh": f32(0.5) * f32(height),
            "z0": f32(z0), "qscale": f32(16777216.0) / (f32(z1) - f32(z0)), "W": width, "H": height}


def dot3(a, b):
    return (a[..., 0] * b[0] + a[..., 1] * b[1]) + a[..., 2] * b[2]


def project(p, v):
    """(ax, ay, qd) of points p [n, 3] (float32), with the splat's steps for
    k = 1 (project_point: clamped floors, clamped depth code)."""
    d = p - v["o"]
    sx = dot3(d, v["r"]) * v["inv_pitch"] + v["hw"]
    sy = dot3(d, v["u"]) * v["inv_pitch"] + v["hh"]
    z = dot3(d, v["f"])
    fz = np.floor((z - v["z0"]) * v["qscale"])
    qd = np.where(~(fz >= 0), 0, np.where(fz >= f32(16777215.0), (1 << 24) - 1, np.nan_to_num(fz))).astype(np.int64)
    fx = np.clip(np.floor(sx), -1073741824.0, 1073741824.0).astype(np.int64)
    fy = np.clip(np.floor(sy), -1073741824.0, 1073741824.0).astype(np.int64)
    ext = (np.abs(d[..., 0]) + np.abs(d[..., 1])) + np.abs(d[..., 2])
    return fx, fy, qd, ext


def bounds(bb, v, margin_px=2, margin_codes=True):
    """The pre-test's claims for box bb = (lo[3], hi[3]): (x0, x1, y0, y1,
    qlim) or None when the bounds are not established."""
    lo, hi = bb
    corners = np.array([[hi[0] if c & 1 else lo[0], hi[1] if c & 2 else lo[1], hi[2] if c & 4 else lo[2]]
                        for c in range(8)], dtype=f32)
    ax, ay, qd, ext = project(corners, v)
    e = ext.max()
    mag = max(np.abs(ax).max(), np.abs(ay).max())
    if not (e * v["inv_pitch"] < f32(524288.0)) or mag >= (1 << 19):
        return None
    m = e * v["qscale"] * f32(1.0 / 262144.0) + f32(8.0) if margin_codes else f32(0.0)
    qmin = int(qd.min())
    if not (m < f32(16777216.0)) or qmin <= m:
        return None
    return (ax.min() - margin_px, ax.max() + margin_px, ay.min() - margin_px, ay.max() + margin_px,
            qmin - int(math.ceil(float(m))))


def check(rng, trials, margin_px=2, margin_codes=True, shrink=0):
    """Points that break the claims over `trials` random boxes and views
    (`shrink` cells taken off the box's low side: a wrong box)."""
    bad = tested = 0
    for _ in range(trials):
        side = rng.uniform(0.5, 200.0)
        cube_min = rng.uniform(-side, 0, 3)
        cell = side / 2097152.0
        v = view(rng, side, int(rng.integers(64, 4096)), int(rng.integers(64, 4096)))
        # a chunk: grid positions (cell centres) within a small box of the cube
        q0 = rng.integers(0, 2097152 - 4096, 3)
        q = q0 + rng.integers(0, int(rng.choice([2, 64, 4096])), (2048, 3))
        p = (cube_min.astype(f32) + (q.astype(f32) + f32(0.5)) * f32(cell)).astype(f32)
        bb = (p.min(axis=0) + f32(shrink * 16 * cell), p.max(axis=0))
        b = bounds(bb, v, margin_px, margin_codes)
        if b is None:
            continue
        tested += 1
        ax, ay, qd, _ = project(p, v)
        x0, x1, y0, y1, qlim = b
        bad += int(((ax < x0) | (ax > x1) | (ay < y0) | (ay > y1) | (qd < qlim)).sum())
    return bad, tested


def test_pretest_bounds_hold_for_points_inside_the_box():
    bad, tested = check(np.random.default_rng(21), 300)
    assert tested > 250
    assert bad == 0


def test_a_box_short_of_its_records_fails():
    """Bounds computed from a box 16 cells short on its low side (records
    outside it) are broken by those records: the check detects a wrong box."""
    bad, tested = check(np.random.default_rng(22), 300, shrink=1)
    assert tested > 250
    assert bad > 0
