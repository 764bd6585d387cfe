"""The capture kernels' float shortcut for the barycentric rounding of a
quantised coordinate (Section 3.1: every fragment stores its position
quantised to the octree's finest grid).

The exact value is q0 + floor(x / A + 1/2) with x = w1 d1 + w2 d2 (edge
values 0 <= w1, w2, w0 = A - w1 - w2). The kernel estimates t = x / A + 1/2
in float32 with the steps replayed here (every operation rounded to nearest)
and keeps floor(t) only when t's fraction is more than
qerr = 2^-21 (max |d1| + |d2| + 1) from an integer; otherwise it divides
exactly. These checks replay the float steps on the CPU and require the kept
floors to equal the exact ones, on random triangles and on values placed at
the rounding boundaries, where the estimate is most likely to be off."""
import numpy as np

f32 = np.float32


def float_path(w1, w2, A, d1, d2, dmax, band=None):
    """(kept, floor) of the kernel's float estimate; kept False means the
    exact division decides. `band` overrides qerr (to show the checks bite)."""
    fw1, fw2 = f32(float(w1)), f32(float(w2))  # int64 -> float32, one rounding (|w| < 2^53)
    inv_den = f32(1.0) / f32(float(2 * A))
    s = fw1 * f32(d1) + fw2 * f32(d2)
    t = (s + s) * inv_den + f32(0.5)
    fl = np.floor(t)
    fr = t - fl
    q = f32(dmax + 1) * f32(1.0 / 2097152.0)
    if float(q) < (dmax + 1) / 2097152.0:  # the kernel rounds this product up
        q = np.nextafter(q, f32(np.inf))
    if band is not None:
        q = f32(band)
    return bool(fr > q and fr < f32(1.0) - q), int(fl)


def exact(w1, w2, A, d1, d2):
    return (2 * (w1 * d1 + w2 * d2) + A) // (2 * A)


def check(rng, n, amax, dbits, boundary, band=None):
    bad = kept = 0
    for _ in range(n):
        A = int(rng.integers(2, amax))
        d = [int(v) for v in rng.integers(-(1 << dbits), 1 << dbits, size=2)]
        dmax = abs(d[0]) + abs(d[1])
        if boundary:
            # pick w1, w2 so that x / A + 1/2 lands on or next to an integer
            k = int(rng.integers(-dmax // 2 - 1, dmax // 2 + 2)) if dmax else 0
            target = (2 * k - 1) * A  # 2x = target makes x / A + 1/2 = k exactly
            w1 = int(rng.integers(0, A + 1))
            if d[1] == 0:
                continue
            w2 = (target // 2 - w1 * d[0]) // d[1] + int(rng.integers(-2, 3))
            if not (0 <= w2 <= A - w1):
                continue
        else:
            w1 = int(rng.integers(0, A + 1))
            w2 = int(rng.integers(0, A - w1 + 1))
        ok, fl = float_path(w1, w2, A, d[0], d[1], dmax, band)
        if ok:
            kept += 1
            bad += fl != exact(w1, w2, A, d[0], d[1])
    return bad, kept


def test_kept_floors_are_exact_on_random_triangles():
    rng = np.random.default_rng(11)
    for amax, dbits in [(1 << 12, 4), (1 << 24, 8), (1 << 40, 12), (1 << 40, 20)]:
        bad, kept = check(rng, 4000, amax, dbits, False)
        assert bad == 0
        assert kept > 0


def test_kept_floors_are_exact_at_rounding_boundaries():
    rng = np.random.default_rng(12)
    for amax, dbits in [(1 << 16, 6), (1 << 30, 10), (1 << 40, 16)]:
        bad, _ = check(rng, 4000, amax, dbits, True)
        assert bad == 0


def test_without_the_band_the_boundary_cases_fail():
    """The boundary cases do reach float estimates on the wrong side of an
    integer: keeping every floor (no band) gets some of them wrong."""
    rng = np.random.default_rng(12)
    bad = sum(check(rng, 4000, amax, dbits, True, band=0.0)[0] for amax, dbits in [(1 << 30, 10), (1 << 40, 16)])
    assert bad > 0


def test_half_way_values_take_the_exact_division():
    """x / A + 1/2 an integer exactly (a half-way rounding, w1 = A / 2,
    w2 = 0, d1 odd): t's fraction is 0, inside the band, so the exact
    division decides."""
    A = 1 << 20
    for d1 in (1, -1, 3, -5, 7):
        for d2 in (0, 2, -9):
            ok, _ = float_path(A // 2, 0, A, d1, d2, abs(d1) + abs(d2))
            assert not ok
