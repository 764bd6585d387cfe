"""Pins of the gap-filler oracle (CPU): each check ties the oracle to
something other than itself -- a library correlation, the adjoint identity,
exact finite differences of a bilinear form, closed forms."""
import importlib.util
import os

import numpy as np
import pytest

if os.environ.get("FHV_GAPFILL_ORACLE_SRC"):  # a planted mistake (tests/test_oracle_mutations.py)
    _spec = importlib.util.spec_from_file_location("gapfill_under_test", os.environ["FHV_GAPFILL_ORACLE_SRC"])
    G = importlib.util.module_from_spec(_spec)
    _spec.loader.exec_module(G)
else:
    from oracle import gapfill as G

scipy_signal = pytest.importorskip("scipy.signal")


def rnd(rng, *shape):
    return G.bf16_round(rng.standard_normal(shape))


def test_bf16_rounding_known_values():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e38, 1.0 + 2 ** -9])
    exp = np.array([1.0, 1.0, 1.0 + 2 ** -6, -2.5, G.from_bf16_bits(G.bf16_bits([3.0e38]))[0], 1.0])
    # 1 + 2^-8 is half-way between 1 and 1 + 2^-7: ties to even -> 1
    # 1 + 3 * 2^-8 is half-way between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6
    assert (G.bf16_round(vals) == exp).all()
    assert G.bf16_bits([1.0])[0] == 0x3F80 and G.bf16_bits([-2.0])[0] == 0xC000


@pytest.mark.parametrize("ci,co", [(8, 32), (32, 16), (16, 32)])
def test_conv_matches_library_correlation(ci, co):
    rng = np.random.default_rng(ci * 100 + co)
    x = rnd(rng, 2, 5, 7, ci)
    w = rnd(rng, co, 3, 3, ci)
    b = rng.standard_normal(co)
    y = G.conv3x3(x, w, b)
    ref = np.zeros_like(y)
    for n in range(2):
        for o in range(co):
            for c in range(ci):
                ref[n, :, :, o] += scipy_signal.correlate2d(x[n, :, :, c], w[o, :, :, c], mode="same",
                                                            boundary="fill")
            ref[n, :, :, o] += b[o]
    assert np.abs(y - ref).max() < 1e-9


def test_identity_kernel_and_activation_mask():
    rng = np.random.default_rng(3)
    x = rnd(rng, 1, 4, 6, 16)
    w = np.zeros((16, 3, 3, 16))
    w[:, 1, 1, :] = np.eye(16)
    assert np.array_equal(G.conv3x3(x, w), x)
    assert np.array_equal(G.conv3x3(x, w, relu=True), np.maximum(x, 0))
    m = rnd(rng, 1, 4, 6, 16)
    assert np.array_equal(G.conv3x3(x, w, mask=m), np.where(m > 0, x, 0))


def test_flipped_weights_give_the_adjoint():
    """<conv(x, w), dy> = <x, conv(dy, flip(w))>: the input gradient."""
    rng = np.random.default_rng(4)
    x = rnd(rng, 2, 6, 5, 8)
    w = rnd(rng, 32, 3, 3, 8)
    dy = rnd(rng, 2, 6, 5, 32)
    lhs = (G.conv3x3(x, w) * dy).sum()
    rhs = (x * G.conv3x3(dy, G.flip(w))).sum()
    assert abs(lhs - rhs) < 1e-9 * (1 + abs(lhs))


def test_weight_gradient_by_exact_finite_differences():
    """L(w, b) = <conv(x, w, b), dy> is linear in w and b, so a unit step
    changes L by exactly the gradient entry."""
    rng = np.random.default_rng(5)
    x = rnd(rng, 1, 4, 5, 8)
    w = rnd(rng, 16, 3, 3, 8)
    b = rnd(rng, 16)
    dy = rnd(rng, 1, 4, 5, 16)
    dw, db = G.conv3x3_wgrad(x, dy)
    L0 = (G.conv3x3(x, w, b) * dy).sum()
    for idx in [(0, 0, 0, 0), (3, 1, 2, 7), (15, 2, 2, 5), (8, 0, 1, 3)]:
        w2 = w.copy()
        w2[idx] += 1.0
        assert abs((G.conv3x3(x, w2, b) * dy).sum() - L0 - dw[idx]) < 1e-9
    b2 = b.copy()
    b2[6] += 1.0
    assert abs((G.conv3x3(x, w, b2) * dy).sum() - L0 - db[6]) < 1e-9


def test_loss_adam_psnr_closed_forms():
    out = np.array([[0.5, 0.25, 1.0, 9.0]])
    tgt = np.array([[0.0, 0.5, 1.0, -3.0]])
    loss, g = G.loss_and_grad(out, tgt, 2.0)
    assert loss == 0.25 + 0.0625 and np.array_equal(g, [[1.0, -0.5, 0.0, 0.0]])
    # first Adam step moves every parameter by lr * g / (|g| + eps') against g
    p, gr = np.array([1.0, -2.0, 0.5]), np.array([0.3, -4.0, 1e-3])
    p1, m1, v1 = G.adam(p, gr, np.zeros(3), np.zeros(3), 0.01, 0.9, 0.999, 1e-12, 1)
    assert np.allclose(p1, p - 0.01 * np.sign(gr), atol=1e-9)
    assert np.allclose(m1, 0.1 * gr) and np.allclose(v1, 0.001 * gr * gr)
    assert abs(G.psnr(np.full((4, 3), 0.1), np.zeros((4, 3))) - 20.0) < 1e-12


def test_loss_gradient_with_base_by_central_differences():
    """The loss is quadratic in the output, so a central difference is its
    exact derivative: 2 (out + base - target) on RGB, 0 elsewhere."""
    rng = np.random.default_rng(5)
    out = np.round(rng.standard_normal((3, 16)) * 64) / 64
    base = np.round(rng.standard_normal((3, 8)) * 64) / 64
    tgt = np.round(rng.standard_normal((3, 4)) * 64) / 64
    _, g = G.loss_and_grad(out, tgt, 2.0, base)
    eps = 2.0 ** -6
    for i in range(3):
        for c in range(16):
            e = np.zeros_like(out)
            e[i, c] = eps
            lp, _ = G.loss_and_grad(out + e, tgt, 2.0, base)
            lm, _ = G.loss_and_grad(out - e, tgt, 2.0, base)
            assert abs((lp - lm) / (2 * eps) - g[i, c]) < 1e-9
    # the network predicts a residual: an output of target - base is exact
    exact = out.copy()
    exact[:, :3] = tgt[:, :3] - base[:, :3]
    l0, g0 = G.loss_and_grad(exact, tgt, 2.0, base)
    assert l0 == 0.0 and not g0.any()


def test_octahedral_decode_axes():
    codes = np.array([0x7FFF, 0x7FFF << 16, 0, 0x7FFF | (0x7FFF << 16)], np.uint32)
    n = G.oct_decode(codes)
    assert np.allclose(n[0], [1, 0, 0]) and np.allclose(n[1], [0, 1, 0]) and np.allclose(n[2], [0, 0, 1])
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0)


def test_splat_features_follow_the_splat():
    import oracle
    from paper_2211_15460_gb300 import scenes

    w = scenes.workload_spheres_256()
    rec, _, _ = oracle.fragments(w.scene, oracle.NORMAL, None, w.normal_pitch)
    pofa = oracle.pofa_sort(rec)
    cam = w.views[0]
    vis, rgba = oracle.render(pofa, w.scene, cam, w.lights, 1)
    f = G.splat_features(vis, rgba, pofa, cam)
    hit = vis != np.uint64(0xFFFFFFFFFFFFFFFF)
    assert np.array_equal(f[:, 4], hit.astype(np.float64))
    assert np.array_equal(f[hit, :3], rgba[hit, :3].astype(np.float64))
    assert (f[~hit] == 0).all()
    assert (f[hit, 3] > 0).all() and (f[hit, 3] < 1).all()
    assert (np.hypot(f[hit, 5], f[hit, 6]) <= 1.0 + 1e-12).all()


def _facing_quad_features(oracle, depth, normal, cam_axes, z0=-2.0, z1=2.0, W=12, H=10):
    """A square filling the view of a rotated orthographic camera, lying in
    the plane at `depth` along the camera's viewing direction, every vertex
    normal = `normal`; captured and splatted with that camera. Returns
    (features, hit mask)."""
    from paper_2211_15460_gb300 import scenes

    right, up, fwd = (np.asarray(a, np.float64) for a in cam_axes)
    origin = np.array([0.25, -0.5, 0.75])
    cam = scenes.Camera(origin=origin, right=right, up=up, fwd=fwd, pitch=1.0, width=W, height=H, z0=z0, z1=z1)
    corners = [(-W, -H), (W, -H), (W, H), (-W, H)]
    pos = np.array([origin + a * right + b * up + depth * fwd for a, b in corners])
    n = np.asarray(normal, np.float64) / np.linalg.norm(normal)
    sc = scenes.Scene(pos=pos, nrm=np.tile(n, (4, 1)), idx=np.array([[0, 1, 2], [0, 2, 3]]),
                      tri_material=np.zeros(2, np.uint32), albedo=np.ones((1, 3)),
                      cube_min=origin - 16.0, cube_side=32.0)
    rec, _, _ = oracle.fragments(sc, oracle.VIEW, cam, 0.0)
    light = scenes.directional_light(-fwd)[None]
    vis, rgba = oracle.render(rec, sc, cam, light, 1)
    hit = vis != np.uint64(0xFFFFFFFFFFFFFFFF)
    return G.splat_features(vis, rgba, rec, cam), hit


def _rotation(axis, angle):
    a = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def test_splat_features_depth_and_normal_closed_forms(oracle_mod):
    """Channel 3 is the visible point's depth along the view direction,
    normalised over the camera's [z0, z1] (the 24-bit code / 2^24, Section
    3.3's depth test); channels 5 and 6 are the visible surface normal's
    components along the camera's right and up axes. A square facing the
    camera at a known depth, with a known normal, fixes all three by
    geometry: (depth - z0) / (z1 - z0), n.right, n.up."""
    R = _rotation((0.3, 1.0, -0.4), 0.7)
    axes = (R @ [1.0, 0, 0], R @ [0, 1.0, 0], R @ [0, 0, -1.0])
    right, up, fwd = axes
    # normal with distinct components on right, up and the view direction
    n = 0.28 * right + 0.55 * up - 0.786 * fwd
    n /= np.linalg.norm(n)
    for depth in (-1.5, -0.25, 0.5, 1.25):
        f, hit = _facing_quad_features(oracle_mod, depth, n, axes)
        assert hit.all()
        # position quantum of the 32-unit cube is 2^-16 per axis: depth error <= sqrt(3) 2^-16 / 4
        assert np.abs(f[:, 3] - (depth + 2.0) / 4.0).max() < 2.0 ** -15
        # octahedral snorm16 code: each decoded component within 1e-4
        assert np.abs(f[:, 5] - n @ right).max() < 2e-4
        assert np.abs(f[:, 6] - n @ up).max() < 2e-4
    # depth order: nearer squares get smaller codes, linearly
    d = [float(_facing_quad_features(oracle_mod, z, n, axes)[0][0, 3]) for z in (-1.0, 0.0, 1.0)]
    assert abs((d[1] - d[0]) - 0.25) < 2.0 ** -14 and abs((d[2] - d[1]) - 0.25) < 2.0 ** -14
