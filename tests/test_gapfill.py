"""Gap-filler kernels (tcgen05 convolutions, weight gradient, flip, loss,
Adam, splat features) through the C ABI against the fp64 oracle.

Tolerances follow the arithmetic: the convolution multiplies BF16 values
exactly and accumulates at most 288 products in FP32 (relative error ~2e-5 of
the sum of |terms|) before one rounding to BF16, so an output may differ from
the oracle's correctly rounded value by one BF16 step where the FP32 sum
straddles a rounding boundary. Weight gradients are FP32 sums over pixels
(different order, atomics): 1e-5 of the sum of |terms|.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import gapfill as G  # noqa: E402
from paper_2211_15460_gb300 import fhv  # noqa: E402


def to_dev_bf16(a):
    return torch.from_numpy(G.bf16_bits(a).view(np.int16)).cuda()


def from_dev_bf16(t):
    return G.from_bf16_bits(t.cpu().numpy().view(np.uint16))


def rnd(rng, *shape, scale=1.0):
    return G.bf16_round(scale * rng.standard_normal(shape))


def ws():
    return torch.zeros(256, dtype=torch.uint8, device="cuda")


def bf16_close(got, ref):
    """At most one BF16 step apart (relative 2^-7 of the larger magnitude, or
    tiny absolute near zero)."""
    err = np.abs(got - ref)
    bound = np.maximum(np.abs(got), np.abs(ref)) * 2.0 ** -7 + 1e-6
    return bool((err <= bound).all()), float((err / bound).max())


SHAPES = [(1, 1, 1), (1, 3, 128), (2, 5, 130), (1, 4, 257), (3, 2, 37)]
PAIRS = [(8, 32), (8, 16), (16, 32), (16, 16), (32, 32), (32, 16)]


@pytest.mark.parametrize("ci,co", PAIRS)
@pytest.mark.parametrize("shape", SHAPES)
def test_conv_forward(ci, co, shape):
    n, h, w = shape
    rng = np.random.default_rng(ci * 1000 + co * 10 + h + w)
    x = rnd(rng, n, h, w, ci)
    wt = rnd(rng, co, 3, 3, ci, scale=0.2)
    b = rng.standard_normal(co).astype(np.float32)
    mask = rnd(rng, n, h, w, co)
    y = torch.empty(n * h * w * co, dtype=torch.int16, device="cuda")
    w_ = ws()
    for relu, use_mask, use_bias in ((False, False, False), (True, False, True), (False, True, True)):
        y.fill_(0x7FC0)  # NaN pattern: every output must be written
        fhv.fhv_conv3x3_bf16(to_dev_bf16(x), n, h, w, ci, to_dev_bf16(wt),
                             torch.from_numpy(b).cuda() if use_bias else None, co, relu,
                             to_dev_bf16(mask) if use_mask else None, y, w_)
        torch.cuda.synchronize()
        ref = G.conv3x3(x, wt, b.astype(np.float64) if use_bias else None, relu, mask if use_mask else None)
        got = from_dev_bf16(y).reshape(n, h, w, co)
        ok, worst = bf16_close(got, ref)
        assert ok, (relu, use_mask, use_bias, worst)
    assert fhv.fhv_read_status(w_) == (fhv.FHV_OK, 0)


@pytest.mark.parametrize("ci,co", PAIRS)
@pytest.mark.parametrize("shape", [(1, 3, 128), (2, 5, 130), (1, 33, 71), (4, 16, 16)])
def test_conv_weight_gradient(ci, co, shape):
    n, h, w = shape
    rng = np.random.default_rng(ci * 7 + co + h * w)
    x = rnd(rng, n, h, w, ci)
    dy = rnd(rng, n, h, w, co)
    dw = torch.zeros(co * 9 * ci, dtype=torch.float32, device="cuda")
    db = torch.zeros(co, dtype=torch.float32, device="cuda")
    w_ = ws()
    fhv.fhv_conv3x3_wgrad_bf16(to_dev_bf16(x), to_dev_bf16(dy), n, h, w, ci, co, dw, db, w_)
    torch.cuda.synchronize()
    assert fhv.fhv_read_status(w_) == (fhv.FHV_OK, 0)
    ref_w, ref_b = G.conv3x3_wgrad(x, dy)
    mag_w, mag_b = G.conv3x3_wgrad(np.abs(x), np.abs(dy))
    gw = dw.cpu().numpy().astype(np.float64).reshape(co, 3, 3, ci)
    gb = db.cpu().numpy().astype(np.float64)
    assert (np.abs(gw - ref_w) <= 1e-5 * mag_w + 1e-6).all()
    assert (np.abs(gb - ref_b) <= 1e-5 * mag_b + 1e-6).all()


@pytest.mark.parametrize("ci,co", [(32, 32), (16, 32), (32, 16)])
def test_input_gradient_through_flipped_weights(ci, co):
    """dX = conv(dY, flip(W)) masked by the layer input, as the backward pass
    runs it; the flip itself is exact."""
    rng = np.random.default_rng(ci + 3 * co)
    n, h, w = 2, 7, 131
    x_prev = G.bf16_round(np.maximum(rng.standard_normal((n, h, w, ci)), 0))  # a ReLU output
    wt = rnd(rng, co, 3, 3, ci, scale=0.2)
    dy = rnd(rng, n, h, w, co)
    wf = torch.empty(9 * ci * co, dtype=torch.int16, device="cuda")
    fhv.fhv_conv3x3_flip_bf16(to_dev_bf16(wt), ci, co, wf)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev_bf16(wf).reshape(ci, 3, 3, co), G.flip(wt))
    dx = torch.empty(n * h * w * ci, dtype=torch.int16, device="cuda")
    w_ = ws()
    fhv.fhv_conv3x3_bf16(to_dev_bf16(dy), n, h, w, co, wf, None, ci, False, to_dev_bf16(x_prev), dx, w_)
    torch.cuda.synchronize()
    ref = G.conv3x3(dy, G.flip(wt), mask=x_prev)
    ok, worst = bf16_close(from_dev_bf16(dx).reshape(n, h, w, ci), ref)
    assert ok, worst


def test_loss_and_adam():
    rng = np.random.default_rng(9)
    P = 1000
    out = rnd(rng, P, 16)
    tgt = rng.random((P, 4)).astype(np.float32)
    grad = torch.empty(P * 16, dtype=torch.int16, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    base = rnd(rng, P, 8)
    for b in (None, base):
        loss.zero_()
        fhv.fhv_gapfill_loss(to_dev_bf16(out), None if b is None else to_dev_bf16(b), torch.from_numpy(tgt).cuda(), P,
                             0.5, loss, grad)
        torch.cuda.synchronize()
        ref_l, ref_g = G.loss_and_grad(out, tgt.astype(np.float64), 0.5, b)
        assert abs(loss.item() - ref_l) < 1e-6 * ref_l
        ok, worst = bf16_close(from_dev_bf16(grad).reshape(P, 16), ref_g)
        assert ok, worst
    img = torch.empty(P * 4, dtype=torch.float32, device="cuda")
    fhv.fhv_gapfill_compose(to_dev_bf16(out), to_dev_bf16(base), P, img)
    torch.cuda.synchronize()
    ref_img = out[:, :3] + base[:, :3]
    assert np.abs(img.cpu().numpy().reshape(P, 4)[:, :3] - ref_img).max() <= 1e-6 * np.abs(ref_img).max()
    assert (img.cpu().numpy().reshape(P, 4)[:, 3] == 1).all()
    n = 4099
    p = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    m = (0.1 * rng.standard_normal(n)).astype(np.float32)
    v = (rng.random(n) * 0.01).astype(np.float32)
    dp, dg, dm, dv = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    out16 = torch.empty(n, dtype=torch.int16, device="cuda")
    fhv.fhv_adam_bf16(dp, dg, dm, dv, n, 1e-3, 0.9, 0.999, 1e-8, 7, out16)
    torch.cuda.synchronize()
    rp, rm, rv = G.adam(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64), v.astype(np.float64), 1e-3,
                        0.9, 0.999, 1e-8, 7)
    assert np.abs(dp.cpu().numpy() - rp).max() < 1e-5
    assert np.abs(dm.cpu().numpy() - rm).max() < 1e-6 and np.abs(dv.cpu().numpy() - rv).max() < 1e-6
    assert (dg.cpu().numpy() == 0).all()
    assert np.array_equal(from_dev_bf16(out16), G.bf16_round(dp.cpu().numpy()))


def test_splat_features_against_oracle():
    import oracle
    from paper_2211_15460_gb300 import scenes
    from paper_2211_15460_gb300.pipeline import PlainFHV

    w = scenes.workload_spheres_256()
    p = PlainFHV(w)
    p.build()
    p.render(0)
    torch.cuda.synchronize()
    cam = w.views[0]
    feat = torch.empty(cam.width * cam.height * 8, dtype=torch.int16, device="cuda")
    fhv.fhv_splat_features(p.vis[0], p.rgba[0], p.pofa, cam, feat)
    torch.cuda.synchronize()
    rec, _, _ = oracle.fragments(w.scene, oracle.NORMAL, None, w.normal_pitch)
    pofa = oracle.pofa_sort(rec)
    vis, rgba = oracle.render(pofa, w.scene, cam, w.lights, 1)
    ref = G.splat_features(vis, rgba, pofa, cam)
    got = from_dev_bf16(feat).reshape(-1, 8)
    # colours and normals within the render tolerance before one BF16 rounding
    err = np.abs(got - ref)
    assert (err <= np.abs(ref) * 2.0 ** -7 + 2e-4).all(), err.max()
    assert np.array_equal(got[:, 4], ref[:, 4])
