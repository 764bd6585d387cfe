"""Gap-filler training path on the GPU: the training pairs against the
oracle (features of the FHV splat; the target is the view's own capture
splatted with its camera), one training step's gradients against the fp64
oracle of the whole network, and a short training run that must beat the
plain splat on held-out views."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import gapfill as G  # noqa: E402
from paper_2211_15460_gb300 import fhv, gapfill, scenes  # noqa: E402


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def test_pairs_against_oracle(orc):
    sc = scenes.spheres_scene(77)
    cap = scenes.orbit_camera(sc, 256, 256)
    pm = gapfill.PairMaker(sc, cap, 6, gapfill.spheres_light())
    view = scenes.orbit_camera(sc, 256, 256, orbit_deg=-37.0)
    cam = gapfill.crop_camera(view, 128, 0, 128, 128)
    feat = torch.empty((128, 128, 8), dtype=torch.int16, device="cuda")
    tgt = torch.empty(128 * 128 * 4, dtype=torch.float32, device="cuda")
    vis = torch.empty(128 * 128, dtype=torch.int64, device="cuda")
    rgba = torch.empty(128 * 128 * 4, dtype=torch.float32, device="cuda")
    pm.make(cam, feat, tgt, vis, rgba)
    torch.cuda.synchronize()
    L = gapfill.spheres_light()
    # the FHV: PPFL of the capture view, splatted from the crop's camera
    nc, _, crec, _ = orc.ppfl(sc, cap, 1 << 22)
    vis_o, rgba_o = orc.render(crec[:nc], sc, cam, L, 1)
    ref_f = G.splat_features(vis_o, rgba_o, crec[:nc], cam)
    got_f = G.from_bf16_bits(feat.cpu().numpy().view(np.uint16)).reshape(-1, 8)
    assert np.array_equal(got_f[:, 4], ref_f[:, 4])
    assert (np.abs(got_f - ref_f) <= np.abs(ref_f) * 2.0 ** -7 + 2e-4).all()
    # direct capture from the view, nearest fragment per pixel
    n, head, prec, nxt = orc.ppfl(sc, cam, 1 << 20)
    vis_t, rgba_t = orc.render(prec[:n], sc, cam, L, 1)
    assert np.abs(tgt.cpu().numpy().reshape(-1, 4) - rgba_t).max() < 1e-4
    # where the capture view grazed a surface, the splat shows a farther
    # surface or nothing: many pixels differ from the direct capture
    assert (np.abs(rgba_o[:, :3] - rgba_t[:, :3]).max(axis=1) > 0.05).sum() > 20


def oracle_network_grads(net, x, tgt):
    """fp64 forward/backward of the whole network with BF16 storage of every
    activation and activation gradient (as the device stores them)."""
    w = [G.from_bf16_bits(t.cpu().numpy().view(np.uint16)).reshape(co, 3, 3, ci)
         for t, (ci, co) in zip(net.w16, gapfill.LAYERS)]
    b = [t.cpu().numpy().astype(np.float64) for t in net.b32]
    acts = [x]
    for li in range(6):
        acts.append(G.bf16_round(G.conv3x3(acts[-1], w[li], b[li], relu=li < 5)))
    _, g = G.loss_and_grad(acts[-1], tgt, 1.0, x)
    d = G.bf16_round(g)
    dws = [None] * 6
    for li in range(5, -1, -1):
        dws[li] = G.conv3x3_wgrad(acts[li], d)
        if li > 0:
            d = G.bf16_round(G.conv3x3(d, G.flip(w[li]), mask=acts[li]))
    return dws


def test_train_step_gradients_against_oracle():
    net = gapfill.GapFiller(seed=3)
    rng = np.random.default_rng(5)
    n, h, w = 2, 6, 20
    x = np.zeros((n, h, w, 8))
    x[..., :7] = G.bf16_round(rng.random((n, h, w, 7)))
    tgt = rng.random((n, h, w, 4)).astype(np.float32)
    ref = oracle_network_grads(net, x, tgt.astype(np.float64))
    dx = torch.from_numpy(G.bf16_bits(x).view(np.int16)).cuda()
    dt = torch.from_numpy(tgt.reshape(-1)).cuda()
    # one step with lr = 0 leaves the weights; read the gradients before Adam clears them
    acts, grads = net.buffers(n, h, w)
    net.forward(dx, n, h, w)
    fhv.fhv_gapfill_loss(acts[-1], dx, dt, n * h * w, 1.0, net.loss, grads[6])
    for li in range(5, -1, -1):
        ci, co = gapfill.LAYERS[li]
        fhv.fhv_conv3x3_wgrad_bf16(acts[li], grads[li + 1], n, h, w, ci, co, net.gw[li], net.gb[li], net.ws)
        if li > 0:
            fhv.fhv_conv3x3_bf16(grads[li + 1], n, h, w, co, net.wf16[li], None, ci, False, acts[li], grads[li],
                                 net.ws)
    torch.cuda.synchronize()
    assert fhv.fhv_read_status(net.ws) == (fhv.FHV_OK, 0)
    for li in range(6):
        rw, rb = ref[li]
        gw = net.gw[li].cpu().numpy().astype(np.float64).reshape(rw.shape)
        gb = net.gb[li].cpu().numpy().astype(np.float64)
        scale = np.abs(rw).max() + 1e-12
        # BF16 storage between layers: a rounding that flips on one side
        # propagates, so compare to 2 % of the layer's largest entry
        assert np.abs(gw - rw).max() <= 2e-2 * scale, li
        assert np.abs(gb - rb).max() <= 2e-2 * (np.abs(rb).max() + 1e-12), li


def test_short_training_beats_the_plain_splat():
    feat, tgt = gapfill.make_dataset(512, seed=1)
    vf, vt = gapfill.make_dataset(64, seed=2)  # other scenes
    net = gapfill.GapFiller(seed=0)
    hist = gapfill.train(net, feat, tgt, epochs=6, batch=32, lr=2e-3)
    assert hist[-1] < hist[0]
    base, learned = gapfill.evaluate(net, vf, vt, vf.shape[0], 128, 128)
    assert learned < base, (base, learned)
    assert fhv.fhv_read_status(net.ws) == (fhv.FHV_OK, 0)
