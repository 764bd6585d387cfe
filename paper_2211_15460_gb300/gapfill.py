"""Learned gap-filler for sparse FHV splats (no counterpart in the paper).

A 6-layer 3x3 convolutional network (8 -> 32 -> 32 -> 32 -> 32 -> 32 -> 16
channels, ReLU between layers; the first 3 output channels are an RGB
correction added to the splat's RGB) fills the holes and undersampled gaps of
a 1 x 1 splat of an FHV -- here the PPFL captured from one view, seen from
another. Its input is the
splat's features (fhv_splat_features: RGB, depth, coverage, normal in the
camera frame); its target is a direct capture of the same view, i.e. a PPFL
captured with the view's own camera and splatted with that camera, which
keeps the nearest fragment per pixel (a z-buffer render; the identity-view
reprojection property). Training uses pairs the method itself produces.

Everything that computes runs in the library's kernels: BF16 tcgen05
convolutions (forward, input gradient through flipped weights, weight and
bias gradients), the loss and Adam. This module holds parameters and
buffers and sequences the calls.
"""
from __future__ import annotations

import math

import numpy as np

from . import fhv, scenes

LAYERS = [(8, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 16)]


def _bf16_bits(a: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


class GapFiller:
    """Parameters (FP32 master + BF16 copies), Adam state and activation
    buffers of the network on one device."""

    def __init__(self, seed: int = 0, device: str = "cuda"):
        import torch

        self.device = device
        rng = np.random.default_rng(seed)
        self.w32, self.b32, self.gw, self.gb = [], [], [], []
        self.mw, self.vw, self.mb, self.vb = [], [], [], []
        self.w16, self.wf16 = [], []
        for li, (ci, co) in enumerate(LAYERS):
            std = math.sqrt(2.0 / (9 * ci)) * (0.1 if li == len(LAYERS) - 1 else 1.0)
            w = (rng.standard_normal((co, 3, 3, ci)) * std).astype(np.float32)
            if ci == 8:
                w[..., 7] = 0.0  # the input's spare channel
            self.w32.append(torch.from_numpy(w.reshape(-1)).to(device))
            self.b32.append(torch.zeros(co, dtype=torch.float32, device=device))
            for lst, n in ((self.gw, w.size), (self.mw, w.size), (self.vw, w.size), (self.gb, co), (self.mb, co),
                           (self.vb, co)):
                lst.append(torch.zeros(n, dtype=torch.float32, device=device))
            self.w16.append(torch.from_numpy(_bf16_bits(w.reshape(-1)).view(np.int16)).to(device))
            self.wf16.append(torch.empty(w.size, dtype=torch.int16, device=device))
        self.ws = torch.zeros(256, dtype=torch.uint8, device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.steps = 0
        self._bufs = {}
        self._flip()

    def _flip(self, stream=None):
        for li, (ci, co) in enumerate(LAYERS):
            fhv.fhv_conv3x3_flip_bf16(self.w16[li], ci, co, self.wf16[li], stream)

    def buffers(self, n: int, h: int, w: int):
        """Activations a[0..6] (a[0] is the input) and gradients d[1..6]."""
        import torch

        key = (n, h, w)
        if key not in self._bufs:
            P = n * h * w
            acts = [None] + [torch.empty(P * co, dtype=torch.int16, device=self.device) for _, co in LAYERS]
            grads = [None] + [torch.empty(P * co, dtype=torch.int16, device=self.device) for _, co in LAYERS]
            self._bufs = {key: (acts, grads)}  # keep one shape resident
        return self._bufs[key]

    def forward(self, feat, n: int, h: int, w: int, stream=None):
        """feat: BF16 NHWC, 8 channels. Returns the activation list; the last
        entry holds the output (16 channels, RGB first)."""
        acts, _ = self.buffers(n, h, w)
        acts[0] = feat
        last = len(LAYERS) - 1
        for li, (ci, co) in enumerate(LAYERS):
            fhv.fhv_conv3x3_bf16(acts[li], n, h, w, ci, self.w16[li], self.b32[li], co, li < last, None, acts[li + 1],
                                 self.ws, stream)
        return acts

    def train_step(self, feat, target, n: int, h: int, w: int, lr: float, stream=None) -> None:
        """One step on a batch: forward, squared-error loss on RGB (its sum is
        added to self.loss), backward, Adam. The loss gradient is taken as
        out - target (Adam does not depend on its scale)."""
        acts, grads = self.buffers(n, h, w)
        self.forward(feat, n, h, w, stream)
        P = n * h * w
        fhv.fhv_gapfill_loss(acts[-1], feat, target, P, 1.0, self.loss, grads[len(LAYERS)], stream)
        for li in range(len(LAYERS) - 1, -1, -1):
            ci, co = LAYERS[li]
            fhv.fhv_conv3x3_wgrad_bf16(acts[li], grads[li + 1], n, h, w, ci, co, self.gw[li], self.gb[li], self.ws,
                                       stream)
            if li > 0:
                # input gradient, times the ReLU derivative of the layer's input
                fhv.fhv_conv3x3_bf16(grads[li + 1], n, h, w, co, self.wf16[li], None, ci, False, acts[li], grads[li],
                                     self.ws, stream)
        self.steps += 1
        for li in range(len(LAYERS)):
            fhv.fhv_adam_bf16(self.w32[li], self.gw[li], self.mw[li], self.vw[li], self.w32[li].numel(), lr, 0.9,
                              0.999, 1e-8, self.steps, self.w16[li], stream)
            fhv.fhv_adam_bf16(self.b32[li], self.gb[li], self.mb[li], self.vb[li], self.b32[li].numel(), lr, 0.9,
                              0.999, 1e-8, self.steps, None, stream)
        self._flip(stream)


# --------------------------------------------------------------- training data

class PairMaker:
    """Splat / direct-capture pairs of one scene's FHV at 1 x 1 footprint.

    The FHV is the PPFL captured from the capture camera (1-Pass/View): seen
    from another viewpoint its splat is sparse where surfaces were grazing in
    the capture view. A view is splatted into features; the target is the
    view's own PPFL capture splatted with the same camera (nearest fragment
    per pixel)."""

    def __init__(self, scene, capture, depth: int, lights, device="cuda"):
        import torch

        from .pipeline import PlainFHV

        self.scene = scene
        self.w = scenes.Workload("pairs", scene, capture, depth, [capture], lights)
        self.p = PlainFHV(self.w, device=device)
        self.p.capture_ppfl()
        self.n = fhv.fhv_get_count(self.p.ppfl)[1]
        self.lights = self.p.lights
        self.device = device
        self.ws = fhv.workspace(fhv.FHV_RENDER_WS_BYTES, device)
        self._cap = {}
        self.torch = torch

    def _frags(self, cam):
        key = (cam.width, cam.height)
        if key not in self._cap:
            torch = self.torch
            head = torch.empty(cam.width * cam.height, dtype=torch.int32, device=self.device)
            cap = max(1 << 16, cam.width * cam.height * 16)
            fb = fhv.FragBuf(cap, self.device)
            wsb = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_PPFL, self.scene.n_tri, cam.width, cam.height, 1, 0)
            self._cap[key] = [head, fb, fhv.workspace(wsb.workspace_bytes, self.device)]
        return self._cap[key]

    def make(self, cam, feat_out, target_out, vis, rgba, stream=None) -> None:
        """Features of the FHV splat into feat_out (BF16 NHWC 8) and the
        direct capture's RGBA into target_out (FP32 [H*W*4])."""
        p = self.p
        fhv.fhv_render_view(p.ppfl.rec, p.ppfl.capacity, p.ppfl.count, p.scene, p.scene.albedo, self.lights,
                            p.n_lights, cam, 1, vis, rgba, self.ws, stream)
        fhv.fhv_splat_features(vis, rgba, p.ppfl.rec, cam, feat_out, stream)
        head, fb, wsb = self._frags(cam)
        fhv.fhv_capture_ppfl(p.scene, cam, head, fb, wsb, stream)
        fhv.fhv_render_view(fb.rec, fb.capacity, fb.count, p.scene, p.scene.albedo, self.lights, p.n_lights, cam, 1,
                            vis, target_out, self.ws, stream)


def crop_camera(cam, x0: int, y0: int, cw: int, ch: int):
    """The camera of the cw x ch window at pixel (x0, y0) of `cam` (same pitch)."""
    c = scenes.Camera(cam.origin, cam.right, cam.up, cam.fwd, cam.pitch, cw, ch, cam.z0, cam.z1)
    dx = (x0 + cw / 2.0) - cam.width / 2.0
    dy = (y0 + ch / 2.0) - cam.height / 2.0
    o = (cam.origin.astype(np.float64) + dx * float(cam.pitch) * cam.right.astype(np.float64)
         + dy * float(cam.pitch) * cam.up.astype(np.float64))
    c.origin = o.astype(np.float32)
    return c


def spheres_light():
    """The directional light of the sphere scenes the pairs are made from."""
    return scenes.directional_light((1.0, 1.0, 1.0))[None]


def make_dataset(n_crops: int, seed: int = 0, res: int = 256, crop: int = 128, views_per_scene: int = 16,
                 depth: int = 6, device="cuda"):
    """n_crops (features, targets) of crop x crop pixels from config-1-style
    scenes (8 seeded UV-spheres): per scene a res x res capture, views at
    orbit offsets of +-U[10, 60] degrees, each view split into its
    (res / crop)^2 windows. Returns (feat [n][crop][crop][8] BF16,
    target [n][crop*crop*4] FP32)."""
    import torch

    per_view = (res // crop) ** 2
    feat = torch.empty((n_crops, crop, crop, 8), dtype=torch.int16, device=device)
    tgt = torch.empty((n_crops, crop * crop * 4), dtype=torch.float32, device=device)
    vis = torch.empty(crop * crop, dtype=torch.int64, device=device)
    rgba = torch.empty(crop * crop * 4, dtype=torch.float32, device=device)
    rng = np.random.default_rng(seed)
    k = 0
    s = 0
    while k < n_crops:
        sc = scenes.spheres_scene(seed * 100003 + s)
        cap = scenes.orbit_camera(sc, res, res)
        pm = PairMaker(sc, cap, depth, spheres_light(), device)
        for _ in range(views_per_scene):
            if k >= n_crops:
                break
            deg = float(rng.uniform(10.0, 60.0)) * (1.0 if rng.random() < 0.5 else -1.0)
            view = scenes.orbit_camera(sc, res, res, orbit_deg=deg)
            for q in range(per_view):
                if k >= n_crops:
                    break
                qx, qy = q % (res // crop), q // (res // crop)
                pm.make(crop_camera(view, qx * crop, qy * crop, crop, crop), feat[k], tgt[k], vis, rgba)
                k += 1
        s += 1
    return feat, tgt


def train(net: GapFiller, feat, tgt, epochs: int, batch: int = 64, lr: float = 2e-3, seed: int = 0,
          log=None) -> list:
    """Shuffled mini-batches over the crops; returns the mean squared error
    (per RGB channel) of every epoch."""
    import torch

    n, h, w, _ = feat.shape
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    hist = []
    bf = torch.empty((batch, h, w, 8), dtype=torch.int16, device=feat.device)
    bt = torch.empty((batch, h * w * 4), dtype=torch.float32, device=feat.device)
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(feat.device)
        net.loss.zero_()
        seen = 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            torch.index_select(feat, 0, idx, out=bf)
            torch.index_select(tgt, 0, idx, out=bt)
            net.train_step(bf, bt, batch, h, w, lr)
            seen += batch * h * w
        torch.cuda.synchronize()
        mse = net.loss.item() / max(1, 3 * seen)
        hist.append(mse)
        if log:
            log(ep, mse)
    return hist


def evaluate(net: GapFiller, feat, tgt, n: int, h: int, w: int):
    """(mse of the plain splat, mse of the gap-filled image) per RGB channel
    against the targets."""
    import torch

    acts = net.forward(feat, n, h, w)
    out = torch.zeros(1, dtype=torch.float64, device=feat.device)
    fhv.fhv_gapfill_loss(acts[-1], feat, tgt, n * h * w, 1.0, out, None)
    # the plain splat: a zero correction on top of the splat's RGB
    zero = torch.zeros(n * h * w * 16, dtype=torch.int16, device=feat.device)
    base = torch.zeros(1, dtype=torch.float64, device=feat.device)
    fhv.fhv_gapfill_loss(zero, feat, tgt, n * h * w, 1.0, base, None)
    torch.cuda.synchronize()
    P3 = 3.0 * n * h * w
    return base.item() / P3, out.item() / P3


def psnr(mse: float) -> float:
    """Peak signal-to-noise ratio in dB of a mean squared error on [0, 1] colours."""
    return float("inf") if mse <= 0 else 10.0 * math.log10(1.0 / mse)


def time_conv(cin: int, cout: int, h: int, w: int, reps: int, seed: int = 0) -> dict:
    """Times one convolution layer (ReLU on) on random BF16 data with CUDA
    events after three warm-up calls."""
    import torch

    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    x = (torch.randn(h * w * cin, generator=g) * 0.5).to(torch.bfloat16).view(torch.int16).cuda()
    wt = (torch.randn(cout * 9 * cin, generator=g) * 0.1).to(torch.bfloat16).view(torch.int16).cuda()
    b = torch.zeros(cout, device="cuda")
    y = torch.empty(h * w * cout, dtype=torch.int16, device="cuda")
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        fhv.fhv_conv3x3_bf16(x, 1, h, w, cin, wt, b, cout, True, None, y, ws)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fhv.fhv_conv3x3_bf16(x, 1, h, w, cin, wt, b, cout, True, None, y, ws)
    e.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(e) / reps
    flops = 2.0 * 9 * cin * cout * h * w
    return {"cin": cin, "cout": cout, "h": h, "w": w, "ms": ms, "tflops": flops / ms / 1e9,
            "status": fhv.fhv_read_status(ws)[1]}


def time_wgrad(cin: int, cout: int, n: int, h: int, w: int, reps: int, seed: int = 0) -> dict:
    """Times the weight gradient of one layer on random BF16 activations and
    output gradients (a training batch is n crops of h x w) with CUDA events
    after three warm-up calls."""
    import torch

    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    x = (torch.randn(n * h * w * cin, generator=g) * 0.5).to(torch.bfloat16).view(torch.int16).cuda()
    dy = (torch.randn(n * h * w * cout, generator=g) * 0.5).to(torch.bfloat16).view(torch.int16).cuda()
    dw = torch.zeros(cout * 9 * cin, device="cuda")
    db = torch.zeros(cout, device="cuda")
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        fhv.fhv_conv3x3_wgrad_bf16(x, dy, n, h, w, cin, cout, dw, db, ws)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fhv.fhv_conv3x3_wgrad_bf16(x, dy, n, h, w, cin, cout, dw, db, ws)
    e.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(e) / reps
    flops = 2.0 * 9 * cin * cout * n * h * w
    return {"wgrad": True, "cin": cin, "cout": cout, "n": n, "h": h, "w": w, "ms": ms, "tflops": flops / ms / 1e9,
            "gbs": n * h * w * (cin + cout) * 2 / ms / 1e6, "status": fhv.fhv_read_status(ws)[1]}


def time_network(h: int, w: int, reps: int, seed: int = 0) -> dict:
    """Times the whole network's forward pass (six convolutions) on random
    BF16 features with freshly initialised weights, CUDA events around each
    pass after three warm-up passes."""
    import torch

    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    feat = (torch.rand(h * w * 8, generator=g)).to(torch.bfloat16).view(torch.int16).cuda()
    net = GapFiller(seed=seed)
    for _ in range(3):
        net.forward(feat, 1, h, w)
    ms = []
    for _ in range(reps):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        net.forward(feat, 1, h, w)
        e.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(e))
    flops = sum(2.0 * 9 * ci * co for ci, co in LAYERS) * h * w
    nbytes = sum((ci + co) * 2 for ci, co in LAYERS) * h * w
    best = min(ms)
    return {"network": LAYERS, "h": h, "w": w, "ms_min": best, "ms_mean": sum(ms) / len(ms),
            "tflops": flops / best / 1e9, "gbs": nbytes / best / 1e6, "status": fhv.fhv_read_status(net.ws)[1]}


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="time one gap-filler convolution layer, its weight gradient, or the "
                                             "whole network")
    ap.add_argument("--cin", type=int, default=32)
    ap.add_argument("--cout", type=int, default=32)
    ap.add_argument("--h", type=int, default=1080)
    ap.add_argument("--w", type=int, default=1920)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--network", action="store_true", help="the six-layer forward pass instead of one layer")
    ap.add_argument("--wgrad", action="store_true", help="the weight gradient of one layer over a training batch")
    ap.add_argument("--batch", type=int, default=64, help="--wgrad: crops per batch")
    args = ap.parse_args()
    if args.wgrad:
        print(json.dumps(time_wgrad(args.cin, args.cout, args.batch, args.h, args.w, args.reps)))
    elif args.network:
        print(json.dumps(time_network(args.h, args.w, args.reps)))
    else:
        print(json.dumps(time_conv(args.cin, args.cout, args.h, args.w, args.reps)))
