"""Oracle of the learned gap-filler: plain fp64 numpy, written from the
definitions (test infrastructure only; the library never imports it).

The network has no counterpart in the paper; what it computes is fixed by
the definitions below:

* 3x3 convolution with zero padding, NHWC activations, weights
  w[co][ky][kx][ci]: y[n, i, j, co] = b[co] + sum over ky, kx, ci of
  x[n, i + ky - 1, j + kx - 1, ci] * w[co, ky, kx, ci]; then ReLU if asked,
  then y *= 1[mask > 0] if a mask is given;
* its weight gradient: dw[co, ky, kx, ci] = sum over n, i, j of
  dy[n, i, j, co] * x[n, i + ky - 1, j + kx - 1, ci]; db[co] = sum of dy;
* the input gradient is the convolution of dy with the flipped, transposed
  weights wf[ci][ky][kx][co] = w[co][2 - ky][2 - kx][ci];
* loss = sum over pixels and channels 0..2 of (out + base - target)^2, with
  base = the splat's RGB (the network predicts a residual) or 0, gradient
  grad_scale * (out + base - target); the image is out + base;
* Adam with bias correction;
* network inputs from a 1 x 1 splat: rgb, qd / 2^24, coverage, the visible
  record's normal projected on the camera's right and up axes.

BF16 rounding (round to nearest, ties to even) is provided so that tests can
compare with the device's stored BF16 values.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round float values to the nearest BF16 (ties to even), as float64."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(a) -> np.ndarray:
    """uint16 BF16 encodings of float values (round to nearest even)."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def from_bf16_bits(h) -> np.ndarray:
    """BF16 bit patterns (uint16) as float64 values: the top 16 bits of an FP32."""
    return (np.asarray(h, np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def conv3x3(x, w, b=None, relu=False, mask=None) -> np.ndarray:
    """Forward convolution (see the module docstring), fp64."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    n, h, wd, ci = x.shape
    co = w.shape[0]
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.zeros((n, h, wd, co))
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("nijc,oc->nijo", xp[:, ky:ky + h, kx:kx + wd, :], w[:, ky, kx, :])
    if b is not None:
        y += np.asarray(b, np.float64)
    if relu:
        y = np.maximum(y, 0.0)
    if mask is not None:
        y = np.where(np.asarray(mask) > 0, y, 0.0)
    return y


def conv3x3_wgrad(x, dy):
    """(dw, db) of the convolution, fp64."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    n, h, wd, ci = x.shape
    co = dy.shape[-1]
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    dw = np.zeros((co, 3, 3, ci))
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = np.einsum("nijo,nijc->oc", dy, xp[:, ky:ky + h, kx:kx + wd, :])
    return dw, dy.sum(axis=(0, 1, 2))


def flip(w) -> np.ndarray:
    """wf[ci][ky][kx][co] = w[co][2 - ky][2 - kx][ci]."""
    return np.ascontiguousarray(np.asarray(w)[:, ::-1, ::-1, :].transpose(3, 1, 2, 0))


def loss_and_grad(out, target, grad_scale=1.0, base=None):
    """out [..., >=3], target [..., >=3], base [..., >=3] or None: (sum of
    squared errors of out + base, gradient on channels 0..2, 0 elsewhere)."""
    out = np.asarray(out, np.float64)
    d = out[..., :3] - np.asarray(target, np.float64)[..., :3]
    if base is not None:
        d = d + np.asarray(base, np.float64)[..., :3]
    g = np.zeros_like(out)
    g[..., :3] = grad_scale * d
    return float((d * d).sum()), g


def adam(param, grad, m, v, lr, b1, b2, eps, step):
    """One bias-corrected Adam step: (param, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


def oct_decode(code):
    """Octahedral snorm16 pair to a unit normal, fp64 (codes uint32)."""
    code = np.asarray(code, np.uint32)
    x = (code & 0xFFFF).astype(np.uint16).view(np.int16).astype(np.float64) / 32767.0
    y = (code >> 16).astype(np.uint16).view(np.int16).astype(np.float64) / 32767.0
    z = 1.0 - np.abs(x) - np.abs(y)
    fold = z < 0
    qx = (1.0 - np.abs(y)) * np.where(x >= 0, 1.0, -1.0)
    qy = (1.0 - np.abs(x)) * np.where(y >= 0, 1.0, -1.0)
    x = np.where(fold, qx, x)
    y = np.where(fold, qy, y)
    n = np.stack([x, y, z], -1)
    return n / np.linalg.norm(n, axis=-1, keepdims=True)


def splat_features(vis, rgba, records, cam) -> np.ndarray:
    """Network input [H*W, 8] from a 1 x 1 splat's visibility and colours."""
    vis = np.asarray(vis, np.uint64)
    rgba = np.asarray(rgba, np.float64).reshape(-1, 4)
    f = np.zeros((vis.size, 8))
    hit = vis != np.uint64(0xFFFFFFFFFFFFFFFF)
    idx = (vis[hit] & np.uint64((1 << 40) - 1)).astype(np.int64)
    n = oct_decode(records["nrm"][idx])
    f[hit, 0:3] = rgba[hit, 0:3]
    f[hit, 3] = (vis[hit] >> np.uint64(40)).astype(np.float64) / 16777216.0
    f[hit, 4] = 1.0
    f[hit, 5] = n @ np.asarray(cam.right, np.float64)
    f[hit, 6] = n @ np.asarray(cam.up, np.float64)
    return f


def psnr(img, ref, peak=1.0) -> float:
    """Peak signal-to-noise ratio in dB of rgb images (channels 0..2)."""
    d = np.asarray(img, np.float64)[..., :3] - np.asarray(ref, np.float64)[..., :3]
    mse = float((d * d).mean())
    return float("inf") if mse == 0 else 10.0 * np.log10(peak * peak / mse)
