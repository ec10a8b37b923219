"""FP64 CPU oracle of the learned warm-start network (a small U-Net).

TEST INFRASTRUCTURE ONLY: the test suite imports it to check the CUDA layer kernels and
the full network's forward pass and gradients.  The paper has no learned component; the
network is the one the warm-start workload specifies: a 3-level U-Net with 16/32/64
channels; input = 2 channels (the back projection of a noisy sinogram and a CGLS image of
it), outputs = a warm-start image channel and a per-pixel edge-weight map.

Layout here is channels-first ([C][H][W]) float64, written for reading against the
definitions:
  conv3x3:   y[o, i, j] = b[o] + sum_{c, u, v} W[o, c, u, v] x[c, i + u - 1, j + v - 1]
             (zero outside the image)
  maxpool2:  y[c, i, j] = max of x[c, 2i:2i+2, 2j:2j+2]
  upsample2: y[c, i, j] = x[c, i // 2, j // 2]
  head:      o[k, i, j] = hb[k] + sum_c hW[k, c] x[c, i, j];  f0 = o[0];  w = sigmoid(o[1])
  loss:      mean((f0 - f_t)^2) + mean((w - w_t)^2)
  warm start served to the solver: f^(0) = max(base + scale * o0, 0), with base the CGLS
             image the network corrects (the image channel is a residual on it)
"""
from __future__ import annotations

import numpy as np

# (in, out) channels of the 3x3 convolutions, in order; every one is followed by ReLU
CONVS = [(2, 16), (16, 16),          # encoder level 1 (full resolution) -> skip 1
         (16, 32), (32, 32),         # encoder level 2 (1/2)            -> skip 2
         (32, 64), (64, 64),         # bottleneck (1/4)
         (96, 32), (32, 32),         # decoder level 2: [upsampled 64, skip 32]
         (48, 16), (16, 16)]         # decoder level 1: [upsampled 32, skip 16]
HEAD = (16, 2)


def conv3x3(x, W, b):
    C, H, Wd = x.shape
    xp = np.zeros((C, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.empty((W.shape[0], H, Wd))
    for o in range(W.shape[0]):
        acc = np.full((H, Wd), float(b[o]))
        for c in range(C):
            for u in range(3):
                for v in range(3):
                    acc += W[o, c, u, v] * xp[c, u:u + H, v:v + Wd]
        y[o] = acc
    return y


def conv3x3_backward(x, W, dy):
    """Gradients of conv3x3 w.r.t. its input, weights and bias."""
    C, H, Wd = x.shape
    xp = np.zeros((C, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for o in range(W.shape[0]):
        for c in range(C):
            for u in range(3):
                for v in range(3):
                    dW[o, c, u, v] = np.sum(dy[o] * xp[c, u:u + H, v:v + Wd])
                    dxp[c, u:u + H, v:v + Wd] += W[o, c, u, v] * dy[o]
    return dxp[:, 1:-1, 1:-1], dW, dy.sum(axis=(1, 2))


def maxpool2(x):
    C, H, Wd = x.shape
    return x.reshape(C, H // 2, 2, Wd // 2, 2).max(axis=(2, 4))


def maxpool2_backward(x, dy):
    """Routes each gradient to the first maximum of its 2x2 window (row-major order)."""
    C, H, Wd = x.shape
    dx = np.zeros_like(x)
    for c in range(C):
        for i in range(H // 2):
            for j in range(Wd // 2):
                win = x[c, 2 * i:2 * i + 2, 2 * j:2 * j + 2].ravel()
                k = int(np.argmax(win))
                dx[c, 2 * i + k // 2, 2 * j + k % 2] += dy[c, i, j]
    return dx


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


def upsample2_backward(dy):
    C, H, Wd = dy.shape
    return dy.reshape(C, H // 2, 2, Wd // 2, 2).sum(axis=(2, 4))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def warm_start(o0, base, scale: float):
    """The solver's start image from the network's image channel: the channel is a
    residual on the base image in units of `scale`, clamped to the constraint f >= 0
    of Eq. (2)."""
    return np.maximum(np.asarray(base, dtype=np.float64) + scale * np.asarray(o0, dtype=np.float64), 0.0)


def init_params(seed: int):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for ci, co in CONVS:
        W = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        params.append([W, np.zeros(co)])
    params.append([rng.standard_normal(HEAD[::-1]) * np.sqrt(1.0 / HEAD[0]), np.zeros(HEAD[1])])
    return params


def forward(params, x):
    """x: [2][H][W] -> (f0 [H][W], w [H][W], cache)."""
    cache = {"acts": []}
    h = x
    acts = []

    def conv(k, h):
        W, b = params[k]
        z = conv3x3(h, W, b)
        a = np.maximum(z, 0.0)
        acts.append((h, z))
        return a

    e1 = conv(1, conv(0, h))
    e2 = conv(3, conv(2, maxpool2(e1)))
    bt = conv(5, conv(4, maxpool2(e2)))
    d2 = conv(7, conv(6, np.concatenate([upsample2(bt), e2], axis=0)))
    d1 = conv(9, conv(8, np.concatenate([upsample2(d2), e1], axis=0)))
    hW, hb = params[10]
    o = np.einsum("kc,cij->kij", hW, d1) + hb[:, None, None]
    cache.update(acts=acts, e1=e1, e2=e2, bt=bt, d2=d2, d1=d1, o=o)
    return o[0], sigmoid(o[1]), cache


def loss_and_grads(params, x, f_t, w_t):
    """Loss and its gradients w.r.t. every parameter (list like params)."""
    f0, w, c = forward(params, x)
    n = f0.size
    loss = float(np.mean((f0 - f_t) ** 2) + np.mean((w - w_t) ** 2))
    do = np.stack([2.0 * (f0 - f_t) / n, 2.0 * (w - w_t) / n * w * (1.0 - w)])
    grads = [None] * len(params)
    hW, _ = params[10]
    grads[10] = [np.einsum("kij,cij->kc", do, c["d1"]), do.sum(axis=(1, 2))]
    dh = np.einsum("kc,kij->cij", hW, do)
    acts = c["acts"]

    def conv_back(k, dact):
        h, z = acts[k]
        dz = dact * (z > 0)
        dx, dW, db = conv3x3_backward(h, params[k][0], dz)
        grads[k] = [dW, db]
        return dx

    dcat1 = conv_back(8, conv_back(9, dh))              # [32 up + 16 skip]
    dd2 = upsample2_backward(dcat1[:32])
    de1 = dcat1[32:]
    dcat2 = conv_back(6, conv_back(7, dd2))             # [64 up + 32 skip]
    dbt = upsample2_backward(dcat2[:64])
    de2 = dcat2[64:]
    dp2 = conv_back(4, conv_back(5, dbt))
    de2 = de2 + maxpool2_backward(c["e2"], dp2)
    dp1 = conv_back(2, conv_back(3, de2))
    de1 = de1 + maxpool2_backward(c["e1"], dp1)
    conv_back(0, conv_back(1, de1))
    return loss, grads
