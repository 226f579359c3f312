"""Oracle of the dynamic-aperture surrogate network (test infrastructure only).

Plain numpy FP64 forward and backward of the MLP 16 -> 256 -> 256 -> 256 ->
256 -> 2 with exact (erf) GELU, the loss (binary cross-entropy on the
survival logit + masked squared error on the normalised log loss turn) and
Adam.  The paper cites dynamic-aperture estimates based on machine learning
(section "Lattice modelling and single particle tracking"); the network, its
inputs and its loss are this project's reading.

When ``bf16=True`` the oracle rounds to bfloat16 at the same points the GPU
kernels do (weights, layer inputs, activations, back-propagated
pre-activation gradients) and computes everything else in FP64, so it bounds
the GPU's FP32-accumulation error.  Only the tests and the benchmark's CPU
leg may use this module.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

WIDTHS = (16, 256, 256, 256, 256, 2)
N_LAYERS = len(WIDTHS) - 1


def param_shapes():
    """Flat parameter layout: W1 (256x16), b1, W2 (256x256), b2, ..., W5 (2x256), b5.
    W is stored (out, in)."""
    out = []
    for l in range(N_LAYERS):
        out.append((WIDTHS[l + 1], WIDTHS[l]))
        out.append((WIDTHS[l + 1],))
    return out


N_PARAMS = sum(int(np.prod(s)) for s in param_shapes())


def unflatten(flat):
    ps, o = [], 0
    for s in param_shapes():
        n = int(np.prod(s))
        ps.append(np.asarray(flat[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return ps


def flatten(ps):
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in ps])


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), via float32 as the GPU does."""
    a32 = np.asarray(a, dtype=np.float32)
    b = a32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + special.erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + special.erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def forward(flat, X, bf16_points: bool = True):
    """Returns the output (B x 2) and the cache for backward."""
    r = bf16 if bf16_points else (lambda v: np.asarray(v, dtype=np.float64))
    ps = unflatten(flat)
    a = r(X)
    cache = {"a": [a], "z": []}
    for l in range(N_LAYERS - 1):
        W, b = ps[2 * l], ps[2 * l + 1]
        z = a @ r(W).T + b
        a = r(gelu(z))
        cache["z"].append(z)
        cache["a"].append(a)
    W, b = ps[-2], ps[-1]
    out = a @ r(W).T + b
    return out, cache


def loss_and_dout(out, y, t, mask, lam):
    """L = mean_b BCE(logit_b, y_b) + lam * sum_b mask_b (pred_b - t_b)^2 / max(sum mask, 1)."""
    logit, pred = out[:, 0], out[:, 1]
    B = out.shape[0]
    nm = max(float(np.sum(mask)), 1.0)
    bce = np.maximum(logit, 0) - logit * y + np.log1p(np.exp(-np.abs(logit)))
    res = (pred - t) * mask
    L = float(np.mean(bce) + lam * np.sum(res * res) / nm)
    d = np.zeros_like(out)
    d[:, 0] = (special.expit(logit) - y) / B
    d[:, 1] = lam * 2.0 * res / nm
    return L, d


def backward(flat, cache, dout, bf16_points: bool = True):
    """Gradients of the loss with respect to the flat parameters."""
    r = bf16 if bf16_points else (lambda v: np.asarray(v, dtype=np.float64))
    ps = unflatten(flat)
    grads = [None] * len(ps)
    a = cache["a"]
    # head (FP32 CUDA-core layer on the GPU: no rounding of dout)
    grads[-2] = dout.T @ a[-1]
    grads[-1] = dout.sum(axis=0)
    dA = dout @ r(ps[-2])
    for l in range(N_LAYERS - 2, -1, -1):
        dZ = dA * gelu_grad(cache["z"][l])
        dZr = r(dZ)
        grads[2 * l] = dZr.T @ a[l]
        grads[2 * l + 1] = dZ.sum(axis=0)
        if l > 0:
            dA = dZr @ r(ps[2 * l])
    return flatten(grads)


def init_params(seed: int):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for weights and biases."""
    rng = np.random.default_rng(seed)
    ps = []
    for l in range(N_LAYERS):
        lim = 1.0 / math.sqrt(WIDTHS[l])
        ps.append(rng.uniform(-lim, lim, size=(WIDTHS[l + 1], WIDTHS[l])))
        ps.append(rng.uniform(-lim, lim, size=(WIDTHS[l + 1],)))
    return flatten(ps)


def adam(flat, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) with bias correction; returns new (flat, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
