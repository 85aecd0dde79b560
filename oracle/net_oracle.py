"""CPU FP64 oracle of the learned initial guess / preconditioner network.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The library never imports it, and it
shares no code with the CUDA path.

The network maps a right-hand side of the normal equations (A^T b, scaled to
unit RMS) to an approximation of the solution x (same scale).  It is a plain
4-layer 3D convolutional net over the first three modes of the tensor; the
fourth mode is a batch index (one 3D field per fourth-mode slice):

    h0 = u                                   (1 channel)
    h1 = relu(conv(h0, W1) + b1)             (32 channels)
    h2 = relu(conv(h1, W2) + b2)             (32 channels)
    h3 = relu(conv(h2, W3) + b3)             (32 channels)
    y  = conv(h3, W4) + b4                   (1 channel)

conv is the 'same' 3x3x3 cross-correlation with zero padding:

    out[o, z, y, x, n] = sum_c sum_{a,b,e in {0,1,2}} W[o, c, a, b, e] * in[c, z+a-1, y+b-1, x+e-1, n]

Tensors here are laid out (channels, n1, n2, n3, n4).  The training loss is the
mean squared error against the target t:  L = mean((y - t)^2).  The optimiser
is Adam (Kingma and Ba, 2015) with bias correction.

Storage precision.  The GPU network keeps weights and inter-layer activations
(and their gradients) in bfloat16 and accumulates in FP32.  With
``quantize=True`` this oracle rounds the same quantities to bfloat16 (round to
nearest even) at the same points, and otherwise computes in FP64, so that the
two agree up to the order of the FP32 accumulations.  With ``quantize=False``
everything stays FP64 (used for the finite-difference checks).
"""
from __future__ import annotations

import numpy as np

CH = 32
LAYERS = ((1, CH), (CH, CH), (CH, CH), (CH, 1))  # (c_in, c_out) per layer


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 value (ties to even), returned as float64.

    bfloat16 is the upper half of an IEEE binary32: round the float32 bit
    pattern at bit 16 (adding 0x7FFF plus the lowest kept bit), keep the top
    16 bits.  Values are first rounded to float32 (the GPU converts from FP32).
    """
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return out.astype(np.float64)


def conv3d(x: np.ndarray, w: np.ndarray, b) -> np.ndarray:
    """'Same' 3x3x3 cross-correlation, zero padding, batched over the last axis.

    x: (C_in, D, H, W, B); w: (C_out, C_in, 3, 3, 3); b: (C_out,) or None.
    """
    cin, d, h, wd, nb = x.shape
    cout = w.shape[0]
    xp = np.zeros((cin, d + 2, h + 2, wd + 2, nb))
    xp[:, 1:-1, 1:-1, 1:-1, :] = x
    y = np.zeros((cout, d, h, wd, nb))
    for a in range(3):
        for bb in range(3):
            for e in range(3):
                y += np.tensordot(w[:, :, a, bb, e], xp[:, a:a + d, bb:bb + h, e:e + wd, :], axes=(1, 0))
    if b is not None:
        y += np.asarray(b, dtype=np.float64)[:, None, None, None, None]
    return y


def conv3d_backward(x: np.ndarray, w: np.ndarray, dy: np.ndarray, need_dx: bool = True):
    """Gradients of conv3d with respect to its input, weights and bias.

    dx[c, v] = sum_o sum_taps W[o, c, tap] dy[o, v - tap]  (adjoint of the correlation)
    dW[o, c, tap] = sum_v dy[o, v] x[c, v + tap]
    db[o] = sum_v dy[o, v]
    """
    cin, d, h, wd, nb = x.shape
    xp = np.zeros((cin, d + 2, h + 2, wd + 2, nb))
    xp[:, 1:-1, 1:-1, 1:-1, :] = x
    dxp = np.zeros_like(xp) if need_dx else None
    dw = np.zeros_like(w, dtype=np.float64)
    for a in range(3):
        for bb in range(3):
            for e in range(3):
                win = xp[:, a:a + d, bb:bb + h, e:e + wd, :]
                dw[:, :, a, bb, e] = np.tensordot(dy, win, axes=([1, 2, 3, 4], [1, 2, 3, 4]))
                if need_dx:
                    dxp[:, a:a + d, bb:bb + h, e:e + wd, :] += np.tensordot(w[:, :, a, bb, e], dy, axes=(0, 0))
    db = dy.sum(axis=(1, 2, 3, 4))
    dx = dxp[:, 1:-1, 1:-1, 1:-1, :] if need_dx else None
    return dx, dw, db


def init_params(rng: np.random.Generator):
    """He-normal weights (std sqrt(2 / fan_in), fan_in = 27 c_in), zero biases; the last layer is scaled by 0.1."""
    params = []
    for li, (ci, co) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (27 * ci))
        w = rng.standard_normal((co, ci, 3, 3, 3)) * std
        if li == len(LAYERS) - 1:
            w *= 0.1
        params.append((w, np.zeros(co)))
    return params


def quantize_params(params):
    return [(bf16_round(w), np.asarray(b, dtype=np.float64)) for w, b in params]


def forward(params, u: np.ndarray, quantize: bool = True):
    """Network output y (n1, n2, n3, n4) for the input field u (same shape), plus the activations.

    With quantize, the weights must already be bfloat16 values (quantize_params)
    and h1..h3 are rounded to bfloat16 after the ReLU, as the GPU stores them.
    """
    q = bf16_round if quantize else (lambda a: a)
    h = [np.asarray(u, dtype=np.float64)[None]]
    for li, (w, b) in enumerate(params):
        z = conv3d(h[-1], w, b)
        if li < len(params) - 1:
            h.append(q(np.maximum(z, 0.0)))
        else:
            y = z[0]
    return y, h


def loss_and_grads(params, u: np.ndarray, t: np.ndarray, quantize: bool = True):
    """L = mean((y - t)^2) and its gradients [(dW, db)] per layer (backpropagation).

    With quantize, the gradient with respect to each stored activation
    (dL/dh after the ReLU mask, the input of the next backward convolution)
    is rounded to bfloat16, as the GPU stores it.
    """
    q = bf16_round if quantize else (lambda a: a)
    y, h = forward(params, u, quantize)
    diff = y - np.asarray(t, dtype=np.float64)
    n = diff.size
    loss = float(np.mean(diff * diff))
    g = (2.0 / n) * diff[None]  # dL/dy, one channel
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        w, _ = params[li]
        if li == len(params) - 1:
            g = q(g)
        dx, dw, db = conv3d_backward(h[li], w, g, need_dx=li > 0)
        grads[li] = (dw, db)
        if li > 0:
            g = q(dx * (h[li] > 0.0))  # through the ReLU that produced h[li]
    return loss, grads


def adam_step(params, grads, state, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) of FP64 master parameters.

    state: dict with 't' (step count) and per-tensor 'm', 'v' lists (created on the first call).
      m <- beta1 m + (1 - beta1) g;  v <- beta2 v + (1 - beta2) g^2
      p <- p - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)
    """
    flat_p = [a for wb in params for a in wb]
    flat_g = [a for wb in grads for a in wb]
    if "m" not in state:
        state["t"] = 0
        state["m"] = [np.zeros_like(a, dtype=np.float64) for a in flat_p]
        state["v"] = [np.zeros_like(a, dtype=np.float64) for a in flat_p]
    state["t"] += 1
    t = state["t"]
    out = []
    for k, (p, g) in enumerate(zip(flat_p, flat_g)):
        m = beta1 * state["m"][k] + (1.0 - beta1) * g
        v = beta2 * state["v"][k] + (1.0 - beta2) * g * g
        state["m"][k], state["v"][k] = m, v
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        out.append(p - lr * mhat / (np.sqrt(vhat) + eps))
    return [(out[2 * i], out[2 * i + 1]) for i in range(len(params))]


def to_channels_first(a: np.ndarray) -> np.ndarray:
    """(n1, n2, n3, n4) -> (1, n1, n2, n3, n4)."""
    return np.asarray(a, dtype=np.float64)[None]


def pack_params(params) -> np.ndarray:
    """Flat parameter vector: for each layer W (c_out, c_in, 3, 3, 3) in C order, then b."""
    return np.concatenate([np.concatenate([np.ravel(w), np.ravel(b)]) for w, b in params])


def unpack_params(flat: np.ndarray):
    params, k = [], 0
    for ci, co in LAYERS:
        nw = co * ci * 27
        w = np.asarray(flat[k:k + nw], dtype=np.float64).reshape(co, ci, 3, 3, 3)
        k += nw
        b = np.asarray(flat[k:k + co], dtype=np.float64)
        k += co
        params.append((w, b))
    return params


def n_params() -> int:
    return sum(co * ci * 27 + co for ci, co in LAYERS)
