"""Oracle: the period-proposal CNN in FP64 NumPy (TEST INFRASTRUCTURE ONLY).

The learned proposal is not in the paper; its network is defined here in the
plainest form so that the GPU training kernels can be checked against it:
  x0 [B, L, 6]  ->  conv(6 -> 64) + ReLU  ->  4 x [conv(64 -> 64) + ReLU]
                ->  conv(64 -> 1)  ->  logits [B, L]
(the six input channels: the coarse S/N, the valid-bin mask and the S/N at the
bins of the periods 2P, P/2, 3P and P/3; the network takes them as given)
every conv with kernel 9 and zero padding: y[l, co] = b[co] + sum_k sum_ci
W[k, co, ci] x[l + k - 4, ci]. Loss: BCE with logits, positives weighted by
pos_weight, mean over B L. Update: Adam (beta 0.9, 0.999, eps 1e-8, bias-corrected).
Parameters flatten in the order W1 [9,64,6], b1, (W_k [9,64,64], b_k) k = 2..5,
W6 [9,64] (the one output channel), b6.
"""
from __future__ import annotations

import numpy as np

K = 9
C = 64
IN_CH = 6
SHAPES = [("W1", (K, C, IN_CH)), ("b1", (C,))]
for _k in range(2, 6):
    SHAPES += [(f"W{_k}", (K, C, C)), (f"b{_k}", (C,))]
SHAPES += [("W6", (K, 1, C)), ("b6", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(flat):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def shifted(x, k):
    """x[:, l + k - 4, :] with zeros outside [0, L)."""
    B, L, Ci = x.shape
    out = np.zeros_like(x)
    s = k - K // 2
    if s >= 0:
        out[:, :L - s, :] = x[:, s:, :]
    else:
        out[:, -s:, :] = x[:, :L + s, :]
    return out


def conv(x, W, b):
    y = np.zeros(x.shape[:2] + (W.shape[1],))
    for k in range(K):
        y += shifted(x, k) @ W[k].T
    return y + b


def round_bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _rw(p, k, bf16):
    """Weights of layer k as the arithmetic uses them: the 64 -> 64 layers
    compute with BF16 weights in the BF16 mode."""
    w = p[f"W{k}"]
    return round_bf16(w) if (bf16 and 2 <= k <= 5) else w


def forward(params, x0, bf16=False):
    """bf16=True rounds what the GPU kernels round: the layer outputs (after
    ReLU) and the 64 -> 64 weights; everything else stays FP64."""
    p = unflatten(params)
    acts = [np.asarray(x0, np.float64)]
    pre = []
    for k in range(1, 6):
        z = conv(acts[-1], _rw(p, k, bf16), p[f"b{k}"])
        pre.append(z)
        a = np.maximum(z, 0.0)
        acts.append(round_bf16(a) if bf16 else a)
    logits = conv(acts[-1], p["W6"], p["b6"])[..., 0]
    return logits, acts, pre


def bce(logits, labels, pos_weight):
    z = np.asarray(logits, np.float64)
    y = np.asarray(labels, np.float64)
    sp = np.logaddexp(0.0, z)          # softplus(z)
    spn = np.logaddexp(0.0, -z)        # softplus(-z)
    n = z.size
    loss = np.sum(pos_weight * y * spn + (1 - y) * sp) / n
    sig = 1.0 / (1.0 + np.exp(-z))
    dz = (pos_weight * y * (sig - 1.0) + (1 - y) * sig) / n
    return loss, dz


def conv_backward(x, W, dy):
    """Gradients of y = conv(x, W, b): dW, db, dx."""
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    for k in range(K):
        xs = shifted(x, k)
        dW[k] = np.einsum("blo,bli->oi", dy, xs)
        # x[l + k - 4] feeds y[l]: dx[m] += dy[m - k + 4] W[k]
        dx += shifted(dy @ W[k], K - 1 - k)
    db = dy.sum(axis=(0, 1))
    return dW, db, dx


def backward(params, x0, labels, pos_weight, bf16=False):
    """Loss and gradients. bf16=True also rounds the gradients of the layer
    outputs (after the ReLU mask, taken from the rounded activations) as the GPU
    stores them."""
    p = unflatten(params)
    logits, acts, pre = forward(params, x0, bf16)
    loss, dz = bce(logits, labels, pos_weight)
    g = {}
    dy = dz[..., None]
    dW, db, dx = conv_backward(acts[5], p["W6"], dy)
    g["W6"], g["b6"] = dW, db
    for k in range(5, 0, -1):
        mask = (acts[k] > 0) if bf16 else (pre[k - 1] > 0)
        dpre = dx * mask
        if bf16:
            dpre = round_bf16(dpre)
        dW, db, dx = conv_backward(acts[k - 1], _rw(p, k, bf16), dpre)
        g[f"W{k}"], g[f"b{k}"] = dW, db
    return loss, flatten(g)


def adam(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed):
    rng = np.random.default_rng(seed)
    d = {}
    for name, shp in SHAPES:
        if name.startswith("b"):
            d[name] = np.zeros(shp)
        else:
            fan_in = shp[0] * shp[2]
            d[name] = rng.normal(0.0, np.sqrt(2.0 / fan_in), shp)
    d["b6"] = np.array([-4.0])
    return flatten(d)
