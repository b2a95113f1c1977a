"""Oracle of the warm-start network (test infrastructure only): plain numpy FP64 forward and
backward of the circular 1D convolutional network, same parameter layout as the CUDA kernels
(per layer: weights [out][in][K] then bias [out]); loss mean((y - t)^2)."""
from __future__ import annotations

import numpy as np


def layers(params, chans, K):
    out, off = [], 0
    for l in range(len(chans) - 1):
        ci, co = chans[l], chans[l + 1]
        W = params[off:off + co * ci * K].reshape(co, ci, K); off += co * ci * K
        b = params[off:off + co]; off += co
        out.append((W, b))
    return out


def conv(x, W, b):
    """y[b][o][x] = b[o] + sum_{c,k} W[o][c][k] x[b][c][(x + k - K/2) mod n]."""
    K = W.shape[2]
    h = K // 2
    y = np.zeros((x.shape[0], W.shape[0], x.shape[2]))
    for k in range(K):
        xs = np.roll(x, -(k - h), axis=2)           # xs[..., i] = x[..., i + k - h]
        y += np.einsum("oc,bcn->bon", W[:, :, k], xs)
    return y + b[None, :, None]


def forward(params, chans, K, x):
    acts = [np.asarray(x, np.float64)]
    L = len(chans) - 1
    for l, (W, b) in enumerate(layers(params, chans, K)):
        z = conv(acts[-1], W, b)
        acts.append(np.maximum(z, 0.0) if l < L - 1 else z)
    return acts


def loss_and_grad(params, chans, K, x, t):
    params = np.asarray(params, np.float64)
    acts = forward(params, chans, K, x)
    y = acts[-1]
    m = y.size
    loss = float(np.sum((y - t) ** 2) / m)
    dz = 2.0 * (y - t) / m
    grads = []
    Ls = layers(params, chans, K)
    L = len(Ls)
    for l in range(L - 1, -1, -1):
        W, b = Ls[l]
        a = acts[l]
        Kk = W.shape[2]
        h = Kk // 2
        dW = np.zeros_like(W)
        for k in range(Kk):
            dW[:, :, k] = np.einsum("bon,bcn->oc", dz, np.roll(a, -(k - h), axis=2))
        db = dz.sum(axis=(0, 2))
        grads.append((dW, db))
        if l > 0:
            da = np.zeros_like(a)
            for k in range(Kk):
                # d/da[c][i] of sum W[o][c][k] a[c][i + k - h] -> dz shifted back
                da += np.roll(np.einsum("oc,bon->bcn", W[:, :, k], dz), (k - h), axis=2)
            dz = da * (a > 0)
    flat = []
    for dW, db in reversed(grads):
        flat.append(dW.reshape(-1)); flat.append(db)
    return loss, np.concatenate(flat)
