"""FP64 reference of the learned pressure stage's network (TEST INFRASTRUCTURE ONLY).

A plain numpy statement of a 3-D convolutional network: 3x3x3 kernels, zero
padding, stride 1, ReLU between layers, no activation after the last layer,
mean-squared-error loss.  It is the oracle for the GPU's BF16 implicit-GEMM
convolution kernels (forward, data gradient, weight gradient).  The paper has
no learned component; this network is the learned stage of the hot path's
specification, so the reference is the textbook definition of the operations:

    y[z,y,x,o] = b[o] + sum_{t, c} x[z+dz_t, y+dy_t, x+dx_t, c] W[t, c, o]

with tap t = (dz+1)*9 + (dy+1)*3 + (dx+1), offsets in {-1, 0, 1}, and x = 0
outside the grid.  Activations are (nz, ny, nx, C) arrays (x fastest, channels
innermost), matching the grid's cell order.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shifted(x, dz, dy, dx):
    """s[z,y,x] = x[z+dz, y+dy, x+dx] (zero outside)."""
    nz, ny, nx = x.shape[:3]
    out = np.zeros_like(x)
    zs = slice(max(0, -dz), nz - max(0, dz)); zd = slice(max(0, dz), nz - max(0, -dz))
    ys = slice(max(0, -dy), ny - max(0, dy)); yd = slice(max(0, dy), ny - max(0, -dy))
    xs = slice(max(0, -dx), nx - max(0, dx)); xd = slice(max(0, dx), nx - max(0, -dx))
    out[zs, ys, xs] = x[zd, yd, xd]
    return out


def conv_fwd(x, W, b):
    """x (nz,ny,nx,Ci), W (27,Ci,Co), b (Co) -> (nz,ny,nx,Co)."""
    y = np.zeros(x.shape[:3] + (W.shape[2],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += shifted(x, dz, dy, dx) @ W[t]
    return y + b


def conv_dgrad(dy_, W):
    """gradient of sum(dy * conv_fwd(x)) with respect to x."""
    dx_ = np.zeros(dy_.shape[:3] + (W.shape[1],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        dx_ += shifted(dy_, -dz, -dy, -dx) @ W[t].T
    return dx_


def conv_wgrad(x, dy_):
    """gradients with respect to W (27,Ci,Co) and b (Co)."""
    Ci, Co = x.shape[3], dy_.shape[3]
    dW = np.zeros((27, Ci, Co))
    for t, (dz, dy, dx) in enumerate(TAPS):
        dW[t] = shifted(x, dz, dy, dx).reshape(-1, Ci).T @ dy_.reshape(-1, Co)
    return dW, dy_.reshape(-1, Co).sum(0)


def net_forward(x, params):
    """params: list of (W, b); returns the activations of every layer (pre-ReLU kept)."""
    acts = [x]
    pre = []
    h = x
    for k, (W, b) in enumerate(params):
        z = conv_fwd(h, W, b)
        pre.append(z)
        h = np.maximum(z, 0.0) if k + 1 < len(params) else z
        acts.append(h)
    return acts, pre


def mse(pred, target):
    return float(np.mean((pred - target) ** 2))


def net_loss_and_grads(x, target, params):
    """MSE loss over all cells and its gradients with respect to every (W, b)."""
    acts, pre = net_forward(x, params)
    out = acts[-1]
    n = out.size
    g = 2.0 * (out - target) / n
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        if k + 1 < len(params):
            g = g * (pre[k] > 0.0)
        dW, db = conv_wgrad(acts[k], g)
        grads[k] = (dW, db)
        if k > 0:
            g = conv_dgrad(g, params[k][0])
    return mse(out, target), grads
