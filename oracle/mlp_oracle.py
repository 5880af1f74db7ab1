"""FP64 reference of the learned drag / torque closure network.

TEST INFRASTRUCTURE ONLY: the plain, slow reference that the CUDA training and inference
kernels are checked against. Only tests/, the smoke check and the benchmark's baseline legs
may import it.

The network is a multilayer perceptron x -> relu(W1 x + b1) -> relu(W2 h1 + b2) -> W3 h2 + b3
trained by mean-squared error with Adam (Kingma & Ba, 2015: m <- b1 m + (1 - b1) g,
v <- b2 v + (1 - b2) g^2, p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)). The
CUDA path stores weights and activations in bfloat16 and accumulates in FP32; with
``bf16=True`` this reference rounds the same quantities to bfloat16 at the same points (the
inputs, the weights, the hidden activations and the back-propagated activation gradients)
and computes everything else in FP64, so the two differ only by accumulation order and
precision. The paper has no network; this closure is an addition outside it.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64. bfloat16 keeps the
    top 16 bits of an IEEE binary32 value; inputs are first rounded to binary32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(a)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def init_params(sizes, seed):
    """He-uniform weights (bound sqrt(6 / fan_in)) and zero biases for layer widths `sizes`
    (e.g. [256, 128, 128, 6]); W[l] has shape (sizes[l+1], sizes[l])."""
    g = np.random.Generator(np.random.PCG64(seed))
    p = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        bound = np.sqrt(6.0 / a)
        p.append([g.uniform(-bound, bound, size=(b, a)), np.zeros(b)])
    return p


def _q(x, bf16):
    return bf16_round(x) if bf16 else np.asarray(x, dtype=np.float64)


def forward(params, X, bf16=False):
    """Returns (Y, cache). X: (B, K). Hidden layers use relu; the last layer is linear."""
    h = _q(X, bf16)
    cache = [h]
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = h @ _q(W, bf16).T + b
        if l < L - 1:
            h = _q(np.maximum(z, 0.0), bf16)
            cache.append(h)
        else:
            h = z
    return h, cache


def loss_and_grads(params, X, T, bf16=False):
    """Mean-squared error over all B x O outputs, and its gradient for every W and b."""
    Y, cache = forward(params, X, bf16)
    B, O = Y.shape
    R = Y - T
    loss = float(np.sum(R * R) / (B * O))
    d = 2.0 * R / (B * O)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        dq = _q(d, bf16)  # the CUDA path keeps each layer's output gradient in bfloat16
        grads[l] = [dq.T @ cache[l], dq.sum(0)]
        if l > 0:
            d = (dq @ _q(W, bf16)) * (cache[l] > 0.0)
    return loss, grads


def adam_init(params):
    return [[np.zeros_like(W), np.zeros_like(b)] for W, b in params], [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1), in place on params, m, v."""
    c1 = 1.0 - beta1 ** t
    c2 = 1.0 - beta2 ** t
    for l in range(len(params)):
        for k in range(2):
            g = grads[l][k]
            m[l][k] = beta1 * m[l][k] + (1.0 - beta1) * g
            v[l][k] = beta2 * v[l][k] + (1.0 - beta2) * g * g
            params[l][k] = params[l][k] - lr * (m[l][k] / c1) / (np.sqrt(v[l][k] / c2) + eps)
    return params


def stencil_features(rho, u, centers, up, n_side, h, u_ref, walls=(0, 0, 0)):
    """Closure inputs written out: for each particle p and node (i, j, k) of an n_side^3
    stencil at x_p + h (i - (n_side - 1)/2, ...), the trilinear interpolation of (rho - 1, u)
    from the 8 surrounding lattice sites (periodic axes wrap, walled axes clamp), minus the
    particle velocity for u, divided by u_ref. rho: (nz, ny, nx); u: (nz, ny, nx, 3).
    Returns (np, n_side^3 * 4), nodes in (k, j, i) order, 4 values per node."""
    nz, ny, nx = rho.shape
    dims = (nx, ny, nz)
    D = 2 if nz == 1 else 3
    out = np.zeros((len(centers), n_side ** 3 * 4))
    for p in range(len(centers)):
        for k in range(n_side):
            for j in range(n_side):
                for i in range(n_side):
                    ijk = (i, j, k)
                    lo, hi, w1 = [0, 0, 0], [0, 0, 0], [0.0, 0.0, 0.0]
                    for a in range(D):
                        pos = centers[p][a] + h * (ijk[a] - 0.5 * (n_side - 1))
                        f = np.floor(pos)
                        w1[a] = pos - f
                        a0, a1 = int(f), int(f) + 1
                        if walls[a]:
                            a0, a1 = min(max(a0, 0), dims[a] - 1), min(max(a1, 0), dims[a] - 1)
                        else:
                            a0, a1 = a0 % dims[a], a1 % dims[a]
                        lo[a], hi[a] = a0, a1
                    acc = np.zeros(4)
                    for c in range(8 if D == 3 else 4):
                        s = [hi[a] if (c >> a) & 1 else lo[a] for a in range(3)]
                        w = 1.0
                        for a in range(D):
                            w *= w1[a] if (c >> a) & 1 else 1.0 - w1[a]
                        acc[0] += w * (rho[s[2], s[1], s[0]] - 1.0)
                        acc[1:] += w * u[s[2], s[1], s[0]]
                    q = (k * n_side + j) * n_side + i
                    out[p, 4 * q] = acc[0] / u_ref
                    out[p, 4 * q + 1:4 * q + 4] = (acc[1:] - up[p]) / u_ref
    return out
