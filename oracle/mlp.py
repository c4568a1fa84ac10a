"""FP64 reference of the kNN-patch normal-proposal network (test
infrastructure only).

The network is a project extension, not part of the paper: it proposes
initial normals in place of the random ones of Sec. 5.1.  Layout of the flat
parameter vector (float32 on the library side):

    W1 [64][64] (out, in), b1 [64], W2 [64][64], b2 [64], W3 [64][64], b3 [64],
    W4 [3][64], b4 [3]                      -- 12,675 values

Forward: z1 = W1 x + b1, h1 = relu(z1), z2 = W2 h1 + b2, h2 = relu(z2),
z3 = W3 h2 + b3, h3 = relu(z3), y = W4 h3 + b4.  Loss over a batch of B rows:
L = (1/B) sum_rows |y - t|^2.  ``bf16=True`` rounds x, the weights and the
hidden activations to bfloat16 (round to nearest even), which is where the
tensor-core kernels round; sums stay in double.

Feature definition (per point i): its 16 nearest other points j_1..j_16
(ascending squared float32 distance, ties to the smaller index), offsets
o_k = (p_jk - p_i) / s_i with s_i = sqrt(mean_k |p_jk - p_i|^2), then
(p_i - c) / R with c the mean of all points and R = sqrt(mean |p - c|^2);
51 values, zero-padded to 64.
"""
from __future__ import annotations

import numpy as np

SIZES = [("W1", (64, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)),
         ("W3", (64, 64)), ("b3", (64,)), ("W4", (3, 64)), ("b4", (3,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[n], np.float64).ravel() for n, _ in SIZES])


def to_bf16(x):
    """Round float64/float32 values to bfloat16 (nearest even) and back."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X, bf16=False):
    P = unpack(theta)
    rd = to_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    x = rd(X)
    W = {k: (rd(v) if k.startswith("W") else v) for k, v in P.items()}
    z1 = x @ W["W1"].T + W["b1"]
    h1 = rd(np.maximum(z1, 0.0))
    z2 = h1 @ W["W2"].T + W["b2"]
    h2 = rd(np.maximum(z2, 0.0))
    z3 = h2 @ W["W3"].T + W["b3"]
    h3 = rd(np.maximum(z3, 0.0))
    y = h3 @ W["W4"].T + W["b4"]
    return y, dict(x=x, W=W, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3)


def loss_and_grad(theta, X, T, bf16=False):
    """Mean squared error and its gradient with respect to every parameter."""
    y, c = forward(theta, X, bf16)
    B = len(X)
    r = y - np.asarray(T, np.float64)
    L = float((r * r).sum() / B)
    W = c["W"]
    dy = 2.0 * r / B
    g = {}
    g["W4"] = dy.T @ c["h3"]
    g["b4"] = dy.sum(0)
    dz3 = (dy @ W["W4"]) * (c["z3"] > 0)
    g["W3"] = dz3.T @ c["h2"]
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ W["W3"]) * (c["z2"] > 0)
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ W["W2"]) * (c["z1"] > 0)
    g["W1"] = dz1.T @ c["x"]
    g["b1"] = dz1.sum(0)
    return L, pack(g)


def init_params(seed=0):
    """He-style initialisation from the counter-based stream (weights
    N(0, 2 / fan_in), biases 0)."""
    import synth
    parts = {}
    s = 0
    for name, shape in SIZES:
        if name.startswith("W"):
            fan_in = shape[1]
            parts[name] = synth.normal(seed, 800 + s, int(np.prod(shape))).reshape(shape) * np.sqrt(
                2.0 / fan_in)
        else:
            parts[name] = np.zeros(shape)
        s += 1
    return pack(parts)


def features(points, k=16):
    """Patch features (see the module docstring), brute force."""
    p = np.asarray(points, np.float32)
    n = len(p)
    p64 = p.astype(np.float64)
    c = p64.mean(0)
    R = np.sqrt(((p64 - c) ** 2).sum(1).mean())
    X = np.zeros((n, 64))
    def fmaf(a, b, c):  # float32 fused multiply-add via one rounding of the double result
        return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(
            np.float32)

    for i in range(n):
        d = p - p[i]
        dd = fmaf(d[:, 2], d[:, 2], fmaf(d[:, 1], d[:, 1], d[:, 0] * d[:, 0]))
        order = np.lexsort((np.arange(n), dd))
        nb = [j for j in order if j != i][:k]
        o = (p64[nb] - p64[i])
        s = np.sqrt((o * o).sum(1).mean())
        if s > 0:
            o = o / s
        X[i, :3 * len(nb)] = o.ravel()
        X[i, 48:51] = (p64[i] - c) / R if R > 0 else 0.0
    return X
