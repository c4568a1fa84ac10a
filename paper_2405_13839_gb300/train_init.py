"""Train the warm-start network on converged orientations of synthetic shapes.

Labels are the library's own converged DWG normals (level-set update, random
initial normals), with the global sign of each shape chosen to agree with
its analytic outward normals; inputs are the library's patch features
(dwg_mlp_features).  Training runs on the GPU with the library's tensor-core
forward/backward kernels (dwg_mlp_grad) and its Adam step (dwg_mlp_adam);
torch only holds the device arrays and draws the minibatch indices.

    python -m paper_2405_13839_gb300.train_init --out warm_start.npy
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

from . import dwg  # noqa: E402

DEFAULT_WEIGHTS = os.path.join(HERE, "warm_start.npy")
N_PARAMS = dwg.MLP_PARAMS


def he_init(seed: int) -> np.ndarray:
    """Weights N(0, 2 / fan_in) from the counter-based stream, biases 0."""
    parts = []
    shapes = [(64, 64), (64,), (64, 64), (64,), (64, 64), (64,), (3, 64), (3,)]
    for s, shape in enumerate(shapes):
        k = int(np.prod(shape))
        if len(shape) == 2:
            parts.append(synth.normal(seed, 800 + s, k) * np.sqrt(2.0 / shape[1]))
        else:
            parts.append(np.zeros(k))
    return np.concatenate(parts).astype(np.float32)


def training_shapes(seed: int, count: int):
    """Spheres, tori, ellipsoids, metaballs and unions, 20k-60k points,
    noise 0-0.5 % of the diagonal."""
    out = []
    for k in range(count):
        kind = k % 5
        n = int(20_000 + 40_000 * synth.uniform(seed, 10 + k, 1)[0])
        noise = 0.005 * synth.uniform(seed, 40 + k, 1)[0]
        s = seed * 1000 + k
        if kind == 0:
            p, nt = synth.sphere(n, seed=s, radius=0.5 + synth.uniform(s, 1, 1)[0])
        elif kind == 1:
            R = 1.0
            r = 0.15 + 0.35 * synth.uniform(s, 2, 1)[0]
            p, nt = synth.torus(n, seed=s, R=R, r=r)
        elif kind == 2:
            ax = 0.3 + 0.7 * synth.uniform(s, 3, 3)
            q, nt = synth.ellipsoid_points(n, ax, seed=s, stream=5)
            p = q.astype(np.float32)
        elif kind == 3:
            p, nt = synth.metaballs(n, 0, seed=s, blobs=6, res=80)
        else:
            p, nt = synth.union_of_shapes(n, n_tori=3, n_ellipsoids=3, seed=s, noise=0.0)
        if noise > 0:
            p = synth.add_noise(p, noise, seed=s)
        out.append((p, nt))
    return out


def label_shape(p, nt):
    """Converged DWG normals of one shape, signed outward, and its features."""
    n = len(p)
    h = dwg.dwg_create(p)
    try:
        depth = min(10, max(5, int(round(0.5 * np.log2(n)))))
        dwg.dwg_set_update(h, depth, 10, dwg.DWG_UPDATE_LEVELSET)
        dwg.dwg_set_params(h, dwg.DWG_KERNEL_SCREENED, _eps(p), 10.0, 40, 0.1)
        dwg.dwg_set_init(h, dwg.DWG_INIT_RANDOM, 1)
        out = np.zeros((n, 3), np.float32)
        dwg.dwg_orient(h, out)
        X = np.zeros((n, 64), np.float32)
        dwg.dwg_mlp_features(h, X)
    finally:
        dwg.dwg_destroy(h)
    s = 1.0 if np.sum(out * nt) >= 0 else -1.0
    return X, (s * out).astype(np.float32)


def _eps(p):
    ext = float((p.max(0) - p.min(0)).max())
    return 0.5 * ext / np.sqrt(len(p))


def train(X, T, steps=3000, batch=8192, lr=2e-3, seed=0, log=None):
    import torch
    dev = torch.device("cuda")
    dX = torch.from_numpy(X).to(dev)
    dT = torch.from_numpy(T).to(dev)
    P = torch.from_numpy(he_init(seed)).to(dev)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    g = torch.zeros_like(P)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    losses = []
    for step in range(1, steps + 1):
        idx = torch.randint(0, len(X), (batch,), device=dev, generator=gen)
        bx = dX.index_select(0, idx).contiguous()
        bt = dT.index_select(0, idx).contiguous()
        lr_t = lr * (0.1 ** (step / steps))
        L = dwg.dwg_mlp_grad(P, bx, bt, g)
        dwg.dwg_mlp_adam(P, g, m, v, step, lr_t)
        losses.append(L)
        if log and (step % 500 == 0 or step == 1):
            log(f"step {step} loss {L:.4f}")
    return P.cpu().numpy(), losses


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--shapes", type=int, default=25)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    t0 = time.time()
    Xs, Ts = [], []
    for p, nt in training_shapes(args.seed, args.shapes):
        X, T = label_shape(p, nt)
        Xs.append(X)
        Ts.append(T)
    X = np.vstack(Xs)
    T = np.vstack(Ts)
    print(f"labels: {len(X)} rows from {args.shapes} shapes in {time.time() - t0:.1f}s",
          flush=True)
    P, losses = train(X, T, steps=args.steps, seed=args.seed, log=lambda s: print(s, flush=True))
    np.save(args.out, P)
    print(f"saved {args.out}; loss {losses[0]:.4f} -> {np.mean(losses[-50:]):.4f}; "
          f"total {time.time() - t0:.1f}s")


if __name__ == "__main__":
    main()
