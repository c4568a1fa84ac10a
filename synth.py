"""Seeded synthetic point clouds and random inputs.

This module is shared by the tests, the benchmark and the smoke check.  It
holds the random streams and the shape samplers only: nothing here evaluates
a winding number or touches the orientation method.

Random numbers come from a counter-based generator, splitmix64 (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
2014): value i of stream (seed, stream) is splitmix64's output function
applied to  key + (i + 1) * GAMMA,  with  key = mix(seed * 2^32 + stream).
Uniform doubles take the top 53 bits.  The CUDA library implements the same
definition for its on-device random normal initialisation, so the two can be
compared without passing numbers between them.

Shapes are generated in float64 and returned as float32 (the library's input
type); analytic normals are returned alongside for orientation checks.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    s = (np.uint64(seed & 0xFFFFFFFF) << np.uint64(32)) | np.uint64(stream & 0xFFFFFFFF)
    return _mix(np.array([s], dtype=np.uint64))[0]


def u64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    key = stream_key(seed, stream)
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + i * GAMMA)


def uniform(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): top 53 bits of each 64-bit value times 2^-53."""
    return (u64(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    out = np.empty(2 * m)
    out[0::2] = z[:m]
    out[1::2] = z[m:]
    return out[:count]


def random_unit_normals(n: int, seed: int, stream: int = 7) -> np.ndarray:
    """Uniform directions on S^2: z = 1 - 2 u0, phi = 2 pi u1 (uniforms 2i, 2i+1).

    This is the definition the library's on-device RANDOM initialisation
    follows (it evaluates it in float32 arithmetic).
    """
    u = uniform(seed, stream, 2 * n).reshape(n, 2)
    z = 1.0 - 2.0 * u[:, 0]
    phi = 2.0 * np.pi * u[:, 1]
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def _as_f32(p: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(p, dtype=np.float32)


def bbox_diag(p: np.ndarray) -> float:
    p = np.asarray(p, dtype=np.float64)
    return float(np.linalg.norm(p.max(0) - p.min(0)))


# ----------------------------------------------------------------------------
# shapes
# ----------------------------------------------------------------------------

def sphere(n: int, seed: int = 0, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Uniform points on a sphere by normalising isotropic Gaussians."""
    g = normal(seed, 1, 3 * n).reshape(n, 3)
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    p = np.asarray(center) + radius * g
    return _as_f32(p), g.copy()


def fibonacci_sphere(n: int, radius: float = 1.0):
    """Deterministic near-uniform sphere sampling (golden-angle spiral)."""
    i = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * i / n
    phi = np.pi * (3.0 - math.sqrt(5.0)) * i
    s = np.sqrt(1.0 - z * z)
    u = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
    return _as_f32(radius * u), u


def torus(n: int, seed: int = 0, R: float = 1.0, r: float = 0.3, noise: float = 0.0):
    """Area-uniform samples on a torus about the z axis.

    u (around the axis) is uniform; v (around the tube) is drawn by rejection
    with acceptance (R + r cos v) / (R + r), which makes the density uniform
    in area.  noise is the isotropic per-coordinate Gaussian sigma as a
    fraction of the bounding-box diagonal of the clean torus.
    """
    pts = []
    nrm = []
    got = 0
    batch = 0
    while got < n:
        m = 2 * (n - got) + 64
        u = 2 * np.pi * uniform(seed, 100 + batch, m)
        v = 2 * np.pi * uniform(seed, 200 + batch, m)
        acc = uniform(seed, 300 + batch, m) < (R + r * np.cos(v)) / (R + r)
        u, v = u[acc], v[acc]
        cu, su, cv, sv = np.cos(u), np.sin(u), np.cos(v), np.sin(v)
        pts.append(np.stack([(R + r * cv) * cu, (R + r * cv) * su, r * sv], 1))
        nrm.append(np.stack([cv * cu, cv * su, sv], 1))
        got += len(u)
        batch += 1
    p = np.concatenate(pts)[:n]
    nt = np.concatenate(nrm)[:n]
    if noise > 0:
        diag = math.sqrt((2 * (R + r)) ** 2 * 2 + (2 * r) ** 2)
        p = p + noise * diag * normal(seed, 400, 3 * n).reshape(n, 3)
    return _as_f32(p), nt


def ellipsoid_points(n: int, axes, seed: int, stream: int):
    """Near-area-uniform ellipsoid samples (sphere samples, rejection on the
    area-element ratio), with analytic outward normals."""
    a = np.asarray(axes, dtype=np.float64)
    out_p, out_n = [], []
    got, b = 0, 0
    while got < n:
        m = 3 * (n - got) + 64
        g = normal(seed, stream * 1000 + b, 3 * m).reshape(m, 3)
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        x = g * a
        # the map S^2 -> ellipsoid, g -> a*g, scales area by prod(a) * |g / a|;
        # |g / a| <= 1 / min(a), so accept with probability min(a) * |g / a|
        acc = uniform(seed, stream * 1000 + b + 500, m) < a.min() * np.linalg.norm(g / a, axis=1)
        x = x[acc]
        nn = x / a ** 2
        nn /= np.linalg.norm(nn, axis=1, keepdims=True)
        out_p.append(x)
        out_n.append(nn)
        got += len(x)
        b += 1
    return np.concatenate(out_p)[:n], np.concatenate(out_n)[:n]


def add_noise(p: np.ndarray, level: float, seed: int, stream: int = 900) -> np.ndarray:
    """Isotropic Gaussian noise with sigma = level * bbox diagonal."""
    p64 = np.asarray(p, dtype=np.float64)
    sig = level * bbox_diag(p64)
    return _as_f32(p64 + sig * normal(seed, stream, p64.size).reshape(p64.shape))


def uniform_box(n: int, lo, hi, seed: int, stream: int = 950) -> np.ndarray:
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    u = uniform(seed, stream, 3 * n).reshape(n, 3)
    return _as_f32(lo + u * (hi - lo))


def default_eps(area_total: float, n: int) -> float:
    """Softening length: half the mean point spacing sqrt(A / N)."""
    return 0.5 * math.sqrt(area_total / max(n, 1))


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def workload_sphere2k():
    """2,000 uniform unit-sphere points (seed 0), area weight 4 pi / N."""
    n = 2000
    p, nt = sphere(n, seed=0)
    a = np.full(n, 4 * np.pi / n, dtype=np.float32)
    return dict(name="sphere-2k", points=p, normals_true=nt, weights=a,
                eps=default_eps(4 * np.pi, n), depth=5, max_iters=30, tol=0.1)


def workload_torus100k(noise: float = 0.005):
    """100,000 torus points (R=1, r=0.3), Gaussian noise 0.5% of the diagonal."""
    n = 100_000
    R, r = 1.0, 0.3
    p, nt = torus(n, seed=0, R=R, r=r, noise=noise)
    area = 4 * np.pi ** 2 * R * r
    a = np.full(n, area / n, dtype=np.float32)
    return dict(name="torus-100k", points=p, normals_true=nt, weights=a,
                eps=default_eps(area, n), depth=8, max_iters=30, tol=0.1)


# ----------------------------------------------------------------------------
# metaballs: the zero level set of a sum of Gaussian blobs
# ----------------------------------------------------------------------------
_TET6 = np.array([[0, 1, 3, 7], [0, 3, 2, 7], [0, 2, 6, 7], [0, 6, 4, 7], [0, 4, 5, 7],
                  [0, 5, 1, 7]])


def metaball_field(centres, sigmas, thresh):
    c = np.asarray(centres, np.float64)
    s2 = 2.0 * np.asarray(sigmas, np.float64) ** 2

    def f(x):
        x = np.asarray(x, np.float64)
        v = -thresh * np.ones(len(x))
        g = np.zeros_like(x)
        for ck, sk in zip(c, s2):
            d = x - ck
            e = np.exp(-(d * d).sum(1) / sk)
            v += e
            g += (-2.0 / sk) * e[:, None] * d
        return v, g
    return f


def _marching_tets(f, lo, hi, res):
    """Triangles of {f = 0} on a res^3 grid over [lo, hi] (marching tetrahedra)."""
    ax = [np.linspace(lo[k], hi[k], res + 1) for k in range(3)]
    X, Y, Z = np.meshgrid(ax[0], ax[1], ax[2], indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    V = np.concatenate([f(P[i:i + 2_000_000])[0] for i in range(0, len(P), 2_000_000)])
    V = V.reshape(res + 1, res + 1, res + 1)
    corners = [(v & 1, (v >> 1) & 1, (v >> 2) & 1) for v in range(8)]
    cv = np.stack([V[a:a + res, b:b + res, c:c + res] for a, b, c in corners], -1).reshape(-1, 8)
    act = np.nonzero((cv.min(1) < 0) & (cv.max(1) > 0))[0]
    i = act // (res * res)
    j = (act // res) % res
    k = act % res
    h = (np.asarray(hi) - np.asarray(lo)) / res
    base = np.asarray(lo) + np.stack([i, j, k], 1) * h
    off = np.array(corners, np.float64) * h
    cx = base[:, None, :] + off[None, :, :]
    cv = cv[act]
    tris = []
    for tet in _TET6:
        x = cx[:, tet]
        v = cv[:, tet]
        pos = v > 0
        npos = pos.sum(1)
        for m_pos in (1, 3):
            sel = npos == m_pos
            if not sel.any():
                continue
            xs, vs, ps = x[sel], v[sel], pos[sel]
            lone = np.argmax(ps == (m_pos == 1), axis=1)
            pts = []
            for t in range(1, 4):
                other = (lone + t) % 4
                xa = xs[np.arange(len(xs)), lone]
                xb = xs[np.arange(len(xs)), other]
                fa = vs[np.arange(len(vs)), lone]
                fb = vs[np.arange(len(vs)), other]
                pts.append(xa + (fa / (fa - fb))[:, None] * (xb - xa))
            tris.append(np.stack(pts, 1))
        sel = npos == 2
        if sel.any():
            xs, vs, ps = x[sel], v[sel], pos[sel]
            o = np.argsort(~ps, axis=1, kind="stable")  # two positives first
            a0, a1, b0, b1 = o[:, 0], o[:, 1], o[:, 2], o[:, 3]
            r = np.arange(len(xs))

            def ep(a, b):
                fa, fb = vs[r, a], vs[r, b]
                return xs[r, a] + (fa / (fa - fb))[:, None] * (xs[r, b] - xs[r, a])
            q0, q1, q2, q3 = ep(a0, b0), ep(a0, b1), ep(a1, b1), ep(a1, b0)
            tris.append(np.stack([q0, q1, q2], 1))
            tris.append(np.stack([q0, q2, q3], 1))
    return np.concatenate(tris, 0)


def metaballs(n_surface, n_outliers=0, seed=0, blobs=12, res=160):
    """Samples of the zero level set of sum_k exp(-|x - c_k|^2 / (2 s_k^2)) - 1/2
    (c_k ~ U[-0.6, 0.6]^3, s_k ~ U[0.12, 0.22]): marching tetrahedra on a
    res^3 grid, area-proportional triangle sampling, three Newton projections
    onto f = 0; analytic outward normals -grad f / |grad f|.  Outliers are
    uniform in the bounding box and get NaN normals."""
    c = -0.6 + 1.2 * uniform(seed, 600, 3 * blobs).reshape(blobs, 3)
    s = 0.12 + 0.10 * uniform(seed, 601, blobs)
    f = metaball_field(c, s, 0.5)
    lo = c.min(0) - 3 * s.max()
    hi = c.max(0) + 3 * s.max()
    tri = _marching_tets(f, lo, hi, res)
    area = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1)
    cdf = np.cumsum(area)
    cdf /= cdf[-1]
    pick = np.searchsorted(cdf, uniform(seed, 602, n_surface))
    pick = np.minimum(pick, len(tri) - 1)
    u = uniform(seed, 603, 2 * n_surface).reshape(n_surface, 2)
    flip = u.sum(1) > 1
    u[flip] = 1 - u[flip]
    T = tri[pick]
    x = T[:, 0] + u[:, :1] * (T[:, 1] - T[:, 0]) + u[:, 1:] * (T[:, 2] - T[:, 0])
    for _ in range(3):
        v, g = f(x)
        x = x - (v / np.maximum((g * g).sum(1), 1e-300))[:, None] * g
    _, g = f(x)
    nrm = -g / np.linalg.norm(g, axis=1, keepdims=True)
    if n_outliers:
        bl, bh = x.min(0), x.max(0)
        o = bl + uniform(seed, 604, 3 * n_outliers).reshape(n_outliers, 3) * (bh - bl)
        x = np.vstack([x, o])
        nrm = np.vstack([nrm, np.full((n_outliers, 3), np.nan)])
    return _as_f32(x), nrm


def workload_metaballs1m():
    """1,000,000 points: 990,000 on a 12-blob metaball surface plus 1 % uniform
    outliers; a_i = 1 (Sec. 5.1 dense-cloud weights); Barnes-Hut at theta 0.5."""
    p, nt = metaballs(990_000, 10_000, seed=0)
    n = len(p)
    # total area estimated from the spacing of the surface samples is not
    # needed for a_i = 1; eps from the bounding box as the library default
    ext = float((p.max(0) - p.min(0)).max())
    return dict(name="metaballs-1m", points=p, normals_true=nt,
                weights=np.ones(n, np.float32), eps=0.5 * ext / np.sqrt(n), depth=10,
                max_iters=30, tol=0.1, theta=0.5)


def workload_batch64(seed=0, n_clouds=64, lo=5_000, hi=500_000):
    """64 clouds with sizes log-uniform in [5,000, 500,000]: spheres, tori
    and metaball surfaces (uniform choice), Gaussian noise U[0, 1 %] of each
    cloud's diagonal, each placed in its own region of space (clouds never
    interact: each has its own octree and iso-value)."""
    u = uniform(seed, 700, n_clouds)
    sizes = np.round(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
    kind = (uniform(seed, 701, n_clouds) * 3).astype(int)
    noise = 0.01 * uniform(seed, 702, n_clouds)
    pts, nrms, offs = [], [], [0]
    for c in range(n_clouds):
        n = int(sizes[c])
        if kind[c] == 0:
            p, nt = sphere(n, seed=seed * 1000 + c)
        elif kind[c] == 1:
            p, nt = torus(n, seed=seed * 1000 + c)
        else:
            p, nt = metaballs(n, 0, seed=seed * 1000 + c, blobs=6, res=72)
        if noise[c] > 0:
            p = add_noise(p, float(noise[c]), seed=seed * 1000 + c)
        pts.append(p)
        nrms.append(nt)
        offs.append(offs[-1] + n)
    return dict(name="batch-64", points=np.ascontiguousarray(np.vstack(pts), dtype=np.float32),
                normals_true=np.vstack(nrms), offsets=np.array(offs, dtype=np.int64),
                kinds=kind, sizes=sizes, max_iters=30, tol=0.1)


def _rotation(seed, stream):
    q = normal(seed, stream, 4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def union_of_shapes(n, n_tori=20, n_ellipsoids=20, seed=0, noise=0.0025, labels=False):
    """Samples of the boundary of a union of randomly posed tori (R ~ U[0.08,
    0.2], r ~ U[0.2 R, 0.4 R]) and ellipsoids (semi-axes ~ U[0.04, 0.15]) with
    centres ~ U[0, 1]^3: area-uniform samples of each primitive, those inside
    another primitive dropped, subsampled to exactly n; Gaussian noise sigma
    = noise x bounding-box diagonal; analytic outward normals.  With labels,
    also the index of the primitive each sample lies on: the union has
    several connected components, and each one can settle in either
    orientation (a component whose normals point inward has w of the wrong
    sign inside, the level set of the global iso-value does not pass near
    it, and no face turns it)."""
    prims = []
    for k in range(n_tori + n_ellipsoids):
        c = uniform(seed, 1000 + k, 3)
        Rm = _rotation(seed, 2000 + k)
        if k < n_tori:
            R = 0.08 + 0.12 * uniform(seed, 3000 + k, 1)[0]
            r = R * (0.2 + 0.2 * uniform(seed, 4000 + k, 1)[0])
            prims.append(("t", c, Rm, (R, r), 4 * np.pi ** 2 * R * r))
        else:
            ax = 0.04 + 0.11 * uniform(seed, 5000 + k, 3)
            p_ = 1.6075
            area = 4 * np.pi * ((ax[0] ** p_ * ax[1] ** p_ + ax[0] ** p_ * ax[2] ** p_ +
                                 ax[1] ** p_ * ax[2] ** p_) / 3) ** (1 / p_)
            prims.append(("e", c, Rm, ax, area))

    def inside(x, k):
        kind, c, Rm, prm, _ = prims[k]
        y = (x - c) @ Rm          # local frame
        if kind == "t":
            R, r = prm
            return (np.sqrt(y[:, 0] ** 2 + y[:, 1] ** 2) - R) ** 2 + y[:, 2] ** 2 < r * r
        return ((y / prm) ** 2).sum(1) < 1.0

    total_area = sum(p[4] for p in prims)
    pts, nrms, labs = [], [], []
    for k, (kind, c, Rm, prm, area) in enumerate(prims):
        m = int(np.ceil(1.25 * n * area / total_area)) + 16
        if kind == "t":
            R, r = prm
            q, nt = torus(m, seed=seed * 100 + k, R=R, r=r)
            q = q.astype(np.float64)
        else:
            q, nt = ellipsoid_points(m, prm, seed=seed * 100 + k, stream=60 + k)
        x = q @ Rm.T + c
        nn = nt @ Rm.T
        keep = np.ones(len(x), bool)
        for j in range(len(prims)):
            if j != k:
                keep &= ~inside(x, j)
        pts.append(x[keep])
        nrms.append(nn[keep])
        labs.append(np.full(int(keep.sum()), k, dtype=np.int32))
    P = np.vstack(pts)
    lab = np.concatenate(labs)
    N = np.vstack(nrms)
    if len(P) < n:
        raise ValueError("not enough samples; raise the oversampling factor")
    sel = np.sort(np.argsort(uniform(seed, 6000, len(P)), kind="stable")[:n])
    P, N, lab = P[sel], N[sel], lab[sel]
    if noise > 0:
        diag = bbox_diag(P)
        P = P + noise * diag * normal(seed, 6001, P.size).reshape(P.shape)
    if labels:
        return _as_f32(P), N, lab
    return _as_f32(P), N


def workload_union15m():
    """15,000,000 points on a union of 20 tori and 20 ellipsoids, 0.25 % noise;
    Barnes-Hut path; random initial normals versus the learned warm start."""
    p, nt, lab = union_of_shapes(15_000_000, seed=0, labels=True)
    ext = float((p.max(0) - p.min(0)).max())
    return dict(name="union-15m", points=p, normals_true=nt, labels=lab,
                weights=np.ones(len(p), np.float32), eps=0.5 * ext / np.sqrt(len(p)),
                depth=11, max_iters=30, tol=0.1, theta=0.5)
