"""Checks of a Barnes-Hut far field (Sec. 5.2, "Octree Traversal") against
the exact sum, for any tree that a caller hands in (test helper).

A tree is a dict in the layout of ``dwg_get_tree``: a complete binary tree
over leaves of ``leaf`` consecutive points of a permutation ``perm`` (node 1
the root, node k with children 2k and 2k + 1, the upper half of the slots
the leaves), with per node the area A, the centre c and a radius r.  The
checks here do not assume how the tree was built:

* ``verify_tree`` recomputes A and c of every node from the points in its
  range and checks that r bounds every point's distance from c (exactly for
  a leaf, through the children for an inner node) -- the only property the
  error bound uses;
* ``walk`` applies the opening test of Sec. 5.2 (far when |q - c| exceeds the
  opening radius beta r, or max(beta r, r + the node's largest clamp radius)
  for the modified kernel) in FP64 to every query; a node within a relative
  1e-5 of its radius is "ambiguous": a float32 test may decide it either way;
* ``far_bound`` sums ``oracle.far_field_bound`` over each query's far nodes,
  ambiguous ones included.  Opening a node instead never raises its share:
  a child's radius plus its centre's offset is at most the parent's radius,
  so its gap to the query is at least the parent's and its r at most the
  parent's, and an opened leaf is exact.  So the sum bounds the far-field
  error of every decomposition the float32 test can produce, the group form
  of the test (a node far from a group's box is far from each query in it)
  included;
* ``decomposition_value`` evaluates one query's decomposition in FP64 with
  the oracle's own kernel: the leaves it opens point by point, the far nodes
  as one dipole each.
"""
import numpy as np

import oracle


def build_reference_tree(points, weights, leaf, beta, delta=None):
    """A valid tree in the layout above, built here in FP64 over the oracle's
    Morton order (for checking the checker; any valid hierarchy will do)."""
    p = np.asarray(points, np.float64)
    a = np.asarray(weights, np.float64)
    n = len(p)
    perm = oracle.morton_order(points)
    nb = -(-n // leaf)
    L = 0
    while (1 << L) < nb:
        L += 1
    nleaf = 1 << L
    nn = 2 * nleaf
    A = np.zeros(nn)
    C = np.zeros((nn, 3))
    R = np.zeros(nn)
    ps, as_ = p[perm], a[perm]
    for b in range(nleaf):
        j0, j1 = b * leaf, min((b + 1) * leaf, n)
        if j0 >= j1:
            continue
        k = nleaf + b
        A[k] = as_[j0:j1].sum()
        C[k] = (as_[j0:j1, None] * ps[j0:j1]).sum(0) / A[k]
        R[k] = np.linalg.norm(ps[j0:j1] - C[k], axis=1).max()
    for k in range(nleaf - 1, 0, -1):
        l, r = 2 * k, 2 * k + 1
        A[k] = A[l] + A[r]
        if A[k] > 0:
            C[k] = (A[l] * C[l] + A[r] * C[r]) / A[k]
            R[k] = max([np.linalg.norm(C[ch] - C[k]) + R[ch] for ch in (l, r) if A[ch] > 0])
    ro = opening_radius(dict(perm=perm, area=A, radius=R, leaf=leaf, nodes=nn), beta, delta)
    rec = np.zeros((nn, 4), np.float32)
    rec[:, :3] = C.astype(np.float32)
    rec[:, 3] = np.where(A > 0, (ro * ro).astype(np.float32), -1.0)
    rec[0, 3] = -1.0
    return dict(nodes=nn, leaf=leaf, perm=perm, area=A, centre=C, radius=R, record=rec)


def _node_max(values_sorted, T, n, fn=np.maximum):
    """Per node, the reduction of a per-point array over the node's range."""
    nn, leaf = T["nodes"], T["leaf"]
    nleaf = nn // 2
    out = np.zeros(nn)
    pad = np.zeros(nleaf * leaf)
    pad[:n] = values_sorted
    out[nleaf:] = fn.reduce(pad.reshape(nleaf, leaf), axis=1)
    for k in range(nleaf - 1, 0, -1):
        out[k] = fn(out[2 * k], out[2 * k + 1])
    return out


def opening_radius(T, beta, delta=None):
    """beta r, or with the modified kernel's radii max(beta r, r + the
    largest radius of the node's points)."""
    ro = beta * np.asarray(T["radius"], np.float64)
    if delta is not None:
        n = len(T["perm"])
        dmax = _node_max(np.asarray(delta, np.float64)[T["perm"]], T, n)
        ro = np.maximum(ro, T["radius"] + dmax)
    return ro


def verify_tree(T, points, weights, rtol=1e-12):
    """Raise AssertionError unless T is a valid hierarchy of the points."""
    p = np.asarray(points, np.float64)
    a = np.asarray(weights, np.float64)
    n = len(p)
    perm = np.asarray(T["perm"])
    assert np.array_equal(np.sort(perm), np.arange(n)), "perm is not a permutation"
    nn, leaf = T["nodes"], T["leaf"]
    nleaf = nn // 2
    assert nleaf * leaf >= n and (nleaf // 2) * leaf < max(n, 2 * leaf), "leaf count"
    A, C, R = (np.asarray(T[k], np.float64) for k in ("area", "centre", "radius"))
    scale = np.abs(p).max() + 1.0
    # leaves: sums over their ranges (padding slots carry weight 0)
    ap = np.zeros(nleaf * leaf)
    ap[:n] = a[perm]
    pp = np.zeros((nleaf * leaf, 3))
    pp[:n] = p[perm]
    ap, pp = ap.reshape(nleaf, leaf), pp.reshape(nleaf, leaf, 3)
    a_ref = ap.sum(1)
    AL, CL, RL = A[nleaf:], C[nleaf:], R[nleaf:]
    empty = a_ref == 0
    assert np.all(AL[empty] == 0.0), "an empty leaf has area"
    assert np.all(np.abs(AL - a_ref) <= rtol * 4 * leaf * a_ref), "leaf areas"
    full = ~empty
    c_ref = (ap[:, :, None] * pp).sum(1)[full] / a_ref[full, None]
    assert np.all(np.abs(CL[full] - c_ref) <= rtol * 8 * leaf * scale), "leaf centres"
    dist = np.linalg.norm(pp - CL[:, None, :], axis=2)
    slot = np.arange(nleaf * leaf).reshape(nleaf, leaf) < n
    dmax = np.where(slot, dist, 0.0).max(1)
    bad = full & (RL < dmax * (1 - rtol) - rtol * scale)
    assert not bad.any(), f"{bad.sum()} leaf radii below their points' distance"
    # inner nodes, level by level: sums of the children, radius through them
    first = nleaf // 2
    while first >= 1:
        k = np.arange(first, 2 * first)
        l, r = 2 * k, 2 * k + 1
        assert np.all(np.abs(A[k] - (A[l] + A[r])) <= rtol * 4 * A[k]), "inner areas"
        live = A[k] > 0
        kk, ll, rr = k[live], l[live], r[live]
        c_ref = (A[ll, None] * C[ll] + A[rr, None] * C[rr]) / A[kk, None]
        assert np.all(np.abs(C[kk] - c_ref) <= rtol * 8 * scale), "inner centres"
        need = np.maximum(
            np.where(A[ll] > 0, np.linalg.norm(C[ll] - C[kk], axis=1) + R[ll], 0.0),
            np.where(A[rr] > 0, np.linalg.norm(C[rr] - C[kk], axis=1) + R[rr], 0.0))
        bad = R[kk] < need * (1 - rtol) - rtol * scale
        assert not bad.any(), f"{bad.sum()} inner radii below their children's reach"
        first //= 2


def verify_records(T, beta, delta=None, rtol=1e-6):
    """The float traversal records hold the float centres and the squared
    opening radius (relative rtol; 1e-5 suits radii from another process's
    clamp radii)."""
    A = np.asarray(T["area"])
    rec = np.asarray(T["record"], np.float32)
    live = A > 0
    live[0] = False
    np.testing.assert_array_equal(rec[live, :3], np.asarray(T["centre"])[live].astype(np.float32))
    ro = opening_radius(T, beta, delta)
    ref = ro[live] ** 2
    assert np.all(np.abs(rec[live, 3] - ref) <= rtol * ref + 1e-30), "opening radii"
    assert np.all(rec[~live, 3] < 0), "empty nodes must be marked"


def walk(T, queries, beta, delta=None, kappa=1e-5):
    """Per query, the far nodes (ambiguous ones included), the ambiguous
    subset and the opened leaves of the opening test.  Returns three lists
    of (query index array, node array)."""
    q = np.asarray(queries, np.float64)
    A = np.asarray(T["area"])
    C = np.asarray(T["centre"], np.float64)
    R = np.asarray(T["radius"], np.float64)
    ro = opening_radius(T, beta, delta)
    nleaf = T["nodes"] // 2
    tau = 1e-6 * (1.0 + max(np.abs(q).max(), np.abs(C).max()))
    qi = np.arange(len(q))
    nd = np.ones(len(q), np.int64)
    far_q, far_n, amb_q, amb_n, leaf_q, leaf_n = [], [], [], [], [], []
    while len(qi):
        live = A[nd] > 0
        qi, nd = qi[live], nd[live]
        d = np.linalg.norm(q[qi] - C[nd], axis=1)
        lim = ro[nd]
        far = d > lim * (1 + kappa) + tau
        amb = ~far & (d >= lim * (1 - kappa) - tau) & (d - R[nd] > 2 * tau)
        take = far | amb
        far_q.append(qi[take]); far_n.append(nd[take])
        amb_q.append(qi[amb]); amb_n.append(nd[amb])
        op = ~take
        qi, nd = qi[op], nd[op]
        isleaf = nd >= nleaf
        leaf_q.append(qi[isleaf]); leaf_n.append(nd[isleaf])
        qi, nd = qi[~isleaf], nd[~isleaf]
        qi = np.repeat(qi, 2)
        nd = np.stack([2 * nd, 2 * nd + 1], axis=1).ravel()
    cat = lambda xs: np.concatenate(xs) if xs else np.zeros(0, np.int64)  # noqa: E731
    return ((cat(far_q), cat(far_n)), (cat(amb_q), cat(amb_n)), (cat(leaf_q), cat(leaf_n)))


def far_bound(T, queries, far, lam=0.0, eps=0.0, mass_slack=1e-6):
    """Per query, the sum of far_field_bound over its far nodes: w and grad.
    The far term is placed at the float centre, so the radius grows by the
    centre's rounding offset."""
    q = np.asarray(queries, np.float64)
    fq, fn = far
    C = np.asarray(T["centre"], np.float64)
    cf = C.astype(np.float32).astype(np.float64)
    off = np.linalg.norm(C - cf, axis=1)
    r = np.asarray(T["radius"])[fn] + off[fn]
    d = np.linalg.norm(q[fq] - cf[fn], axis=1)
    mass = np.asarray(T["area"])[fn] * (1 + mass_slack)
    bw, bg = oracle.far_field_bound(mass, r, d, lam=lam, eps=eps)
    sw = np.bincount(fq, weights=bw, minlength=len(q))
    sg = np.bincount(fq, weights=bg, minlength=len(q))
    return sw, sg


def node_moments(T, normals, weights):
    """M = sum a n per node (FP64), from the points in each node's range."""
    perm = np.asarray(T["perm"])
    n = len(perm)
    an = np.asarray(weights, np.float64)[perm, None] * np.asarray(normals, np.float64)[perm]
    nn, leaf = T["nodes"], T["leaf"]
    nleaf = nn // 2
    pad = np.zeros((nleaf * leaf, 3))
    pad[:n] = an
    M = np.zeros((nn, 3))
    M[nleaf:] = pad.reshape(nleaf, leaf, 3).sum(1)
    for k in range(nleaf - 1, 0, -1):
        M[k] = M[2 * k] + M[2 * k + 1]
    return M


def decomposition_value(T, points, normals, weights, queries, far, leaves, kernel=0, lam=0.0,
                        eps=0.0, delta=None, grad=True):
    """w (and grad w) of each query's decomposition, in FP64 through
    oracle.gwn: opened leaves point by point, far nodes as one dipole
    (sum a n at the node's FP64 centre)."""
    p = np.asarray(points, np.float64)
    nrm = np.asarray(normals, np.float64)
    a = np.asarray(weights, np.float64)
    q = np.asarray(queries, np.float64)
    perm = np.asarray(T["perm"])
    n, leaf, nleaf = len(p), T["leaf"], T["nodes"] // 2
    M = node_moments(T, normals, weights)
    Mn = np.linalg.norm(M, axis=1)
    C = np.asarray(T["centre"], np.float64)
    fq, fn = far
    lq, ln = leaves
    fo = np.argsort(fq, kind="stable")
    lo = np.argsort(lq, kind="stable")
    fsplit = np.searchsorted(fq[fo], np.arange(len(q) + 1))
    lsplit = np.searchsorted(lq[lo], np.arange(len(q) + 1))
    w = np.zeros(len(q))
    g = np.zeros((len(q), 3))
    for i in range(len(q)):
        nodes = fn[fo[fsplit[i]:fsplit[i + 1]]]
        nodes = nodes[Mn[nodes] > 0]
        lv = ln[lo[lsplit[i]:lsplit[i + 1]]] - nleaf
        idx = np.concatenate([np.arange(b * leaf, min((b + 1) * leaf, n)) for b in lv]) \
            if len(lv) else np.zeros(0, np.int64)
        src = perm[idx]
        P = np.vstack([p[src], C[nodes]])
        N = np.vstack([nrm[src], M[nodes] / Mn[nodes, None]])
        W = np.concatenate([a[src], Mn[nodes]])
        D = None
        if delta is not None:
            D = np.concatenate([np.asarray(delta, np.float64)[src], np.zeros(len(nodes))])
        if len(P) == 0:
            continue
        res = oracle.gwn(P, N, W, q[i:i + 1], kernel=kernel, eps=eps, lam=lam, grad=grad,
                         delta=D)
        if grad:
            w[i], g[i] = res[0][0], res[1][0]
        else:
            w[i] = res[0]
    return (w, g) if grad else w


def node_dipole_spread(T, points, normals, weights):
    """D = sum_j m_j (p_j - c)^T per node (3 x 3, FP64, m = a n / 4 pi): the
    next term of a node's expansion about its centre c."""
    perm = np.asarray(T["perm"])
    n = len(perm)
    p = np.asarray(points, np.float64)[perm]
    m = (np.asarray(weights, np.float64)[perm, None] *
         np.asarray(normals, np.float64)[perm]) / (4 * np.pi)
    nn, leaf = T["nodes"], T["leaf"]
    nleaf = nn // 2
    C = np.asarray(T["centre"], np.float64)
    # sum m p^T per node, then shift to the node's centre: D = S - M c^T
    mp = np.zeros((nleaf * leaf, 3, 3))
    mp[:n] = m[:, :, None] * p[:, None, :]
    S = np.zeros((nn, 3, 3))
    S[nleaf:] = mp.reshape(nleaf, leaf, 3, 3).sum(1)
    M = np.zeros((nn, 3))
    mm = np.zeros((nleaf * leaf, 3))
    mm[:n] = m
    M[nleaf:] = mm.reshape(nleaf, leaf, 3).sum(1)
    for k in range(nleaf - 1, 0, -1):
        S[k] = S[2 * k] + S[2 * k + 1]
        M[k] = M[2 * k] + M[2 * k + 1]
    return S - M[:, :, None] * C[:, None, :]


def second_order_correction(T, D, queries, far, lam=0.0, eps=0.0):
    """Per query, the sum over its far nodes of the second-order term of the
    far-field expansion (the next term after Sec. 5.2's one dipole per node):
    a source's term is -<m, grad G(p - q)>, so moving it by d = p - c adds
    -<m, Hess G(c - q) d> to first order in d; summed over the node that is
    -<Hess G(c - q), D> (Frobenius), D = sum m (p - c)^T.  Softened potential
    G(rho), rho^2 = |x|^2 + eps^2: Hess = (G1 / rho) I + (G2 - G1 / rho) x x^T
    / rho^2 with G1, G2 its first and second derivatives."""
    q = np.asarray(queries, np.float64)
    fq, fn = far
    C = np.asarray(T["centre"], np.float64)
    x = C[fn] - q[fq]
    rho = np.sqrt((x * x).sum(1) + eps * eps)
    s = np.sqrt(max(lam, 0.0))
    u = s * rho
    e = np.exp(-u)
    g1r = -e * (1 + u) / rho ** 3                 # G1 / rho
    g2 = e * (2 + 2 * u + u * u) / rho ** 3       # G2
    xDx = np.einsum("ki,kij,kj->k", x, D[fn], x)
    trD = np.einsum("kii->k", D[fn])
    corr = -(g1r * trD + (g2 - g1r) * xDx / rho ** 2)
    return np.bincount(fq, weights=corr, minlength=len(q))
