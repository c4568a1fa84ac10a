"""A second-order far field (the one ranked "next" item not built): what it
would buy over Sec. 5.2's one dipole per far node, measured on the CPU in
FP64 against the exact sum.

The correction (tests/bh_check.second_order_correction) is first pinned on
single clusters, where it must cut the error by about the ratio r / d.  Then
on a 100,000-point metaball surface (the workload's shape at a tenth of its
size; leaves of 32 Morton-consecutive points, area-weighted centres, the
per-query opening test) the worst error over 120 queries, on and off the
surface, is compared at three opening angles: the second-order term gains
less than 2x (the error comes from small leaves just past the opening
distance, r / d = theta, where the next term does not converge fast), for
about twice the arithmetic per far term -- so the build keeps the dipole
far field and spends the operations on a smaller opening angle instead."""
import json

import numpy as np
import pytest

import synth
import bh_check


@pytest.mark.parametrize("lam", [0.0, 100.0])
def test_second_order_term_cuts_the_error_of_a_distant_cluster(oracle_mod, lam):
    rng = np.random.default_rng(3)
    for d_over_r in (4.0, 16.0):
        k = 50
        P = rng.normal(size=(k, 3)) * 0.05
        N = rng.normal(size=(k, 3))
        N /= np.linalg.norm(N, axis=1)[:, None]
        A = rng.uniform(0.5, 1.5, k)
        T = bh_check.build_reference_tree(P, A, 64, 2.0)   # one leaf: node 1 holds all
        r = T["radius"][1]
        dirn = np.array([0.3, -0.5, 0.81])
        dirn /= np.linalg.norm(dirn)
        q = T["centre"][1] + d_over_r * r * dirn
        far = (np.array([0]), np.array([1]))
        leaves = (np.zeros(0, np.int64), np.zeros(0, np.int64))
        kern = 1 if lam > 0 else 0
        w1 = bh_check.decomposition_value(T, P, N, A, q[None], far, leaves, kernel=kern,
                                          lam=lam, grad=False)
        D = bh_check.node_dipole_spread(T, P, N, A)
        w2 = w1 + bh_check.second_order_correction(T, D, q[None], far, lam=lam)
        we = oracle_mod.gwn(P, N, A, q[None], kernel=kern, lam=lam, grad=False)
        e1, e2 = abs(w1[0] - we[0]), abs(w2[0] - we[0])
        assert e2 < e1 * 3.0 / d_over_r, (d_over_r, e1, e2)


@pytest.mark.parametrize("lam", [0.0, 100.0])
def test_second_order_far_field_gains_little_on_the_metaballs(oracle_mod, lam):
    p, nt = synth.metaballs(100_000, 0, seed=0)
    n = len(p)
    a = np.ones(n)
    eps = 0.5 * float((p.max(0) - p.min(0)).max()) / np.sqrt(n)
    nrm = nt
    qs = np.vstack([p[(synth.uniform(11, 1, 60) * n).astype(np.int64)],
                    p.min(0) + synth.uniform(11, 2, 180).reshape(60, 3) * (p.max(0) - p.min(0))])
    kern = 1 if lam > 0 else 0
    we = oracle_mod.gwn(p, nrm, a, qs, kernel=kern, eps=eps, lam=lam, grad=False)
    scale = float(np.median(np.abs(we[:60])))
    rows = []
    for theta in (0.3, 0.5, 0.7):
        beta = 1.0 / theta
        T = bh_check.build_reference_tree(p, a, 32, beta)
        far, _, leaves = bh_check.walk(T, qs, beta)
        w1 = bh_check.decomposition_value(T, p, nrm, a, qs, far, leaves, kernel=kern, lam=lam,
                                          eps=eps, grad=False)
        D = bh_check.node_dipole_spread(T, p, nrm, a)
        w2 = w1 + bh_check.second_order_correction(T, D, qs, far, lam=lam, eps=eps)
        e1 = np.abs(w1 - we).max() / scale
        e2 = np.abs(w2 - we).max() / scale
        rows.append({"theta": theta, "first_order_max_rel": e1, "second_order_max_rel": e2,
                     "gain": e1 / e2})
        assert e1 / e2 < 2.0
        assert e1 > 1e-4            # the far field does make an error at this angle
    print(json.dumps({"far_order_study": "metaballs-100k", "lambda": lam, "rows": rows}))
