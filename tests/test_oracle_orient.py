"""The oracle's Algorithm 1 against analytic normals on closed shapes (CPU).

The paper gives no worked example; what pins the iteration is the shapes'
known outward normals: the converged normals must agree with them up to one
global sign (the orientation is defined only up to a flip)."""
import numpy as np
import pytest

import synth


def agreement(n, nt):
    d = np.sum(n * nt, axis=1)
    s = 1.0 if d.sum() >= 0 else -1.0
    return float(np.mean(s * d > 0))


def test_sphere_levelset_converges_to_analytic(oracle_mod):
    W = synth.workload_sphere2k()
    n0 = synth.random_unit_normals(2000, seed=1)
    prm = oracle_mod.params(eps=W["eps"], depth=6, max_iters=40, tol=0.1)
    r = oracle_mod.orient(W["points"], W["weights"], n0, prm)
    assert r["converged"] and r["iters"] <= 30
    assert agreement(r["normals"], W["normals_true"]) == 1.0
    # converged normals are outward or inward as a whole; with outward ones
    # w_bar approaches 1/2 (w = 1 inside, 0 outside), with inward ones -1/2
    assert abs(abs(r["iso"][-1]) - 0.5) < 0.05
    # mean alignment with the analytic normal (cf. Fig. 2's mean dot near 1)
    s = np.sign(np.sum(r["normals"] * W["normals_true"]))
    assert np.mean(s * np.sum(r["normals"] * W["normals_true"], axis=1)) > 0.98


@pytest.mark.parametrize("lam,kernel", [(0.0, 0), (10.0, 1)])
def test_torus_levelset_converges_to_analytic(oracle_mod, lam, kernel):
    n = 3000
    p, nt = synth.torus(n, seed=0)
    area = 4 * np.pi ** 2 * 0.3
    a = np.full(n, area / n)
    n0 = synth.random_unit_normals(n, seed=1)
    prm = oracle_mod.params(kernel=kernel, lam=lam, eps=synth.default_eps(area, n), depth=6,
                            max_iters=40, tol=0.1)
    r = oracle_mod.orient(p, a, n0, prm)
    assert agreement(r["normals"], nt) >= 0.999
    assert r["stat"][-1] < 1.0


def test_point_gradient_update_stalls(oracle_mod):
    """The point form n <- -grad w(p) / |grad w(p)| (one reading of Eq. 4)
    does not orient a sphere consistently from random normals: it stalls in
    domains of opposite orientation, which is why the level-set rule of
    Eq. 7 is the update of the hot path."""
    W = synth.workload_sphere2k()
    n0 = synth.random_unit_normals(2000, seed=1)
    prm = oracle_mod.params(eps=W["eps"], depth=6, max_iters=40, tol=0.1,
                            mode=oracle_mod.MODE_DIRECT)
    r = oracle_mod.orient(W["points"], W["weights"], n0, prm)
    assert agreement(r["normals"], W["normals_true"]) < 0.9


def test_mean_change_rule_stops_at_the_first_small_mean_change(oracle_mod):
    """Rule 1 stops after the first iteration whose mean |n_new - n_old| (the
    quantity of Fig. 6) is at most the chord 2 sin(tol / 2); replaying the
    iterations one by one finds the same stopping point."""
    n = 1200
    p, nt = synth.torus(n, seed=4)
    area = 4 * np.pi ** 2 * 0.3
    a = np.full(n, area / n)
    n0 = synth.random_unit_normals(n, seed=2)
    tol = 0.5
    prm = oracle_mod.params(kernel=1, lam=10.0, eps=synth.default_eps(area, n), depth=5,
                            max_iters=40, tol=tol, rule=1)
    r = oracle_mod.orient(p, a, n0, prm)
    chord = 2 * np.sin(np.radians(tol) / 2)
    cur = n0.copy()
    stop = None
    for t in range(1, 41):
        nxt = oracle_mod.iterate(p, a, cur, prm)["normals"]
        md = np.mean(np.linalg.norm(nxt - cur, axis=1))
        cur = nxt
        if md <= chord:
            stop = t
            break
    assert stop is not None and r["iters"] == stop and r["converged"]
    np.testing.assert_array_equal(r["normals"], cur)
    assert agreement(r["normals"], nt) >= 0.99


@pytest.mark.parametrize("noise", [0.0, 0.005])
def test_top1_statistic_plateaus_above_the_tolerance(oracle_mod, noise):
    """On a 5,000-point torus, clean or with 0.5 % noise, the level-set update
    of Eq. 7 settles -- every normal agrees with the analytic one and the mean
    change over all points (the measure of Fig. 6) falls far below the chord
    of 0.1 deg -- while the mean change of the 1 % most-changed points (the
    rule of Sec. 5.1) stays at a few tenths of a degree: a handful of points
    keep switching between nearby marching-cubes faces' k-nearest sets.  The
    top-1 % rule at 0.1 deg is then never met, which is why the benchmarks on
    noisy and large clouds stop on the Fig. 6 measure."""
    n, depth = 5000, 6
    p, nt = synth.torus(n, seed=0, noise=noise)
    area = 4 * np.pi ** 2 * 0.3
    a = np.full(n, area / n)
    prm = oracle_mod.params(eps=synth.default_eps(area, n), depth=depth, max_iters=1, tol=0.1)
    cur = synth.random_unit_normals(n, seed=1)
    top, mean = [], []
    for _ in range(25):
        r = oracle_mod.iterate(p, a, cur, prm)
        top.append(oracle_mod.top1_mean(r["dtheta"]))
        mean.append(np.mean(np.linalg.norm(r["normals"] - cur, axis=1)))
        cur = r["normals"]
    chord = 2 * np.sin(np.radians(0.1) / 2)
    assert agreement(cur, nt) == 1.0
    assert max(mean[18:]) <= 0.2 * chord
    assert 0.2 <= min(top[18:]) and max(top[18:]) <= 2.0, top[18:]


def _two_spheres():
    pa, na = synth.sphere(3000, seed=1)
    pb, nb = synth.sphere(1500, seed=2)
    pa = pa.astype(np.float64) + [-1.6, 0.0, 0.0]
    pb = 0.6 * pb.astype(np.float64) + [1.6, 0.0, 0.0]
    aa = np.full(3000, 4 * np.pi / 3000)
    ab = np.full(1500, 4 * np.pi * 0.36 / 1500)
    nb0 = nb.copy()
    nb0[pb[:, 2] < 0.0] *= -1.0                      # lower half of B turned inward
    return pa, na, aa, pb, nb, ab, nb0


def mixed_component_runs(oracle_mod, iters=15, depth=6):
    """Sphere B (1,500 points) with its lower half turned inward, alone and
    beside a consistently oriented sphere A (3,000 points, outward or
    inward).  Returns, per run, the share of B's points with outward
    normals after `iters` iterations, and the last iso-value."""
    pa, na, aa, pb, nb, ab, nb0 = _two_spheres()
    runs = {"B alone": (pb, ab, nb0),
            "A outward": (np.vstack([pa, pb]), np.concatenate([aa, ab]), np.vstack([na, nb0])),
            "A inward": (np.vstack([pa, pb]), np.concatenate([aa, ab]), np.vstack([-na, nb0]))}
    out = {}
    for name, (P, A, N0) in runs.items():
        P = P.astype(np.float32)
        prm = oracle_mod.params(eps=0.5 * np.sqrt(A.sum() / len(P)), depth=depth, max_iters=1)
        cur = N0
        for _ in range(iters):
            r = oracle_mod.iterate(P, A, cur, prm)
            cur = r["normals"]
        b = np.sum(cur[-1500:] * nb, axis=1)
        out[name] = (float(np.mean(b > 0)), r["iso"], cur)
    return out


def test_a_mixed_component_heals_alone_but_not_beside_another(oracle_mod):
    """Why a union of separate shapes does not reach one orientation per
    shape: the level set of Eq. 6's single iso-value w_bar only passes near
    the parts whose w crosses w_bar.  Alone, B's iso-value is its own mean and
    B heals to one orientation.  Beside a consistently oriented A, w_bar takes
    A's sign; the half of B oriented the other way has w of the other sign
    next to it, gets no faces, and keeps its normals -- B stays mixed."""
    res = mixed_component_runs(oracle_mod)
    frac, _, _ = res["B alone"]
    assert frac in (0.0, 1.0)
    for name in ("A outward", "A inward"):
        frac, iso, _ = res[name]
        assert 0.3 < frac < 0.7, (name, frac)
        assert np.sign(iso) == (1.0 if name == "A outward" else -1.0)
