"""The allocation-free entry point dwg_eval_w_noalloc, through the C ABI: on
two calls in a row against the handle-based dwg_eval_gwn (w only) and against
the FP64 oracle, at small sizes and at the entry point's size limits.

This file is collected last on purpose: the entry point shares one fixed
device scratch array across calls, and running it after every other test
also checks that nothing earlier leaves that array in a state it relies on.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

MAX_N = 65536       # the entry point's fixed scratch limits
MAX_M = 262144
TOL = 1e-5          # absolute on w, for weights that make w about 1 inside


def _reference(dwglib, p, nrm, a, q, kernel, lam, eps):
    h = dwglib.dwg_create(p)
    try:
        if a is not None:
            dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
        dwglib.dwg_set_normals(h, nrm)
        w = np.zeros(len(q), np.float32)
        dwglib.dwg_eval_gwn(h, q, w, None)
        return w
    finally:
        dwglib.dwg_destroy(h)


def _noalloc(dwglib, torch, p, nrm, a, q, kernel, lam, eps):
    dev = torch.device("cuda")
    dp, dn, dq = (torch.from_numpy(x).to(dev) for x in (p, nrm, q))
    da = None if a is None else torch.from_numpy(a).to(dev)
    out = []
    for _ in range(2):                        # two calls in a row share the scratch
        dw = torch.full((len(q),), float("nan"), dtype=torch.float32, device=dev)
        dwglib.dwg_eval_w_noalloc(dp, dn, da, dq, dw, kernel=kernel, eps=eps, screening=lam)
        out.append(dw.cpu().numpy())
    return out


def _cloud(n, m, seed):
    p, _ = synth.torus(n, seed=seed, noise=0.005)
    nrm = synth.random_unit_normals(n, seed=seed + 10).astype(np.float32)
    q = synth.uniform_box(m, [-1.5, -1.5, -0.6], [1.5, 1.5, 0.6], seed=seed + 20)
    q[:50] = p[:50]                           # queries on input points too
    return p, nrm, q


@pytest.mark.parametrize("n,m,kernel,lam,seed",
                         [(5000, 20000, 0, 0.0, 1), (3001, 7777, 1, 10.0, 2)])
def test_noalloc_matches_handle_path_and_oracle_twice(dwglib, oracle_mod, n, m, kernel, lam,
                                                        seed):
    torch = pytest.importorskip("torch")
    p, nrm, q = _cloud(n, m, seed)
    area = 4 * np.pi ** 2 * 0.3
    a = np.full(n, area / n, np.float32)
    eps = synth.default_eps(area, n)
    w_ref = _reference(dwglib, p, nrm, a, q, kernel, lam, eps)
    w64 = oracle_mod.gwn(p, nrm, a, q, kernel=kernel, eps=eps, lam=lam, grad=False)
    for w in _noalloc(dwglib, torch, p, nrm, a, q, kernel, lam, eps):
        assert np.all(np.isfinite(w))
        assert np.max(np.abs(w - w_ref)) <= TOL, np.max(np.abs(w - w_ref))
        assert np.max(np.abs(w - w64)) <= TOL, np.max(np.abs(w - w64))


def test_noalloc_at_its_size_limits_without_weights(dwglib, oracle_mod):
    """n and m at the fixed scratch's limits (the partial sums then cap the
    source chunks), weights NULL (a_i = 1).  With a_i = 1 w is the
    area-weighted w times n / area, so the tolerance scales with it."""
    torch = pytest.importorskip("torch")
    n, m = MAX_N, MAX_M
    p, nrm, q = _cloud(n, m, 3)
    area = 4 * np.pi ** 2 * 0.3
    eps = synth.default_eps(area, n)
    tol = TOL * n / area
    w_ref = _reference(dwglib, p, nrm, None, q, 1, 100.0, eps)
    rng = np.random.default_rng(4)
    pick = np.concatenate([np.arange(50), rng.choice(m, 2048, replace=False)])
    w64 = oracle_mod.gwn(p, nrm, np.ones(n), q[pick], kernel=1, eps=eps, lam=100.0,
                         grad=False)
    for w in _noalloc(dwglib, torch, p, nrm, None, q, 1, 100.0, eps):
        assert np.all(np.isfinite(w))
        assert np.max(np.abs(w - w_ref)) <= tol, np.max(np.abs(w - w_ref)) / tol
        assert np.max(np.abs(w[pick] - w64)) <= tol, np.max(np.abs(w[pick] - w64)) / tol


def test_noalloc_rejects_sizes_beyond_its_scratch(dwglib):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda")
    big = torch.zeros((MAX_N + 1, 3), dtype=torch.float32, device=dev)
    big[:, 2] = 1.0
    q = torch.zeros((4, 3), dtype=torch.float32, device=dev)
    w = torch.zeros(4, dtype=torch.float32, device=dev)
    with pytest.raises(dwglib.DWGError) as e:
        dwglib.dwg_eval_w_noalloc(big, big, None, q, w, eps=0.01)
    assert e.value.code == dwglib.DWG_ERR_INVALID and "65536" in str(e.value)
    small = torch.zeros((4, 3), dtype=torch.float32, device=dev)
    small[:, 2] = 1.0
    qbig = torch.zeros((MAX_M + 1, 3), dtype=torch.float32, device=dev)
    wbig = torch.zeros(MAX_M + 1, dtype=torch.float32, device=dev)
    with pytest.raises(dwglib.DWGError) as e:
        dwglib.dwg_eval_w_noalloc(small, small, None, qbig, wbig, eps=0.01)
    assert e.value.code == dwglib.DWG_ERR_INVALID and "262144" in str(e.value)


def test_noalloc_rejects_host_and_other_device_memory(dwglib):
    torch = pytest.importorskip("torch")
    with pytest.raises(dwglib.DWGError) as e:     # host memory is not accepted
        dwglib.dwg_eval_w_noalloc(np.ones((4, 3), np.float32), np.ones((4, 3), np.float32),
                                  None, np.zeros((4, 3), np.float32), np.zeros(4, np.float32),
                                  eps=0.01)
    assert e.value.code == dwglib.DWG_ERR_INVALID
    if torch.cuda.device_count() < 2:
        return
    # arrays on cuda:1 while cuda:0 is current: refused before any launch
    other = torch.device("cuda", 1)
    x = torch.ones((4, 3), dtype=torch.float32, device=other)
    w = torch.zeros(4, dtype=torch.float32, device=other)
    with torch.cuda.device(0):
        with pytest.raises(dwglib.DWGError) as e:
            dwglib.dwg_eval_w_noalloc(x, x, None, x, w, eps=0.01)
    assert e.value.code == dwglib.DWG_ERR_INVALID
