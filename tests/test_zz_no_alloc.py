"""The allocation-free entry point dwg_eval_w_noalloc against the handle-based
dwg_eval_gwn (w only), through the C ABI, on two calls in a row.

This file is collected last on purpose: the entry point shares one fixed
device scratch array across calls, and running it after every other test
also checks that nothing earlier leaves that array in a state it relies on.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _reference(dwglib, p, nrm, a, q, kernel, lam, eps):
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
        dwglib.dwg_set_normals(h, nrm)
        w = np.zeros(len(q), np.float32)
        dwglib.dwg_eval_gwn(h, q, w, None)
        return w
    finally:
        dwglib.dwg_destroy(h)


def test_noalloc_matches_handle_path_twice(dwglib):
    torch = pytest.importorskip("torch")
    cases = [(5000, 20000, 0, 0.0, 1), (3001, 7777, 1, 10.0, 2)]
    for n, m, kernel, lam, seed in cases:
        p, _ = synth.torus(n, seed=seed, noise=0.005)
        nrm = synth.random_unit_normals(n, seed=seed + 10).astype(np.float32)
        a = np.full(n, 4 * np.pi ** 2 * 0.3 / n, np.float32)
        q = synth.uniform_box(m, [-1.5, -1.5, -0.6], [1.5, 1.5, 0.6], seed=seed + 20)
        q[:50] = p[:50]                       # queries on input points too
        eps = synth.default_eps(4 * np.pi ** 2 * 0.3, n)
        w_ref = _reference(dwglib, p, nrm, a, q, kernel, lam, eps)
        dev = torch.device("cuda")
        dp, dn, da, dq = (torch.from_numpy(x).to(dev) for x in (p, nrm, a, q))
        dw = torch.full((m,), float("nan"), dtype=torch.float32, device=dev)
        dwglib.dwg_eval_w_noalloc(dp, dn, da, dq, dw, kernel=kernel, eps=eps, screening=lam)
        w = dw.cpu().numpy()
        assert np.all(np.isfinite(w))
        assert np.max(np.abs(w - w_ref)) <= 1e-5, np.max(np.abs(w - w_ref))


def test_noalloc_rejects_sizes_beyond_its_scratch(dwglib):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda")
    big = torch.zeros((65537, 3), dtype=torch.float32, device=dev)
    big[:, 2] = 1.0
    q = torch.zeros((4, 3), dtype=torch.float32, device=dev)
    w = torch.zeros(4, dtype=torch.float32, device=dev)
    with pytest.raises(dwglib.DWGError) as e:
        dwglib.dwg_eval_w_noalloc(big, big, None, q, w, eps=0.01)
    assert e.value.code == dwglib.DWG_ERR_INVALID and "65536" in str(e.value)
    with pytest.raises(dwglib.DWGError) as e:     # host memory is not accepted
        dwglib.dwg_eval_w_noalloc(np.ones((4, 3), np.float32), np.ones((4, 3), np.float32),
                                  None, np.zeros((4, 3), np.float32), np.zeros(4, np.float32),
                                  eps=0.01)
    assert e.value.code == dwglib.DWG_ERR_INVALID
