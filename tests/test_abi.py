"""The C ABI library loads and exports every function include/dwg.h declares
(CPU; no GPU compute)."""
import ctypes
import os
import re

import pytest

from conftest import HAS_GPU

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "dwg.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(dwg_[a-z_]+)\s*\(", hdr)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dwg_create", "dwg_set_params", "dwg_orient", "dwg_eval_gwn", "dwg_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2405_13839_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_abi(dwglib):
    for n in declared_functions():
        assert hasattr(dwglib, n), n


@pytest.mark.skipif(HAS_GPU, reason="checks the no-GPU error path")
def test_create_without_gpu_fails_loudly(dwglib):
    import numpy as np
    with pytest.raises(dwglib.DWGError) as e:
        dwglib.dwg_create(np.zeros((4, 3), np.float32))
    assert e.value.code == dwglib.DWG_ERR_CUDA


def test_binding_constants_match_the_header(dwglib):
    hdr = open(os.path.join(ROOT, "include", "dwg.h")).read()
    consts = dict(re.findall(r"^#define (DWG_[A-Z0-9_]+) (-?\d+)\s*$", hdr, flags=re.M))
    assert "DWG_INIT_PCA" in consts and "DWG_CONV_MEAN" in consts
    for name, value in consts.items():
        if hasattr(dwglib, name):
            assert getattr(dwglib, name) == int(value), name


def test_noalloc_binding_checks_shapes_before_the_call(dwglib):
    """Mismatched lengths and dtypes are refused by the binding before the
    library is called (the library cannot check device array lengths)."""
    import numpy as np
    p = np.zeros((8, 3), np.float32)
    q = np.zeros((5, 3), np.float32)
    w = np.zeros(5, np.float32)
    cases = [
        (p, np.zeros((7, 3), np.float32), None, q, w),          # normals short
        (p, p, np.ones(7, np.float32), q, w),                   # weights short
        (p, p, None, q, np.zeros(4, np.float32)),               # w_out short
        (p, p, None, q, np.zeros((5, 1), np.float32)),          # w_out not 1-D
    ]
    for args in cases:
        with pytest.raises(ValueError):
            dwglib.dwg_eval_w_noalloc(*args, eps=0.01)
    with pytest.raises(TypeError):                              # w_out not float32
        dwglib.dwg_eval_w_noalloc(p, p, None, q, np.zeros(5, np.float64), eps=0.01)


def test_noalloc_binding_refuses_mixed_devices(dwglib):
    torch = pytest.importorskip("torch")
    import numpy as np

    class FakeDev:
        """A float32 array that reports another device (no GPU needed)."""
        def __init__(self, a, device):
            self._a, self.device = a, device
            self.dtype, self.shape, self.ndim = a.dtype, a.shape, a.ndim

    p = torch.zeros((8, 3), dtype=torch.float32)
    q = torch.zeros((5, 3), dtype=torch.float32)
    w = FakeDev(np.zeros(5, np.float32), "cuda:1")
    with pytest.raises(ValueError, match="one device"):
        dwglib.dwg_eval_w_noalloc(p, p, None, q, w, eps=0.01)
