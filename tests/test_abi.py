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
