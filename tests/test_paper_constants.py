"""Defaults that the paper prints (tests/golden/paper_parameters.json)."""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


def load():
    with open(GOLDEN) as f:
        return json.load(f)


def test_oracle_defaults_follow_the_paper(oracle_mod):
    g = load()
    prm = oracle_mod.params()
    assert prm.knn == g["knn_k"]["value"]
    assert prm.tol == g["convergence_threshold_deg"]["value"]


def test_top_fraction_is_one_percent(oracle_mod):
    g = load()
    frac = g["convergence_top_fraction"]["value"]
    v = np.arange(1000, dtype=np.float64)
    k = int(round(frac * 1000))
    assert oracle_mod.top1_mean(v) == v[-k:].mean()


def test_header_defaults_follow_the_paper():
    g = load()
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "dwg.h")).read()
    assert f"tol {g['convergence_threshold_deg']['value']} degrees" in hdr
    assert f"k = {g['knn_k']['value']}" in hdr
