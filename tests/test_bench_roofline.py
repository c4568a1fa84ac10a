"""The bench line's FP32 roofline arithmetic (host logic, CPU only): the
derived peak is SMs x 128 lanes x clock / FP32 operations per interaction,
the measured one the lower of the FMA-pipe and MUFU bounds."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_operation_counts(bench):
    # plain w: 3 sub, 3 fma (rho^2), 3 (<m,d>), 2 mul (inv^3), 1 fma
    assert bench.FP32_OPS[("w", 0)] == 12
    assert bench.FP32_OPS[("wg", 0)] == 20
    # screened w: + rho, its ex2 argument, inv^2, inv + s, the product with e, 1 fma
    assert bench.FP32_OPS[("w", 1)] == 16
    assert bench.FP32_OPS[("wg", 1)] == 27


def test_derived_peak(bench):
    p = bench.alu_peaks("w", 1, 152, 2.07e9)
    assert p["ops"] == 16
    assert p["derived"] == pytest.approx(152 * 128 * 2.07e9 / 16)
    assert "measured" not in p


def test_measured_peak_takes_the_lower_bound(bench):
    sms, f = 152, 2.07e9
    ffma = 0.977 * sms * 128 * f                 # lane operations per second
    rsq, ex2 = sms * 16 * f, sms * 32 * f        # MUFU rates per second
    scr = bench.alu_peaks("w", 1, sms, f, ffma, rsq, ex2)
    # one rsqrt and one ex2 per screened interaction: 1/16 + 1/32 SM cycles
    assert scr["mufu_bound"] == pytest.approx(sms * f / (1 / 16 + 1 / 32))
    assert scr["fma_bound"] == pytest.approx(ffma / 16)
    assert scr["measured"] == pytest.approx(min(ffma / 16, scr["mufu_bound"]))
    assert scr["measured"] == scr["fma_bound"]  # the FMA pipe binds
    plain = bench.alu_peaks("w", 0, sms, f, ffma, rsq, ex2)
    assert plain["mufu_bound"] == pytest.approx(rsq)  # no ex2 without screening
    # a slow MUFU becomes the bound
    slow = bench.alu_peaks("w", 1, sms, f, ffma, rsq / 8, ex2 / 8)
    assert slow["measured"] == slow["mufu_bound"] < slow["fma_bound"]
