"""Pins for the oracle's low-precision rounding (library conversions, exact ties, edges)."""
import numpy as np
import pytest
import torch

from oracle.lowprec import round_to, unit_roundoff


def _samples(seed=0, n=200000):
    g = np.random.default_rng(seed)
    mags = 10.0 ** g.uniform(-10, 6, n)
    x = mags * g.choice([-1.0, 1.0], n)
    return np.concatenate([x, [0.0, -0.0, 65504.0, 65519.9, 65520.0, 1e-8, 6.0e-8, 5.96e-8,
                                1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -8,
                                1.0 + 3 * 2.0 ** -8, 3.0e38, 3.4e38, np.inf, -np.inf]])


def test_fp16_matches_numpy_cast():
    x = _samples()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float64)
    got = round_to(x, "fp16")
    np.testing.assert_array_equal(got, ref)


def test_bf16_matches_torch_cast():
    # torch rounds FP64 -> FP32 -> BF16 (two roundings); on FP32 inputs its cast is a single
    # correctly rounded step, which is what the oracle computes for any input.
    with np.errstate(over="ignore"):
        x = _samples(1).astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = round_to(x, "bf16")
    np.testing.assert_array_equal(got, ref)
    # a value where the two-step route differs: the single rounding keeps 0x1.1ep-9
    assert round_to(float.fromhex("0x1.1effffe01cacbp-9"), "bf16") == float.fromhex("0x1.1ep-9")


def test_fp32_matches_numpy_cast():
    x = _samples(2)
    ref = x.astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(round_to(x, "fp32"), ref)


def test_ties_go_to_even():
    # 1 + 2^-11 lies halfway between the FP16 neighbours 1 and 1 + 2^-10: even is 1.
    assert round_to(1.0 + 2.0 ** -11, "fp16") == 1.0
    # 1 + 3*2^-11 is halfway between 1 + 2^-10 (odd) and 1 + 2^-9 (even).
    assert round_to(1.0 + 3 * 2.0 ** -11, "fp16") == 1.0 + 2.0 ** -9
    assert round_to(1.0 + 2.0 ** -8, "bf16") == 1.0
    assert round_to(65520.0, "fp16") == np.inf  # max + half ulp ties to infinity
    assert round_to(2.0 ** -25, "fp16") == 0.0  # half the smallest subnormal ties to zero


@pytest.mark.parametrize("fmt,u", [("fp32", 2.0 ** -24), ("fp16", 2.0 ** -11),
                                   ("bf16", 2.0 ** -8), ("fp64", 2.0 ** -53)])
def test_relative_error_bound(fmt, u):
    assert unit_roundoff(fmt) == u
    g = np.random.default_rng(3)
    x = g.uniform(0.5, 1000.0, 10000)
    if fmt != "fp64":
        err = np.abs(round_to(x, fmt) - x) / x
        assert err.max() <= u
