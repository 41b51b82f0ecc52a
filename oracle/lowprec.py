"""Round-to-nearest-even emulation of FP32, FP16 and BF16 storage (oracle side).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline leg, never by the product library.

A value is stored in a binary floating-point format with p explicit mantissa
bits and minimum normal exponent emin.  Rounding is done on the exact FP64
value: for |x| with leading-bit exponent e, the spacing of representable values
is q = 2^(max(e, emin) - p), and round(|x| / q) * q with ties to even (numpy's
`rint`) is the correctly rounded result; |x| / q is exact because q is a power
of two.  Results beyond the largest finite value become +-inf, as IEEE 754
round-to-nearest prescribes (the threshold is max + q/2, whose tie goes to the
even neighbour 2^(emax+1), i.e. to infinity).

Parity pin: the FP16 rule is checked against numpy's float16 cast and the BF16
rule against torch's bfloat16 cast (library conversions) in the oracle tests.
"""
from __future__ import annotations

import numpy as np

# (explicit mantissa bits p, minimum normal exponent, largest finite value)
FORMATS = {
    "fp64": None,
    "fp32": (23, -126, float(np.finfo(np.float32).max)),
    "fp16": (10, -14, 65504.0),
    "bf16": (7, -126, float.fromhex("0x1.fep127")),
}


def round_to(x, fmt: str) -> np.ndarray:
    """Round FP64 values to the nearest `fmt` value (ties to even); returned as FP64."""
    x = np.asarray(x, dtype=np.float64)
    spec = FORMATS[fmt]
    if spec is None:
        return x.copy()
    p, emin, vmax = spec
    a = np.abs(x)
    _, e2 = np.frexp(a)  # a = f * 2^e2 with f in [0.5, 1): leading-bit exponent e2 - 1
    e = np.maximum(e2 - 1, emin)
    q = np.ldexp(1.0, e - p)
    with np.errstate(over="ignore", invalid="ignore"):
        r = np.rint(a / q) * q
        r = np.where(r > vmax, np.inf, r)
        r = np.where(np.isfinite(a), r, a)  # inf/nan pass through
    return np.copysign(r, x)


def unit_roundoff(fmt: str) -> float:
    """u = 2^-(p+1) for the format."""
    if fmt == "fp64":
        return 2.0 ** -53
    return 2.0 ** -(FORMATS[fmt][0] + 1)
