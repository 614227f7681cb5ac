"""Per-element bound of the network parity tests (GPU kernels against
oracle/learned.py, which rounds to bfloat16 at the same points as the kernels).

|gpu - ref| <= TOL * (|ref| + scale) for every element, TOL = 2^-6 (four bfloat16
units in the last place), scale = the root mean square of the reference tensor unless
the caller gives one (the scores of one sample, the gradient of one parameter tensor).
Both sides round the same values to bfloat16; they differ only where a float32 sum,
accumulated in another order, lands on the other side of a bfloat16 rounding boundary,
which moves that stored value by one unit (2^-8 relative) and the quantities computed
from it by a fraction of that.
"""
from __future__ import annotations

import numpy as np

TOL = 2.0 ** -6


def assert_close(got, want, what, scale=None):
    """Element-wise |got - want| <= TOL (|want| + scale); returns the worst ratio."""
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    assert got.shape == want.shape, what
    assert np.isfinite(got).all(), what
    if scale is None:
        scale = float(np.sqrt(np.mean(want ** 2))) if want.size else 0.0
    bound = TOL * (np.abs(want) + scale)
    err = np.abs(got - want)
    if not (err <= bound).all():
        k = int(np.argmax(err - bound))
        raise AssertionError("%s: element %d is %r, oracle %r (bound %r)" % (what, k, got[k], want[k], bound[k]))
    nz = bound > 0
    return float((err[nz] / bound[nz]).max()) if nz.any() else 0.0
