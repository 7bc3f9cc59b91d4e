"""Error norms in FP64 (test infrastructure only).

The normwise relative error per signal is the measure every floating-point gate of this
build uses: fp32 results within 1e-6, bf16 within 1e-2 and fp16 within 2e-3 of the FP64
transform of eq. (1).  Pinned in tests/test_oracle_errors.py to values worked out by hand
from the definition below (Pythagorean triples, a zero reference, per-row independence,
FP64 accumulation, invariance under power-of-two scaling), with six planted mistakes that
those pins catch.
"""

import numpy as np


def rel_err_per_signal(y, y_ref):
    """Normwise relative error ||y - y_ref||_2 / ||y_ref||_2 per signal (last axis), FP64.

    Where ||y_ref|| is zero the absolute norm ||y|| is returned for that signal.
    """
    a = np.asarray(y, dtype=np.float64)
    b = np.asarray(y_ref, dtype=np.float64)
    a = a.reshape(-1, a.shape[-1])
    b = b.reshape(-1, b.shape[-1])
    num = np.sqrt(np.sum((a - b) ** 2, axis=1))
    den = np.sqrt(np.sum(b**2, axis=1))
    out = np.where(den > 0, num / np.where(den > 0, den, 1.0), num)
    return out
