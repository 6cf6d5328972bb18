"""Shared helpers for the parity tests (no method arithmetic here)."""
import numpy as np

# FP32 bar: max over elements of |gpu - oracle| / max(|oracle|, FLOOR * rms(oracle)).
# A plain fp32 evaluation of these networks already carries an absolute error of
# about 2e-6 rms (measured against fp64), so near-zero outputs are judged against
# a tenth of the tensor's rms rather than their own magnitude.
FP32_TOL = 1e-4
FLOOR = 0.1


def rel_err(g, o, floor=FLOOR):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    if o.size == 0:
        return 0.0
    rms = np.sqrt(np.mean(o * o))
    den = np.maximum(np.abs(o), floor * rms)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.abs(g - o) / den))


def median_rel(g, o, floor=FLOOR):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    rms = np.sqrt(np.mean(o * o))
    den = np.maximum(np.abs(o), floor * rms)
    den = np.where(den > 0, den, 1.0)
    return float(np.median(np.abs(g - o) / den))
