"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_err(got, ref):
    """max |got - ref| / max |ref| (0 when both vanish)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    den = np.abs(ref).max()
    num = np.abs(got - ref).max()
    if den == 0:
        return float(num)
    return float(num / den)


def per_slice_err(got, ref):
    """Worst rel_err over the leading axes (component, mode) of [c][m][r][z] grids."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    worst = 0.0
    lead = ref.shape[:-2]
    for idx in np.ndindex(*lead):
        worst = max(worst, rel_err(got[idx], ref[idx]))
    return worst


def by_id(p):
    order = np.argsort(p["id"], kind="stable")
    return {k: v[order] for k, v in p.items()}
