"""Error measures between two conservative states W[M, ncells] (SoA layout of
include/hrm.h)."""
from __future__ import annotations

import numpy as np


def rel_l1(W, Wref):
    """Per-variable sum|W - Wref| / sum|Wref|."""
    num = np.abs(W - Wref).sum(axis=1)
    den = np.abs(Wref).sum(axis=1)
    return num / np.where(den == 0, 1.0, den)


def rel_l1_state(W, Wref, N, D):
    """Per-variable relative L1 error in which each momentum component is
    measured against the flow's momentum magnitude sum |rho u| (vector norm),
    so that a component that is zero in the reference (a direction the flow
    does not move in yet) is not divided by round-off; the partial densities,
    energy and volume fractions use sum |Wref_m|."""
    err = rel_l1(W, Wref)
    mom = Wref[N:N + D]
    mag = np.sqrt((mom ** 2).sum(axis=0)).sum()
    if mag > 0:
        for d in range(D):
            err[N + d] = np.abs(W[N + d] - Wref[N + d]).sum() / mag
    return err
