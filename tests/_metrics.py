"""Error measures used by the parity tests.

e_H = max_ij |H_ij - H_ref,ij| / A_ij with A_ij = sum_p w_p (|phi_i v phi_j| + 1/2 |grad phi_i . grad phi_j|);
where A_ij = 0 the element must be exactly 0. e_n = max_p |n_p - n_ref,p| / D_p with
D_p = sum_ij |phi_i P_ij phi_j| (D_p = 0: exactly 0). Both are relative to the sum of the
magnitudes of the terms, the scale at which a summation's rounding error is bounded.
"""
import numpy as np


def rel_err(x, ref, denom):
    x, ref, denom = np.asarray(x), np.asarray(ref), np.asarray(denom)
    d = np.abs(x - ref)
    zero = denom == 0
    if np.any(d[zero] != 0):
        return np.inf
    return float(np.max(np.where(zero, 0.0, d / np.where(zero, 1.0, denom)), initial=0.0))
