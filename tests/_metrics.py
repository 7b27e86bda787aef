"""Error measures used by the parity tests.

e_H = max_ij |H_ij - H_ref,ij| / max(A_ij, f * max A) with
A_ij = sum_p w_p (|phi_i v phi_j| + 1/2 |grad phi_i . grad phi_j|), and
e_n = max_p |n_p - n_ref,p| / max(D_p, f * max D) with D_p = sum_ij |phi_i P_ij phi_j|,
f = 1e-10. The denominators are the sums of the magnitudes of the terms, the scale at which
a summation's rounding error is bounded. The floor f * max handles points and elements made
only of spline values within ~1e-3 bohr of a cutoff, where R_f -> 0 like (rc - r)^3 and FP64
keeps only absolute accuracy: two correct FP64 evaluations of the same spline differ there by
~1e-11 relative (see test_spline_near_cutoff_is_only_absolutely_accurate). Below the floor the
bar becomes absolute: |error| <= tol * 1e-10 * max D.
"""
import numpy as np

FLOOR = 1e-10


def rel_err(x, ref, denom, floor=FLOOR):
    x, ref, denom = np.asarray(x), np.asarray(ref), np.asarray(denom)
    d = np.abs(x - ref)
    if denom.size == 0:
        return 0.0
    den = np.maximum(denom, floor * float(np.max(denom)))
    zero = den == 0
    if np.any(d[zero] != 0):
        return np.inf
    return float(np.max(np.where(zero, 0.0, d / np.where(zero, 1.0, den)), initial=0.0))


def raw_rel_err(x, ref, denom):
    """The same without the floor (reported, not asserted)."""
    return rel_err(x, ref, denom, floor=0.0)
