"""Pins for the oracle's basis functions: radial spline, real spherical harmonics, gradients.

Each pin comes from outside the oracle: a library routine (scipy's natural cubic spline and
complex spherical harmonics), textbook closed forms of low-order harmonics, orthonormality
under an exact product quadrature, the O(h^4) convergence of a cubic spline, and central
finite differences for the gradient.
"""
import math

import numpy as np
import pytest
from scipy.interpolate import CubicSpline
from scipy.special import sph_harm_y

from oracle import Oracle
from paper_1912_06636_gb300 import synth


def _single_atom(ls, alphas, n_rgrid=1000, rc=6.0, n_rad=8, nt=4, nphi=5):
    sp = synth.Species(ls=ls, alphas=alphas, rc=rc)
    return synth.make_system([[0.0, 0.0, 0.0]], [0], [sp], n_rad, nt, nphi, n_rgrid=n_rgrid)


def test_spline_matches_scipy_natural_spline():
    s = _single_atom([0, 1, 2, 3], [10.0, 1.5, 0.4, 0.1])
    o = Oracle(s)
    delta = math.log(s.r_last / s.r0) / (s.n_rgrid - 1)
    rng = np.random.Generator(np.random.PCG64(7))
    knots = np.arange(s.n_rgrid, dtype=np.float64)
    for f in range(len(s.fn_l)):
        cs = CubicSpline(knots, s.fn_table[f], bc_type="natural")
        for r in np.exp(rng.uniform(math.log(2e-4), math.log(5.9), 200)):
            R, dR = o.radial(f, r)
            sc = math.log(r / s.r0) / delta
            ref = float(cs(sc))
            scale = np.abs(s.fn_table[f]).max()
            assert abs(R - ref) <= 1e-13 * scale
            # compare dR/ds, the quantity the spline defines
            assert abs(dR * r * delta - float(cs(sc, 1))) <= 1e-12 * scale


def test_spline_interpolates_nodes_and_cutoff():
    s = _single_atom([0, 2], [1.5, 0.6])
    o = Oracle(s)
    rg = synth.log_grid(s.n_rgrid, s.r0, s.r_last)
    for f in range(2):
        for k in [1, 17, 300, 650, 800]:
            R, _ = o.radial(f, rg[k])
            # s = ln(r_k/r0)/Delta lands on k only up to rounding, hence a few ulps
            assert abs(R - s.fn_table[f, k]) <= 1e-13 * max(1.0, abs(s.fn_table[f, k]))
        assert o.radial(f, 6.0) == (0.0, 0.0)
        assert o.radial(f, 7.5) == (0.0, 0.0)
        # below r0 the radial part is taken at r0
        assert o.radial(f, 0.5e-4) == o.radial(f, 1e-4)


def test_spline_error_falls_as_h4():
    """Error against the analytic Gaussian falls ~16x per halving of the log-grid spacing."""
    l, a = 1, 1.5
    errs = []
    for n in (500, 1000, 2000):
        s = _single_atom([l], [a], n_rgrid=n)
        o = Oracle(s)
        rr = np.linspace(0.05, 4.5, 400)
        ref = synth.radial_function(rr, l, a, 6.0)
        got = np.array([o.radial(0, r)[0] for r in rr])
        errs.append(np.abs(got - ref).max())
    assert errs[0] / errs[1] > 10.0 and errs[1] / errs[2] > 10.0
    assert errs[1] < 1e-7


def _real_from_complex(l, m, theta, phi):
    """Real harmonics without the Condon-Shortley phase, from scipy's complex ones (which carry it)."""
    if m == 0:
        return sph_harm_y(l, 0, theta, phi).real
    Y = sph_harm_y(l, abs(m), theta, phi)
    sgn = (-1) ** abs(m)
    return math.sqrt(2.0) * sgn * (Y.real if m > 0 else Y.imag)


@pytest.mark.parametrize("l", range(0, 7))
def test_ylm_matches_scipy(l):
    rng = np.random.Generator(np.random.PCG64(l))
    for _ in range(25):
        v = rng.standard_normal(3)
        r = np.linalg.norm(v)
        theta, phi = math.acos(v[2] / r), math.atan2(v[1], v[0])
        got = Oracle.ylm(l, *v)
        for i, m in enumerate(range(-l, l + 1)):
            assert abs(got[i] - _real_from_complex(l, m, theta, phi)) < 1e-13


def test_ylm_textbook_low_orders():
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    c2 = 0.5 * math.sqrt(15.0 / math.pi)
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(20):
        x, y, z = rng.standard_normal(3)
        r2 = x * x + y * y + z * z
        r = math.sqrt(r2)
        assert abs(Oracle.ylm(0, x, y, z)[0] - 0.5 / math.sqrt(math.pi)) < 1e-15
        assert np.allclose(Oracle.ylm(1, x, y, z), [c1 * y / r, c1 * z / r, c1 * x / r], atol=1e-15, rtol=0)
        want2 = [c2 * x * y / r2, c2 * y * z / r2, 0.25 * math.sqrt(5.0 / math.pi) * (3 * z * z - r2) / r2,
                 c2 * x * z / r2, 0.5 * c2 * (x * x - y * y) / r2]
        assert np.allclose(Oracle.ylm(2, x, y, z), want2, atol=1e-15, rtol=0)


def test_ylm_orthonormal_to_l6():
    """Gauss-Legendre(12) x uniform(14) integrates products of degree <= 12 exactly."""
    dirs, w = synth.angular_product_grid(12, 14)
    rows = []
    for l in range(7):
        vals = np.array([Oracle.ylm(l, *d) for d in dirs])  # [n, 2l+1]
        rows.append(vals)
    Y = np.concatenate(rows, axis=1)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-13


def test_gradient_matches_finite_differences():
    s = synth.make_system([[0.0, 0.0, 0.0], [1.1, -0.4, 0.7]], [0, 1],
                          [synth.Species([0, 1, 2, 3], [1.5, 0.8, 0.6, 0.4]), synth.Species([0, 1], [2.0, 0.5])],
                          6, 4, 5)
    o = Oracle(s)
    rng = np.random.Generator(np.random.PCG64(11))
    pts = rng.uniform(-2.5, 2.5, (40, 3))
    _, g = o.eval_dense(pts)
    h = 1e-5
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fp, _ = o.eval_dense(pts + e)
        fm, _ = o.eval_dense(pts - e)
        fd = (fp - fm) / (2 * h)
        assert np.abs(fd - g[:, :, c]).max() < 1e-8 * max(1.0, np.abs(g).max())


def test_polar_axis_and_nucleus_are_reported():
    import oracle as orc

    s = _single_atom([0, 1], [1.5, 0.8])
    o = Oracle(s)
    with pytest.raises(orc.OracleError):
        o.eval_dense(np.array([[0.0, 0.0, 0.7]]))
    with pytest.raises(orc.OracleError):
        o.eval_dense(np.array([[0.0, 0.0, 0.0]]))


def test_spline_near_cutoff_is_only_absolutely_accurate():
    """Near the cutoff the spline crosses zero, so R is ill-conditioned in r: moving r by a
    few ulps (the rounding of s = ln(r/r0)/Delta is ~1e-13 at s ~ 970) changes R by ~1e-12
    relative while the change stays ~1e-21 of the table's scale. Two correct FP64 evaluations
    therefore agree there only absolutely, which is why the parity measures floor their
    denominators (tests/_metrics.py)."""
    s = synth.config_water(n_rad=4, n_theta=2, n_phi=3)
    o = Oracle(s)
    f = 2  # l = 1, alpha = 0.4: non-negligible all the way to the cutoff
    scale = np.abs(s.fn_table[f]).max()
    worst_rel = 0.0
    for r in np.linspace(5.95, 5.9999, 200):
        r2 = r * (1.0 + 4e-16)
        R1, _ = o.radial(f, r)
        R2, _ = o.radial(f, r2)
        assert abs(R1 - R2) <= 1e-15 * scale
        if R1 != 0.0:
            worst_rel = max(worst_rel, abs(R1 - R2) / abs(R1))
    assert worst_rel > 1e-13
