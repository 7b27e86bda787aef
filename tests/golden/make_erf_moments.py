"""Writes erf_moments.txt: I_l(a) = int_0^inf r^(2l+1) exp(-a r^2) erf(r) dr.

Closed form: I_0(a) = 1 / (2 a sqrt(a + 1)) (the b = 1 case of
int_0^inf r exp(-a r^2) erf(b r) dr = b / (2 a sqrt(a + b^2))), and
I_l(a) = (-d/da)^l I_0(a). These are the radial integrals of the erf(r)/r attraction
between two same-centre functions r^l exp(-alpha r^2) (a = alpha + beta) used by the
single-atom closed-form pins of the Hamiltonian. Evaluated with sympy at 40 digits.
Run: python tests/golden/make_erf_moments.py
"""
from pathlib import Path

import sympy as sp

a = sp.symbols("a", positive=True)
I0 = 1 / (2 * a * sp.sqrt(a + 1))
lines = ["# l a I_l(a)   (I_l = (-d/da)^l [1/(2 a sqrt(a+1))])"]
for l in range(0, 5):
    expr = (-1) ** l * sp.diff(I0, a, l)
    for aval in ["3", "3.2", "3.5", "3.85", "4", "4.2", "11.5", "20"]:
        val = sp.N(expr.subs(a, sp.Rational(aval)), 40)
        lines.append(f"{l} {aval} {val}")
Path(__file__).with_name("erf_moments.txt").write_text("\n".join(lines) + "\n")
