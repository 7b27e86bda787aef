"""Pins for the oracle's second derivatives: the solid harmonics' monomial expansion, the radial
spline's second derivative, the basis-function Hessian and the density Hessian (Sec. 2, the
density derivatives needed for forces and stresses).

What fixes each piece independently of the oracle's own formulas:
  * S_lm / r^l equals the oracle's Y_lm (Legendre recurrence in spherical coordinates) for every
    l <= 6; S_lm is harmonic (trace of its Hessian 0) and homogeneous of degree l (x . grad S = l S);
  * R'' against central differences of R' between the knots;
  * the Cartesian phi, grad phi equal the spherical-coordinate ones;
  * the trace of the basis Hessian equals (g'' + (2l+2) g'/r) S (S harmonic, degree l), and the
    Hessian equals central differences of the analytic gradient;
  * the density Hessian equals central differences of the density gradient, is symmetric in its
    two indices by construction of the component list, and for a rank-one P = c c^T equals the
    closed form 2 (c.grad phi)(c.grad phi)^T + 2 (c.phi)(c.hess phi).
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1912_06636_gb300 import synth

PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


@pytest.fixture(scope="module")
def water():
    s = synth.config_water(n_rad=14, n_theta=6, n_phi=7, max_batch_points=50)
    return s, Oracle(s)


def test_solid_harmonics_match_ylm_and_are_harmonic():
    rng = np.random.Generator(np.random.PCG64(5))
    for l in range(7):
        for _ in range(12):
            x = rng.normal(size=3) * rng.uniform(0.3, 3.0)
            r = np.linalg.norm(x)
            S, G, Hs = Oracle.solid(l, *x)
            Y = Oracle.ylm(l, *x)
            scale = max(np.abs(S).max(), 1e-300)
            assert np.allclose(S / r ** l, Y, rtol=0, atol=1e-13 * max(np.abs(Y).max(), 1.0)), l
            # harmonic and homogeneous of degree l
            lap = Hs[:, 0] + Hs[:, 3] + Hs[:, 5]
            assert np.all(np.abs(lap) <= 1e-12 * scale / max(r * r, 1e-300) * 10 + 1e-13), l
            assert np.allclose(G @ x, l * S, rtol=0, atol=1e-12 * scale), l


def test_solid_harmonic_derivatives_match_differences():
    rng = np.random.Generator(np.random.PCG64(6))
    h = 1e-5
    for l in range(1, 7):
        x = rng.normal(size=3)
        S, G, Hs = Oracle.solid(l, *x)
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            Sp, Gp, _ = Oracle.solid(l, *(x + e))
            Sm, Gm, _ = Oracle.solid(l, *(x - e))
            assert np.allclose(G[:, c], (Sp - Sm) / (2 * h), rtol=0, atol=1e-8 * (1 + np.abs(S).max()))
            for k, (a, b) in enumerate(PAIRS):
                if b == c:
                    assert np.allclose(Hs[:, k], (Gp[:, a] - Gm[:, a]) / (2 * h), rtol=0, atol=1e-8 * (1 + np.abs(G).max()))


def test_radial_second_derivative(water):
    s, o = water
    rng = np.random.Generator(np.random.PCG64(7))
    h = 1e-6
    for f in range(len(s.fn_l)):
        for r in rng.uniform(0.05, 0.9 * s.fn_cutoff[f], size=8):
            R, dR, d2R = o.radial2(f, r)
            R1, dR1 = o.radial(f, r)
            assert R == R1 and dR == dR1
            _, dRp, _ = o.radial2(f, r + h)
            _, dRm, _ = o.radial2(f, r - h)
            fd = (dRp - dRm) / (2 * h)
            assert abs(d2R - fd) <= 1e-5 * (abs(d2R) + abs(dR) / r + 1e-8), (f, r)


def test_cartesian_basis_equals_spherical(water):
    s, o = water
    rng = np.random.Generator(np.random.PCG64(8))
    pts = s.pt_xyz[rng.choice(s.n_points, 50, replace=False)]
    phi, grad = o.eval_dense(pts)
    phi2, grad2, _ = o.eval_dense2(pts)
    assert np.allclose(phi2, phi, rtol=0, atol=1e-12 * np.abs(phi).max())
    assert np.allclose(grad2, grad, rtol=0, atol=1e-12 * np.abs(grad).max())


def test_basis_hessian_laplacian_and_differences(water):
    s, o = water
    rng = np.random.Generator(np.random.PCG64(9))
    pts = s.pt_xyz[rng.choice(s.n_points, 40, replace=False)]
    phi, grad, hess = o.eval_dense2(pts)
    # trace = (g'' + (2l+2) g'/r) S for phi = g S, g = R / r^l
    col = 0
    for A, sp in enumerate(s.atom_species):
        for f in range(s.species_fn_offset[sp], s.species_fn_offset[sp + 1]):
            l = int(s.fn_l[f])
            for p, x0 in enumerate(pts):
                x = x0 - s.atom_xyz[A]
                r = np.linalg.norm(x)
                R, dR, d2R = o.radial2(f, r)
                g1 = dR / r ** l - l * R / r ** (l + 1)
                g2 = d2R / r ** l - 2 * l * dR / r ** (l + 1) + l * (l + 1) * R / r ** (l + 2)
                S, _, _ = Oracle.solid(l, *x)
                want = (g2 + (2 * l + 2) * g1 / r) * S
                tr = hess[p, col:col + 2 * l + 1, 0] + hess[p, col:col + 2 * l + 1, 3] + hess[p, col:col + 2 * l + 1, 5]
                scale = np.abs(hess[p, col:col + 2 * l + 1]).max() + 1e-300
                assert np.allclose(tr, want, rtol=0, atol=1e-11 * scale), (A, f, p)
            col += 2 * l + 1
    # Hessian against central differences of the analytic gradient (error ~ h^2: 2e-9 of the
    # largest element at h = 1e-6 on this grid, 2e-7 at 1e-5)
    h = 1e-6
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        _, gp, _ = o.eval_dense2(pts + e)
        _, gm, _ = o.eval_dense2(pts - e)
        fd = (gp - gm) / (2 * h)
        for k, (a, b) in enumerate(PAIRS):
            if b == c:
                assert np.allclose(hess[:, :, k], fd[:, :, a], rtol=0, atol=2e-8 * np.abs(hess).max()), (k, c)


def test_density_hessian_differences_and_rank_one(water):
    s, o = water
    rng = np.random.Generator(np.random.PCG64(10))
    pts = s.pt_xyz[rng.choice(s.n_points, 40, replace=False)]
    P = synth.density_matrix(s, 4)
    H, Dh = o.density_hessian(pts, P)
    h = 1e-6  # difference error ~ h^2: 2.6e-7 of Dh at 1e-6, 2.6e-5 at 1e-5
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        gp, _ = o.density_gradient(pts + e, P)
        gm, _ = o.density_gradient(pts - e, P)
        fd = (gp - gm) / (2 * h)
        for k, (a, b) in enumerate(PAIRS):
            if b == c:
                assert np.all(np.abs(H[:, k] - fd[:, a]) <= 1e-6 * Dh[:, k] + 1e-12), (k, c)
    # rank one: n = (c . phi)^2
    cvec = rng.normal(size=o.nb)
    phi, grad, hess = o.eval_dense2(pts)
    H1, Dh1 = o.density_hessian(pts, np.outer(cvec, cvec))
    u = phi @ cvec
    du = np.einsum("pic,i->pc", grad, cvec)
    ddu = np.einsum("pik,i->pk", hess, cvec)
    want = np.stack([2 * du[:, a] * du[:, b] + 2 * u * ddu[:, k] for k, (a, b) in enumerate(PAIRS)], axis=1)
    assert np.allclose(H1, want, rtol=0, atol=1e-12 * np.abs(want).max())
    # and its magnitude sums: 2 (sum |c d_a d_b phi|)(sum |c phi|) + 2 (sum |c d_a phi|)(sum |c d_b phi|)
    ac = np.abs(cvec)
    U = np.abs(phi) @ ac
    dU = np.einsum("pic,i->pc", np.abs(grad), ac)
    ddU = np.einsum("pik,i->pk", np.abs(hess), ac)
    wantD = np.stack([2 * ddU[:, k] * U + 2 * dU[:, a] * dU[:, b] for k, (a, b) in enumerate(PAIRS)], axis=1)
    assert np.allclose(Dh1, wantD, rtol=1e-13, atol=0)


def _atom_of(s):
    out = []
    for A, sp in enumerate(s.atom_species):
        for f in range(s.species_fn_offset[sp], s.species_fn_offset[sp + 1]):
            out += [A] * (2 * int(s.fn_l[f]) + 1)
    return np.array(out)


def _moved(s, A, c, d):
    import copy

    s2 = copy.copy(s)
    ax = np.array(s.atom_xyz, dtype=float).copy()
    ax[A, c] += d
    s2.atom_xyz = ax
    return Oracle(s2)


def test_pulay_forces_routes_and_fixed_grid_derivatives(water):
    """Local Pulay forces (Sec. 2): the matrix-element route 2 sum_{i in at} sum_j (n_ij M^c_ij - q_ij S^c_ij)
    equals the point-by-point definition; with the grid held fixed, the q part is exactly
    +d/dR tr(q S(R)) and the potential part (difference of two potentials, the kinetic part
    cancels) exactly -d/dR tr(n H_pot(R)), checked by central differences."""
    s, o = water
    rng = np.random.Generator(np.random.PCG64(12))
    v = s.potential()
    P = synth.density_matrix(s, 3)
    X = rng.normal(size=(o.nb, o.nb))
    Q = (X + X.T) / 10
    M, S, AM, AS = o.pulay_matrices(s.pt_xyz, s.pt_w, v)
    # the magnitude sums bound the matrices and exceed them where signs cancel
    assert np.all(np.abs(M) <= AM * (1 + 1e-14)) and np.all(np.abs(S) <= AS * (1 + 1e-14))
    assert np.max(AM - np.abs(M)) > 1e-3 * AM.max() and np.max(AS - np.abs(S)) > 1e-3 * AS.max()
    F = o.pulay_forces(s.pt_xyz, s.pt_w, v, P, Q)
    at = _atom_of(s)
    F2 = np.zeros_like(F)
    for c in range(3):
        r = 2 * ((P * M[c]).sum(1) - (Q * S[c]).sum(1))
        for A in range(len(s.atom_species)):
            F2[A, c] = r[at == A].sum()
    assert np.allclose(F2, F, rtol=0, atol=1e-13 * np.abs(F).max())
    h = 1e-5
    zero = np.zeros_like(P)
    Fq = o.pulay_forces(s.pt_xyz, s.pt_w, v, zero, Q)
    v2 = v * 0.5 + 0.3
    Fv = o.pulay_forces(s.pt_xyz, s.pt_w, v, P, zero) - o.pulay_forces(s.pt_xyz, s.pt_w, v2, P, zero)
    for A in range(len(s.atom_species)):
        for c in range(3):
            op, om = _moved(s, A, c, h), _moved(s, A, c, -h)
            Sp, _ = op.overlap(s.pt_xyz, s.pt_w)
            Sm, _ = om.overlap(s.pt_xyz, s.pt_w)
            dq = ((Q * Sp).sum() - (Q * Sm).sum()) / (2 * h)
            assert abs(Fq[A, c] - dq) <= 1e-6 * (abs(dq) + np.abs(Fq).max() * 1e-3), (A, c)
            Hp = op.hamiltonian(s.pt_xyz, s.pt_w, v, 1)[0] - op.hamiltonian(s.pt_xyz, s.pt_w, v2, 1)[0]
            Hm = om.hamiltonian(s.pt_xyz, s.pt_w, v, 1)[0] - om.hamiltonian(s.pt_xyz, s.pt_w, v2, 1)[0]
            dv = -((P * Hp).sum() - (P * Hm).sum()) / (2 * h)
            assert abs(Fv[A, c] - dv) <= 1e-6 * (abs(dv) + np.abs(Fv).max() * 1e-3), (A, c)
