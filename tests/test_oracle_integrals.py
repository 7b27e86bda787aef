"""Pins for the oracle's integrals: closed forms, invariants and brute force.

Closed forms (single atom: partition weight 1; functions with alpha >= 1.5 so the cutoff
smoothing changes them by < 1e-15):
  overlap   S_ij = N_i N_j Gamma(l+3/2) / (2 a^(l+3/2)),  a = alpha_i + alpha_j, same (l, m);
  kinetic   1/2 int grad phi_i . grad phi_j from R' and l(l+1) R / r^2 (Gaussian moments);
  potential int R_i R_j [-Z erf(r)/r + 0.3 exp(-r^2)] r^2 dr with the erf moments of
            tests/golden/erf_moments.txt.
Two-centre s-s and s-p overlap and s-s kinetic energy come from the Gaussian product
theorem. Tolerances come from the quadrature/spline convergence of the grids used here.
"""
import math
from pathlib import Path

import numpy as np
import pytest

from oracle import TERM_KINETIC, TERM_POTENTIAL, Oracle
from paper_1912_06636_gb300 import synth

GOLD = {}
for line in (Path(__file__).parent / "golden" / "erf_moments.txt").read_text().splitlines():
    if line.startswith("#"):
        continue
    l, a, val = line.split()
    GOLD[(int(l), float(a))] = float(val)


def G(n, a):
    """int_0^inf r^n exp(-a r^2) dr."""
    return math.gamma((n + 1) / 2) / (2 * a ** ((n + 1) / 2))


def _basis_list(sys):
    out = []  # (atom, fn, l, m)
    for A, sp in enumerate(sys.atom_species):
        for f in range(sys.species_fn_offset[sp], sys.species_fn_offset[sp + 1]):
            l = int(sys.fn_l[f])
            for m in range(-l, l + 1):
                out.append((A, f, l, m))
    return out


@pytest.fixture(scope="module")
def single_atom():
    sp = synth.Species(ls=[0, 0, 1, 1, 2, 2, 3, 4], alphas=[10.0, 1.5, 1.75, 2.1, 1.5, 2.0, 1.6, 1.75], Z=3.0)
    s = synth.make_system([[0.0, 0.0, 0.0]], [0], [sp], n_rad=120, n_theta=12, n_phi=14, n_rgrid=4000)
    return s, Oracle(s)


def test_single_atom_closed_forms(single_atom):
    s, o = single_atom
    v = s.potential()
    S, _ = o.overlap(s.pt_xyz, s.pt_w)
    T, _ = o.hamiltonian(s.pt_xyz, s.pt_w, None, TERM_KINETIC)
    H, _ = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    bl = _basis_list(s)
    Z = float(s.Z[0])
    for i, (_, fi, li, mi) in enumerate(bl):
        for j, (_, fj, lj, mj) in enumerate(bl):
            if (li, mi) != (lj, mj):
                assert abs(S[i, j]) < 1e-12 and abs(T[i, j]) < 1e-11 and abs(H[i, j]) < 1e-11
                continue
            l = li
            al, be = float(s.fn_alpha[fi]), float(s.fn_alpha[fj])
            a = al + be
            NN = synth.gaussian_norm(l, al) * synth.gaussian_norm(l, be)
            s_ref = NN * G(2 * l + 2, a)
            t_ref = 0.5 * NN * ((l * l + l * (l + 1)) * G(2 * l, a) - 2 * l * a * G(2 * l + 2, a) + 4 * al * be * G(2 * l + 4, a))
            v_ref = NN * (-Z * GOLD[(l, round(a, 6))] + 0.3 * G(2 * l + 2, a + 1.0))
            assert abs(S[i, j] - s_ref) <= 1e-9 * abs(s_ref), (i, j, S[i, j], s_ref)
            assert abs(T[i, j] - t_ref) <= 1e-8 * abs(t_ref), (i, j, T[i, j], t_ref)
            assert abs(H[i, j] - (t_ref + v_ref)) <= 1e-8 * (abs(t_ref) + abs(v_ref)), (i, j)


@pytest.fixture(scope="module")
def two_atoms():
    A = [0.3, -0.2, 0.1]
    B = [1.1, 0.5, -0.4]
    spA = synth.Species(ls=[0], alphas=[1.8])
    spB = synth.Species(ls=[0, 1], alphas=[1.5, 2.2])
    s = synth.make_system([A, B], [0, 1], [spA, spB], n_rad=100, n_theta=24, n_phi=25, n_rgrid=4000)
    return s, Oracle(s)


def test_two_centre_gaussian_product(two_atoms):
    s, o = two_atoms
    S, _ = o.overlap(s.pt_xyz, s.pt_w)
    T, _ = o.hamiltonian(s.pt_xyz, s.pt_w, None, TERM_KINETIC)
    A, B = s.atom_xyz
    al, be = 1.8, 1.5
    p = al + be
    mu = al * be / p
    R2 = float(np.sum((A - B) ** 2))
    Na, Nb = synth.gaussian_norm(0, al), synth.gaussian_norm(0, be)
    s_ss = Na * Nb / (4 * math.pi) * (math.pi / p) ** 1.5 * math.exp(-mu * R2)
    assert abs(S[0, 1] - s_ss) < 2e-7 * s_ss
    assert abs(S[1, 0] - s_ss) < 2e-7 * s_ss
    t_ss = mu * (3.0 - 2.0 * mu * R2) * s_ss
    assert abs(T[0, 1] - t_ss) < 2e-6 * abs(t_ss)
    # s on A with p on B (m = -1, 0, 1 <-> y, z, x)
    be = 2.2
    p = al + be
    mu = al * be / p
    P = (al * A + be * B) / p
    Nb = synth.gaussian_norm(1, be)
    base = Na / math.sqrt(4 * math.pi) * Nb * math.sqrt(3 / (4 * math.pi)) * (math.pi / p) ** 1.5 * math.exp(-mu * R2)
    for k, c in enumerate([1, 2, 0]):
        ref = base * (P[c] - B[c])
        assert abs(S[0, 2 + k] - ref) < 2e-7 * abs(base), (k, S[0, 2 + k], ref)


@pytest.fixture(scope="module")
def small_molecule():
    s = synth.config_water(n_rad=14, n_theta=6, n_phi=7, max_batch_points=50)
    return s, Oracle(s)


def test_symmetry_trace_and_positivity(small_molecule):
    s, o = small_molecule
    v = s.potential()
    H, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    assert np.all(np.abs(H - H.T) <= 1e-15 * A + 1e-300)
    S, _ = o.overlap(s.pt_xyz, s.pt_w)
    P = synth.density_matrix(s, 0)
    P *= 10.0 / np.trace(P @ S)
    n, D, Ne = o.density(s.pt_xyz, P, s.pt_w)
    assert abs(Ne - 10.0) < 1e-12
    assert np.all(n >= -1e-15 * D)


def test_error_denominators(small_molecule):
    """The magnitude sums that scale every parity bar, from their definitions: A_ij =
    sum_p w_p (|phi_i v phi_j| + 1/2 |grad phi_i . grad phi_j|) is the sum of its two terms' sums,
    bounds |H|, and equals the plain sum on the diagonal of a term whose summands are all
    non-negative (w >= 0); for a rank-one P = c c^T, D_p = (sum_i |c_i phi_i|)^2 and the
    gradient's 2 sum_ij |d phi_i P_ij phi_j| = 2 (sum_i |c_i d phi_i|)(sum_j |c_j phi_j|)."""
    s, o = small_molecule
    assert np.all(s.pt_w >= 0)
    v = s.potential()
    H, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    Hp, Ap = o.hamiltonian(s.pt_xyz, s.pt_w, v, TERM_POTENTIAL)
    T, At = o.hamiltonian(s.pt_xyz, s.pt_w, None, TERM_KINETIC)
    S, As = o.overlap(s.pt_xyz, s.pt_w)
    assert np.allclose(A, Ap + At, rtol=1e-14, atol=0)
    assert np.all(np.abs(H) <= A * (1 + 1e-14))
    assert np.allclose(np.diag(At), np.diag(T), rtol=1e-14, atol=0)
    assert np.allclose(np.diag(As), np.diag(S), rtol=1e-14, atol=0)
    assert np.max(np.abs(As - np.abs(S))) > 1e-3 * As.max()  # off-diagonal sign changes count
    rng = np.random.Generator(np.random.PCG64(11))
    c = rng.standard_normal(o.nb)
    pts = s.pt_xyz[::7]
    phi, grad = o.eval_dense(pts)
    n, D, _ = o.density(pts, np.outer(c, c))
    assert np.allclose(n, (phi @ c) ** 2, rtol=1e-12, atol=1e-14 * D.max())
    assert np.allclose(D, (np.abs(phi) @ np.abs(c)) ** 2, rtol=1e-13, atol=0)
    g, Dg = o.density_gradient(pts, np.outer(c, c))
    want = 2 * (np.abs(grad) * np.abs(c)[None, :, None]).sum(axis=1) * (np.abs(phi) @ np.abs(c))[:, None]
    assert np.allclose(Dg, want, rtol=1e-13, atol=0)


def test_linearity_and_terms(small_molecule):
    s, o = small_molecule
    v = s.potential()
    rng = np.random.Generator(np.random.PCG64(5))
    v2 = rng.standard_normal(s.n_points)
    H1, A1 = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    H2, A2 = o.hamiltonian(s.pt_xyz, s.pt_w, v2)
    H12, A12 = o.hamiltonian(s.pt_xyz, s.pt_w, v + v2)
    T, _ = o.hamiltonian(s.pt_xyz, s.pt_w, None, TERM_KINETIC)
    assert np.all(np.abs(H12 - (H1 + H2 - T)) <= 1e-13 * (A1 + A2 + A12))
    H0, _ = o.hamiltonian(s.pt_xyz, s.pt_w, np.zeros(s.n_points))
    assert np.allclose(H0, T, rtol=0, atol=1e-15 * np.abs(T).max())
    S1, _ = o.hamiltonian(s.pt_xyz, s.pt_w, np.ones(s.n_points), TERM_POTENTIAL)
    S, _ = o.overlap(s.pt_xyz, s.pt_w)
    assert np.array_equal(S, S1)


def _rotation(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_rigid_motion_invariance(small_molecule):
    s, o = small_molecule
    v = s.potential()
    H, _ = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    S, _ = o.overlap(s.pt_xyz, s.pt_w)
    Q = _rotation(2)
    shift = np.array([0.37, -1.3, 2.2])
    s2 = synth.System(**{**s.__dict__})
    s2.atom_xyz = np.ascontiguousarray(s.atom_xyz @ Q.T + shift)
    pts2 = np.ascontiguousarray(s.pt_xyz @ Q.T + shift)
    o2 = Oracle(s2)
    H2, _ = o2.hamiltonian(pts2, s.pt_w, v)
    S2, _ = o2.overlap(pts2, s.pt_w)
    for X, Y in ((H, H2), (S, S2)):
        e1, e2 = np.linalg.eigvalsh(X), np.linalg.eigvalsh(Y)
        assert np.abs(e1 - e2).max() < 1e-12 * np.abs(e1).max()
    # translation only: the matrices themselves agree
    s3 = synth.System(**{**s.__dict__})
    s3.atom_xyz = np.ascontiguousarray(s.atom_xyz + shift)
    H3, _ = Oracle(s3).hamiltonian(s.pt_xyz + shift, s.pt_w, v)
    assert np.abs(H3 - H).max() < 1e-12 * np.abs(H).max()


def test_atom_permutation_permutes_blocks(small_molecule):
    s, o = small_molecule
    v = s.potential()
    H, _ = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    s2 = synth.System(**{**s.__dict__})
    order = [2, 0, 1]
    s2.atom_xyz = np.ascontiguousarray(s.atom_xyz[order])
    s2.atom_species = np.ascontiguousarray(s.atom_species[order])
    H2, _ = Oracle(s2).hamiltonian(s.pt_xyz, s.pt_w, v)
    sizes = [10, 5, 5]
    starts = np.cumsum([0] + sizes)
    perm = np.concatenate([np.arange(starts[a], starts[a] + sizes[a]) for a in order])
    assert np.allclose(H2, H[np.ix_(perm, perm)], rtol=0, atol=1e-14 * np.abs(H).max())


def test_bruteforce_equals_pointwise_definition(small_molecule):
    s, o = small_molecule
    v = s.potential()
    P = synth.density_matrix(s, 3)
    H, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    Hb, nb_ = o.bruteforce(s.pt_xyz, s.pt_w, v, P)
    assert np.all(np.abs(H - Hb) <= 1e-14 * A + 1e-300)
    n, D, _ = o.density(s.pt_xyz, P)
    assert np.all(np.abs(n - nb_) <= 1e-14 * D + 1e-300)


def test_block_equals_full(small_molecule):
    s, o = small_molecule
    v = s.potential()
    H, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    F = np.array([0, 3, 7, 12, 19])
    Hb, Ab = o.hamiltonian_block(F, s.pt_xyz, s.pt_w, v)
    assert np.all(np.abs(Hb - H[np.ix_(F, F)]) <= 1e-15 * Ab + 1e-300)


def test_density_gradient_matches_finite_differences(small_molecule):
    """grad n = 2 sum_ij grad phi_i P_ij phi_j against central differences of n itself."""
    s, o = small_molecule
    P = synth.density_matrix(s, 3)
    rng = np.random.Generator(np.random.PCG64(17))
    pts = s.pt_xyz[rng.choice(s.n_points, 60, replace=False)]
    g, Dg = o.density_gradient(pts, P)
    h = 1e-4
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        npl, _, _ = o.density(pts + e, P)
        nmi, _, _ = o.density(pts - e, P)
        fd = (npl - nmi) / (2 * h)
        assert np.all(np.abs(g[:, c] - fd) <= 1e-6 * Dg[:, c] + 1e-12), c


def test_density_gradient_single_s_function():
    """One s function R = N exp(-a r^2) (a large enough that the cutoff smoothing is below 1e-15)
    and P = [[p]]: n = p R^2 / 4 pi, grad n = 2 p R R' r_hat / 4 pi with R' = -2 a r R."""
    a, p = 2.0, 0.7
    sp = synth.Species(ls=[0], alphas=[a], Z=1.0)
    s = synth.make_system([[0.0, 0.0, 0.0]], [0], [sp], n_rad=8, n_theta=4, n_phi=5, n_rgrid=4000)
    o = Oracle(s)
    rng = np.random.Generator(np.random.PCG64(3))
    pts = rng.normal(size=(40, 3)) * 0.8
    g, _ = o.density_gradient(pts, np.array([[p]]))
    r = np.linalg.norm(pts, axis=1)
    N = synth.gaussian_norm(0, a)
    R = N * np.exp(-a * r * r)
    exact = (2 * p * R * (-2 * a * r * R) / (4 * np.pi))[:, None] * pts / r[:, None]
    # the spline reproduces the Gaussian to ~1e-6 relative in its far tail (r ~ 2.7 here)
    assert np.all(np.abs(g - exact) <= 1e-6 * np.abs(exact) + 1e-10 * np.abs(exact).max())
    assert np.all(np.abs(g - exact)[r < 1.5] <= 1e-8 * np.abs(exact)[r < 1.5])


def test_tau_term_pins(small_molecule):
    """The meta-GGA term w vtau 1/2 grad phi_i . grad phi_j: vtau = 1 gives the kinetic term,
    it is linear in vtau and adds to the other terms, and its magnitude sum is its own."""
    from oracle import TERM_TAU

    s, o = small_molecule
    rng = np.random.Generator(np.random.PCG64(23))
    ones = np.ones(s.n_points)
    Hk, Ak = o.hamiltonian(s.pt_xyz, s.pt_w, None, TERM_KINETIC)
    Ht, At = o.hamiltonian_tau(s.pt_xyz, s.pt_w, None, ones, TERM_TAU)
    assert np.allclose(Ht, Hk, rtol=0, atol=1e-14 * np.abs(Ak).max())
    a, b = rng.uniform(-1, 1, s.n_points), rng.uniform(-1, 1, s.n_points)
    Ha, _ = o.hamiltonian_tau(s.pt_xyz, s.pt_w, None, a, TERM_TAU)
    Hb, _ = o.hamiltonian_tau(s.pt_xyz, s.pt_w, None, b, TERM_TAU)
    Hab, Aab = o.hamiltonian_tau(s.pt_xyz, s.pt_w, None, 2 * a - 3 * b, TERM_TAU)
    assert np.allclose(Hab, 2 * Ha - 3 * Hb, rtol=0, atol=1e-13 * np.abs(Aab).max())
    v = s.potential()
    Hall, _ = o.hamiltonian_tau(s.pt_xyz, s.pt_w, v, a, TERM_POTENTIAL | TERM_KINETIC | TERM_TAU)
    Hpk, _ = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    assert np.allclose(Hall, Hpk + Ha, rtol=0, atol=1e-13 * np.abs(Hall).max())
    assert np.allclose(Ha, Ha.T, rtol=0, atol=1e-14 * np.abs(Ha).max())
