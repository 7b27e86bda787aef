"""Pins for the oracle's periodic Hamiltonian h(k) (Eq. HamPeriodic with the Bloch basis of
Eq. Bloch-basis), computed point by point from the Bloch functions:
  * h(k) is Hermitian, h(-k) = conj(h(k)), and h(k + G) = h(k) for reciprocal vectors G
    (e^{i G.T} = 1): a wrong translation or phase argument fails these;
  * the translation sum has converged (one more shell of cells changes nothing);
  * supercell identity: with a lattice-periodic potential and matching grids, the generalised
    spectrum of a cell doubled along a1 at k = 0 is the union of the unit cell's spectra at k = 0
    and k = b1 / 2 (Bloch's theorem), which fixes the Bloch sum, its normalisation per cell and
    the overlap together.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import TERM_KINETIC, TERM_POTENTIAL, Oracle
from paper_1912_06636_gb300 import synth



def _rotation(axis, angle):
    """Rotation matrix about a unit axis (Rodrigues' formula)."""
    u = np.asarray(axis, dtype=np.float64) / np.linalg.norm(axis)
    K = np.array([[0, -u[2], u[1]], [u[2], 0, -u[0]], [-u[1], u[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)


# a skewed cell turned so that no lattice vector lies along a coordinate axis: a mistake that
# mirrors one Cartesian component of the translations then maps no lattice vector onto another
LAT = (np.diag([6.0, 6.5, 7.0]) + np.array([[0, 0, 0], [0.8, 0, 0], [0, 0.5, 0]])) @ _rotation([0.3, -0.5, 0.8], 0.7).T
SPECIES = [synth.Species(ls=[0, 1], alphas=[1.0, 0.8], rc=4.0, Z=1.0),
           synth.Species(ls=[0, 0, 1, 2], alphas=[2.0, 0.7, 1.1, 0.9], rc=4.5, Z=2.0)]
FRAC = [[0.11, 0.23, 0.31], [0.57, 0.61, 0.72]]


@pytest.fixture(scope="module")
def cell():
    s = synth.periodic_cell(LAT, FRAC, [0, 1], SPECIES, n_grid=10)
    return s, Oracle(s)


def test_hermitian_time_reversal_and_reciprocal_shift(cell):
    s, o = cell
    v = synth.periodic_potential(s)
    B = 2 * np.pi * np.linalg.inv(LAT).T
    k = np.array([0.31, -0.17, 0.12])
    H, A = o.periodic_h(LAT, 2, s.pt_xyz, s.pt_w, k, v)
    scale = np.abs(A).max()
    assert np.abs(H).max() > 1e-3 * scale
    assert np.allclose(H, H.conj().T, rtol=0, atol=1e-15 * scale)
    Hm, _ = o.periodic_h(LAT, 2, s.pt_xyz, s.pt_w, -k, v)
    assert np.allclose(Hm, H.conj(), rtol=0, atol=1e-15 * scale)
    for G in (B[0], B[1] - B[2], 2 * B[2]):
        HG, _ = o.periodic_h(LAT, 2, s.pt_xyz, s.pt_w, k + G, v)
        assert np.allclose(HG, H, rtol=0, atol=1e-13 * scale)
    H3, _ = o.periodic_h(LAT, 3, s.pt_xyz, s.pt_w, k, v)
    assert np.allclose(H3, H, rtol=0, atol=1e-15 * scale)


def test_supercell_spectrum_is_union_of_k_spectra():
    n = (6, 6, 6)
    s = synth.periodic_cell(LAT, FRAC, [0, 1], SPECIES, n_grid=n)
    o = Oracle(s)
    Lsc = LAT.copy()
    Lsc[0] *= 2
    frac_sc = [[f[0] / 2, f[1], f[2]] for f in FRAC] + [[(f[0] + 1) / 2, f[1], f[2]] for f in FRAC]
    ssc = synth.periodic_cell(Lsc, frac_sc, [0, 1, 0, 1], SPECIES, n_grid=(2 * n[0], n[1], n[2]))
    osc = Oracle(ssc)
    B = 2 * np.pi * np.linalg.inv(LAT).T
    ev = []
    for k in (np.zeros(3), B[0] / 2):
        h, _ = o.periodic_h(LAT, 2, s.pt_xyz, s.pt_w, k, synth.periodic_potential(s))
        sm, _ = o.periodic_h(LAT, 2, s.pt_xyz, s.pt_w, k, None, TERM_POTENTIAL)
        ev.append(sla.eigh(h, sm, eigvals_only=True))
    hsc, _ = osc.periodic_h(Lsc, 2, ssc.pt_xyz, ssc.pt_w, np.zeros(3), synth.periodic_potential(s, ssc.pt_xyz))
    ssm, _ = osc.periodic_h(Lsc, 2, ssc.pt_xyz, ssc.pt_w, np.zeros(3), None, TERM_POTENTIAL)
    esc = sla.eigh(hsc, ssm, eigvals_only=True)
    want = np.sort(np.concatenate(ev))
    assert esc.shape == want.shape
    assert np.allclose(np.sort(esc), want, rtol=0, atol=1e-10 * np.abs(want).max())


def test_bloch_sum_of_the_image_system_hamiltonian(cell):
    """Eq. Bloch-basis inserted into Eq. HamPeriodic by hand: with chi_i = sum_T e^{i k.T}
    phi_i(r - T),
        h_ij(k) = sum_{T, T'} e^{-i k.T} e^{i k.T'} H^img_{(i, T), (j, T')},
    where H^img is the finite-system Hamiltonian (pinned by the closed forms) of the atoms'
    images R_A + T over the same translations, on the cell's points. This fixes the phase
    convention, the conjugate on the left and both terms' factors of the point-by-point route."""
    s, o = cell
    v = synth.periodic_potential(s)
    r = np.arange(-2, 3)
    cells = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    T = cells @ LAT
    n_atoms = len(s.atom_species)
    img_xyz = (s.atom_xyz[None, :, :] + T[:, None, :]).reshape(-1, 3)
    img_atom = np.tile(np.arange(n_atoms), len(T))
    si = synth.image_system(s, img_xyz, img_atom)
    Hi, _ = Oracle(si).hamiltonian(s.pt_xyz, s.pt_w, v)
    nc, nb = len(T), o.nb
    Hi = Hi.reshape(nc, nb, nc, nb)  # images cell by cell, each with the unit cell's basis order
    B = 2 * np.pi * np.linalg.inv(LAT).T
    for k in (np.zeros(3), np.array([0.31, -0.17, 0.12]), 0.5 * B[1] + 0.25 * B[2]):
        ph = np.exp(1j * (T @ k))
        want = np.einsum("a,aibj,b->ij", ph.conj(), Hi, ph)
        H, A = o.periodic_h(LAT, 2, s.pt_xyz, s.pt_w, k, v)
        assert np.abs(H.imag).max() > 1e-5 * np.abs(A).max() or not k.any()  # not real by accident
        assert np.allclose(H, want, rtol=0, atol=1e-13 * np.abs(A).max())


def test_periodic_error_denominators(cell):
    """A_ij(k) = sum_p w_p (|v| |chi_i| |chi_j| + 1/2 sum_c |d_c chi_i| |d_c chi_j|) bounds |h(k)|
    and equals the diagonal of s(k) and of the kinetic h(k), whose diagonal terms are all
    non-negative."""
    s, o = cell
    k = np.array([0.31, -0.17, 0.12])
    Sk, As = o.periodic_h(LAT, 2, s.pt_xyz, s.pt_w, k, None, TERM_POTENTIAL)
    Tk, At = o.periodic_h(LAT, 2, s.pt_xyz, s.pt_w, k, None, TERM_KINETIC)
    Hk, A = o.periodic_h(LAT, 2, s.pt_xyz, s.pt_w, k, synth.periodic_potential(s))
    assert np.allclose(np.diag(As), np.diag(Sk).real, rtol=1e-13, atol=0)
    assert np.allclose(np.diag(At), np.diag(Tk).real, rtol=1e-13, atol=0)
    assert np.all(np.abs(Hk) <= A * (1 + 1e-13))
    assert np.all(np.abs(Sk) <= As * (1 + 1e-13))
