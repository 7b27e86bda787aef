"""Host side of the periodic path (no GPU): the library's image list covers every image atom
whose functions reach a point of the unit cell (brute force over a wide range of translations),
lists the cell's own atoms first without duplicates, and the image basis map sends each image
function to its unit-cell function."""
import ctypes as C

import numpy as np

from paper_1912_06636_gb300 import nao, synth

LAT = np.diag([6.0, 6.5, 7.0]) + np.array([[0, 0, 0], [0.8, 0, 0], [0, 0.5, 0]])
SPECIES = [synth.Species(ls=[0, 1], alphas=[1.0, 0.8], rc=4.0, Z=1.0),
           synth.Species(ls=[0, 0, 1, 2], alphas=[2.0, 0.7, 1.1, 0.9], rc=4.5, Z=2.0)]
FRAC = [[0.11, 0.23, 0.31], [0.57, 0.61, 0.72]]


def test_images_cover_every_atom_reaching_the_cell():
    s = synth.periodic_cell(LAT, FRAC, [0, 1], SPECIES, n_grid=8)
    reach = float(np.max(s.fn_cutoff))
    xyz, atom, cell = nao.nao_periodic_images(s.atom_xyz, LAT, reach)
    n_at = s.n_atoms
    assert np.array_equal(atom[:n_at], np.arange(n_at)) and np.all(cell[:n_at] == 0)
    keys = {(int(a), tuple(int(c) for c in cc)) for a, cc in zip(atom, cell)}
    assert len(keys) == len(atom)  # no duplicates
    assert np.allclose(xyz, s.atom_xyz[atom] + cell @ LAT)
    # brute force: images within the atom's largest cutoff of some point of the cell
    pts = s.pt_xyz
    rng = range(-5, 6)
    for a in range(n_at):
        rc = max(s.fn_cutoff[f] for f in range(s.species_fn_offset[s.atom_species[a]],
                                               s.species_fn_offset[s.atom_species[a] + 1]))
        for n0 in rng:
            for n1 in rng:
                for n2 in rng:
                    p = s.atom_xyz[a] + np.array([n0, n1, n2]) @ LAT
                    if np.min(np.linalg.norm(pts - p, axis=1)) < rc:
                        assert (a, (n0, n1, n2)) in keys, (a, n0, n1, n2)


def test_basis_map_and_buffer_sizes():
    s = synth.periodic_cell(LAT, FRAC, [0, 1], SPECIES, n_grid=6)
    xyz, atom, cell = nao.nao_periodic_images(s.atom_xyz, LAT, 4.5)
    fm, fi = nao.nao_periodic_basis_map(s, atom)
    per_atom = [sum(2 * int(s.fn_l[f]) + 1 for f in range(s.species_fn_offset[sp], s.species_fn_offset[sp + 1]))
                for sp in s.atom_species]
    first = np.concatenate([[0], np.cumsum(per_atom)])
    assert len(fm) == sum(per_atom[a] for a in atom)
    pos = 0
    for k, a in enumerate(atom):
        assert np.array_equal(fm[pos:pos + per_atom[a]], np.arange(first[a], first[a + 1]))
        assert np.all(fi[pos:pos + per_atom[a]] == k)
        pos += per_atom[a]
    # the image system has exactly that basis
    assert synth.image_system(s, xyz, atom).n_basis == len(fm)
    # too-small output: the count comes back with an error status
    lib = nao.load()
    x = np.ascontiguousarray(s.atom_xyz)
    A = np.ascontiguousarray(LAT.reshape(9))
    n = C.c_int32(0)
    assert lib.nao_periodic_images(x.ctypes.data, s.n_atoms, A.ctypes.data, 4.5, 1, None, None, None, C.byref(n)) != 0
    assert n.value == len(atom)


def test_periodic_grid_is_the_trapezoid_rule_of_the_cell():
    """Weights sum to the cell volume; a lattice-periodic trigonometric polynomial of degree below
    the grid size integrates to its exact mean times the volume (here: the constant term)."""
    s = synth.periodic_cell(LAT, FRAC, [0, 1], SPECIES, n_grid=(8, 9, 10))
    V = abs(np.linalg.det(LAT))
    assert np.isclose(s.pt_w.sum(), V, rtol=1e-14)
    f = s.pt_xyz @ np.linalg.inv(LAT)
    t = 2 * np.pi * f
    g = 0.7 + np.cos(3 * t[:, 0]) * np.sin(2 * t[:, 1]) + np.cos(t[:, 0] - 4 * t[:, 2]) + np.sin(5 * t[:, 1])
    assert abs(np.dot(s.pt_w, g) - 0.7 * V) <= 1e-12 * V
    v = synth.periodic_potential(s)
    assert abs(np.dot(s.pt_w, v) - (-1.0) * V) <= 1e-12 * V


def test_bloch_map_checks():
    """The binding rejects maps that would index outside h(k) or the image table (the kernel
    also skips and counts such entries, so that they can never move a device access)."""
    import pytest

    torch = pytest.importorskip("torch")
    i32 = lambda a: torch.tensor(a, dtype=torch.int32)
    cell = i32([0, 0, 0, 1, 0, 0])  # two images
    assert nao.check_bloch_maps(i32([0, 1, 2]), i32([0, 1, 1]), cell, 3) == 2
    for fm, fi, c in ((i32([0, 3, 2]), i32([0, 1, 1]), cell), (i32([-1, 1, 2]), i32([0, 1, 1]), cell),
                      (i32([0, 1, 2]), i32([0, 2, 1]), cell), (i32([0, 1, 2]), i32([0, -1, 1]), cell),
                      (i32([0, 1, 2]), i32([0, 1, 1]), i32([0, 0, 0, 1]))):
        with pytest.raises(ValueError):
            nao.check_bloch_maps(fm, fi, c, 3)
