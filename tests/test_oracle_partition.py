"""Pins for the oracle's batch partition (Sec. 3.3.1) and reduced basis sets (Sec. 3.3.2).

Partition rule: recursive bisection into ceil(n/B) batches; each split cuts along the axis
of largest extent (ties x < y < z) after ordering by (coordinate, index); the left part
holds floor(n * floor(k/2) / k) points. Pins: the batches cover every point exactly once,
hold at most B points, number ceil(n/B) and are near-equal; each split is a plane; the tie
rule picks x on a cubic lattice; points inside a batch are ordered along one axis.
Relevance rule: function (A, f, m) is in nnz(b) iff some point of b has
(dx*dx + dy*dy) + dz*dz < rc_f*rc_f; pinned by a numpy brute-force scan of every
(point, function) pair (numpy rounds each operation separately, as the rule requires).
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1912_06636_gb300 import synth


def _check_cover(off, perm, n, B):
    assert off[0] == 0 and off[-1] == n
    assert np.array_equal(np.sort(perm), np.arange(n))
    sizes = np.diff(off)
    assert len(sizes) == -(-n // B)
    assert sizes.max() <= B
    k = len(sizes)
    assert sizes.min() >= n // k - 1


@pytest.mark.parametrize("n,B", [(1, 200), (199, 200), (200, 200), (201, 200), (13200, 200), (5003, 97), (4096, 1)])
def test_partition_cover_and_sizes(n, B):
    rng = np.random.Generator(np.random.PCG64(n))
    pts = rng.standard_normal((n, 3)) * np.array([3.0, 1.0, 0.5])
    off, perm = Oracle.partition(pts, B)
    _check_cover(off, perm, n, B)


def test_config_water_gives_66_batches_of_200():
    s = synth.config_water()
    off, perm = Oracle.partition(s.pt_xyz, 200)
    assert len(off) == 67 and np.all(np.diff(off) == 200)


def test_first_cut_is_a_plane_on_largest_axis_and_ties_pick_x():
    g = np.arange(8, dtype=np.float64)
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)  # equal extents
    pts = pts[np.random.Generator(np.random.PCG64(1)).permutation(len(pts))]
    off, perm = Oracle.partition(pts, 64)  # k = 8 -> left holds 4 batches
    left = perm[: off[4]]
    right = perm[off[4]:]
    assert pts[left, 0].max() <= pts[right, 0].min()
    # stretch along z: the first cut must be along z
    pts2 = pts * np.array([1.0, 1.0, 3.0])
    off2, perm2 = Oracle.partition(pts2, 64)
    assert pts2[perm2[: off2[4]], 2].max() <= pts2[perm2[off2[4]:], 2].min()


def test_points_inside_a_batch_are_ordered_along_an_axis():
    s = synth.config_water()
    off, perm = Oracle.partition(s.pt_xyz, 200)
    for b in range(len(off) - 1):
        q = s.pt_xyz[perm[off[b]:off[b + 1]]]
        assert any(np.all(np.diff(q[:, c]) >= 0) for c in range(3))


def test_partition_left_part_is_rounded_down():
    """Worked by hand from the rule. Five points on a line, B = 2: k = 3, the left part holds
    floor(5 * 1 / 3) = 1 point; the remaining four give k = 2 and floor(4 * 1 / 2) = 2. With 201
    points and B = 200 the cut is floor(201 / 2) = 100."""
    x = np.array([3.0, 0.0, 4.0, 1.0, 2.0])
    pts = np.stack([x, np.zeros(5), np.zeros(5)], 1)
    off, perm = Oracle.partition(pts, 2)
    assert off.tolist() == [0, 1, 3, 5]
    assert perm.tolist() == [1, 3, 4, 0, 2]
    line = np.stack([np.arange(201.0), np.zeros(201), np.zeros(201)], 1)
    off, perm = Oracle.partition(line, 200)
    assert off.tolist() == [0, 100, 201] and perm.tolist() == list(range(201))


def test_equal_coordinates_keep_index_order():
    """Worked by hand from the rule: equal coordinates along the cut axis are ordered by point
    index. The x extent (1) is the largest, so the cut is along x; the sorted order is
    (x=0: points 1, 3), (x=1: points 0, 2)."""
    pts = np.array([[1.0, 0.0, 0.0], [0.0, 0.1, 0.0], [1.0, 0.2, 0.0], [0.0, 0.3, 0.0]])
    off, perm = Oracle.partition(pts, 2)
    assert off.tolist() == [0, 2, 4] and perm.tolist() == [1, 3, 0, 2]


def _brute_relevance(sys, pts, off, perm):
    rel_off, rel = [0], []
    for b in range(len(off) - 1):
        q = pts[perm[off[b]:off[b + 1]]]
        base = 0
        for A, sp in enumerate(sys.atom_species):
            d = q - sys.atom_xyz[A][None, :]
            r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
            for f in range(sys.species_fn_offset[sp], sys.species_fn_offset[sp + 1]):
                nm = 2 * int(sys.fn_l[f]) + 1
                rc = float(sys.fn_cutoff[f])
                if np.any(r2 < rc * rc):
                    rel.extend(range(base, base + nm))
                base += nm
        rel_off.append(len(rel))
    return np.array(rel_off), np.array(rel, dtype=np.int32)


def test_relevance_matches_brute_force_scan():
    sp_a = synth.Species([0, 1, 2], [1.0, 0.5, 0.7], rc=3.5)
    sp_b = synth.Species([0, 1], [1.2, 0.4], rc=2.5)
    atoms = [[0, 0, 0], [4.0, 0.5, 0], [-3.0, 2.0, 1.0], [1.0, -4.0, 0.5]]
    s = synth.make_system(atoms, [0, 1, 0, 1], [sp_a, sp_b], 20, 6, 7)
    o = Oracle(s)
    off, perm = Oracle.partition(s.pt_xyz, 37)
    ro, ri = o.relevance(s.pt_xyz, off, perm)
    bo, bi = _brute_relevance(s, s.pt_xyz, off, perm)
    assert np.array_equal(ro, bo) and np.array_equal(ri, bi)
    assert np.diff(ro).min() == 0 and np.diff(ro).max() > 0  # empty and non-empty batches both occur


def test_relevance_boundary_is_strict():
    sp = synth.Species([0, 1], [1.0, 0.5], rc=2.5)
    s = synth.make_system([[0.0, 0.0, 0.0]], [0], [sp], 4, 2, 3)
    o = Oracle(s)
    cases = [([2.5, 0.0, 0.0], False), ([0.0, -2.5, 0.0], False), ([1.5, 2.0, 0.0], False),
             ([np.nextafter(2.5, 0.0), 0.0, 0.0], True), ([2.5, 1e-3, 0.0], False), ([1.5, 1.9999999, 0.0], True)]
    for p, want in cases:
        pts = np.array([p])
        ro, ri = o.relevance(pts, np.array([0, 1]), np.array([0]))
        assert (ro[1] == 4) == want, (p, ro)
