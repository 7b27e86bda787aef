"""Locality of the method (Sec. 3.3.2), from the oracle's partition and reduced basis sets on the
CPU: the functions relevant to a batch stay bounded as the system grows, so the work of the
method, the (batch, function) pairs, grows linearly with the system."""
import numpy as np

from oracle import Oracle
from paper_1912_06636_gb300 import synth


def test_reduced_basis_size_does_not_grow_with_the_system():
    """Sec. 3.3.2: with compact basis functions and spatially compact batches, the number of
    functions relevant to a batch is bounded by what reaches a batch-sized region, not by the
    system. Chains of 4 to 64 atoms (3 bohr apart, 9 functions per atom, cutoff 5 bohr), keeping
    the grid points within the cutoff of some atom (the only points where any function is
    nonzero), partitioned into batches of at most 60 points: the largest |nnz(B)| stays at four
    or five atoms' functions (36 or 45) and the mean levels off, while the batch count and the
    total number of (batch, function) pairs, the work of the method, double with the atoms."""
    sp = synth.Species(ls=[0, 1, 2], alphas=[0.8, 0.5, 0.6], rc=5.0)
    stats = {}
    for n_atoms in (4, 16, 32, 64):
        atoms = np.array([[3.0 * k, 0.0, 0.0] for k in range(n_atoms)])
        s = synth.make_system(atoms, [0] * n_atoms, [sp], n_rad=12, n_theta=5, n_phi=6, max_batch_points=60)
        d2 = ((s.pt_xyz[:, None, :] - atoms[None, :, :]) ** 2).sum(-1).min(axis=1)
        pts = np.ascontiguousarray(s.pt_xyz[d2 < sp.rc ** 2])
        off, perm = Oracle.partition(pts, 60)
        ro, _ = Oracle(s).relevance(pts, off, perm)
        nnz = np.diff(ro)
        stats[n_atoms] = (len(off) - 1, int(nnz.max()), float(nnz.mean()), int(nnz.sum()), s.n_basis)
    assert stats[4][1] == stats[4][4]                      # a small system: the whole basis
    for n in (16, 32, 64):
        assert stats[n][1] <= 45, stats                     # then at most five atoms' functions
    assert abs(stats[64][2] - stats[32][2]) <= 0.1 * stats[32][2]
    for a, b in ((16, 32), (32, 64)):
        assert 1.9 <= stats[b][0] / stats[a][0] <= 2.1      # batches in proportion to atoms
        assert 1.9 <= stats[b][3] / stats[a][3] <= 2.2      # so are the (batch, function) pairs
