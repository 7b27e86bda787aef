"""The library's host set-up steps against the oracle, on the CPU (no GPU, no handle):
the batch partition (Sec. 3.3.1) bit-exact, and the natural cubic spline of the radial tables
(Sec. 3.2.1) to rounding. nao_grid_create runs the same host code, so these parity checks cover it
without a GPU; the GPU tests check the same partition again through nao_export_batches."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_1912_06636_gb300 import nao, synth


def _same_partition(pts, B):
    off, perm = nao.nao_partition_points(pts, B)
    ooff, operm = Oracle.partition(pts, B)
    assert np.array_equal(off, ooff), (len(off), len(ooff))
    assert np.array_equal(perm, operm)
    return off, perm


@pytest.mark.parametrize("n,B", [(1, 200), (199, 200), (200, 200), (201, 200), (5003, 97), (4096, 1), (3000, 7)])
def test_partition_random_clouds(n, B):
    rng = np.random.Generator(np.random.PCG64(100 + n))
    _same_partition(rng.standard_normal((n, 3)) * np.array([3.0, 1.0, 0.5]), B)


def test_partition_ties_duplicates_and_worked_examples():
    g = np.arange(8, dtype=np.float64)
    cube = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)  # equal extents, many equal keys
    cube = cube[np.random.Generator(np.random.PCG64(2)).permutation(len(cube))]
    for B in (64, 50, 13):
        _same_partition(cube, B)
    dup = np.repeat(np.random.Generator(np.random.PCG64(3)).standard_normal((40, 3)), 5, axis=0)  # each point 5 times
    _same_partition(dup, 9)
    _same_partition(np.zeros((17, 3)), 4)  # all points equal: every cut is by index
    off, perm = _same_partition(np.stack([[3.0, 0.0, 4.0, 1.0, 2.0], np.zeros(5), np.zeros(5)], 1), 2)
    assert off.tolist() == [0, 1, 3, 5] and perm.tolist() == [1, 3, 4, 0, 2]


def test_partition_of_molecular_grids():
    s = synth.config_water()
    off, _ = _same_partition(s.pt_xyz, 200)
    assert len(off) == 67 and np.all(np.diff(off) == 200)
    m = synth.random_molecule(6, 77, n_rad=10, n_theta=5, n_phi=6)
    for B in (37, 120, 300):
        _same_partition(m.pt_xyz, B)


def test_partition_rejections():
    with pytest.raises(nao.NaoError):
        nao.nao_partition_points(np.array([[0.0, np.nan, 0.0]]), 10)
    with pytest.raises(nao.NaoError):
        nao.nao_partition_points(np.zeros((5, 3)), 0)
    lib = nao.load()
    import ctypes as C

    x = np.random.Generator(np.random.PCG64(4)).standard_normal((100, 3))
    nb = C.c_int64(0)
    st = lib.nao_partition_points(x.ctypes.data, 100, 10, 3, None, None, C.byref(nb))  # room for 3 of 10 batches
    assert st == 1 and nb.value == 10


def test_radial_spline_equals_the_oracle_spline():
    s = synth.random_molecule(3, 91, n_rad=4, n_theta=2, n_phi=3)
    o = Oracle(s)
    delta = math.log(s.r_last / s.r0) / (s.n_rgrid - 1)
    rng = np.random.Generator(np.random.PCG64(5))
    for f in range(len(s.fn_l)):
        coef = nao.nao_radial_spline(s.fn_table[f])
        assert coef.shape == (s.n_rgrid - 1, 4)
        assert np.array_equal(coef[:, 0], s.fn_table[f, :-1])  # c0 is the node value
        scale = np.abs(s.fn_table[f]).max()
        rc = float(s.fn_cutoff[f])
        for r in np.exp(rng.uniform(math.log(1.5 * s.r0), math.log(0.999 * rc), 300)):
            sc = math.log(r / s.r0) / delta
            k = min(int(math.floor(sc)), s.n_rgrid - 2)
            t = sc - k
            c = coef[k]
            R = c[0] + t * (c[1] + t * (c[2] + t * c[3]))
            dRds = c[1] + t * (2 * c[2] + 3 * t * c[3])
            Ro, dRo = o.radial(f, r)
            assert abs(R - Ro) <= 1e-13 * scale
            assert abs(dRds - dRo * r * delta) <= 1e-12 * scale


def test_radial_spline_rejections():
    with pytest.raises(nao.NaoError):
        nao.nao_radial_spline(np.array([1.0, 2.0, 3.0]))  # fewer than 4 nodes
    with pytest.raises(nao.NaoError):
        nao.nao_radial_spline(np.array([1.0, np.inf, 3.0, 4.0, 5.0]))
