"""The oracle spread over threads (tests/_oracle_par.py) equals the single-threaded oracle: the
integrals differ only by the order in which the slices' compensated sums are added (well below
1e-14 of the magnitude sums), the per-point densities are identical."""
import numpy as np

import oracle
from paper_1912_06636_gb300 import synth
from tests import _oracle_par
from tests._metrics import raw_rel_err


def test_threads_match_serial():
    s = synth.config_water(n_rad=12, n_theta=5, n_phi=6)
    v = s.potential()
    P = synth.density_matrix(s, 0)
    o = oracle.Oracle(s)
    H, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    Hp, Ap = _oracle_par.hamiltonian(s, s.pt_xyz, s.pt_w, v)
    assert raw_rel_err(Hp, H, A) <= 1e-14 and raw_rel_err(Ap, A, A) <= 1e-14
    F = np.array([0, 3, 7, 11, 19])
    Hb, Ab = o.hamiltonian_block(F, s.pt_xyz, s.pt_w, v)
    Hbp, Abp = _oracle_par.hamiltonian_block(s, F, s.pt_xyz, s.pt_w, v)
    assert raw_rel_err(Hbp, Hb, Ab) <= 1e-14
    assert np.allclose(Hb, H[np.ix_(F, F)], rtol=0, atol=1e-14 * A.max())
    n, D, _ = o.density(s.pt_xyz, P)
    n_p, D_p = _oracle_par.density(s, s.pt_xyz, P)
    assert np.array_equal(n, n_p) and np.array_equal(D, D_p)
