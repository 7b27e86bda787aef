"""Local Pulay force terms on the GPU (Sec. 2): the matrix elements M^c = <d_c phi_i| -1/2 lap + v
|phi_j> and S^c = <d_c phi_i|phi_j> against the oracle, and the forces 2 sum_{i on a} sum_j
(n_ij M^c_ij - q_ij S^c_ij) against the oracle's point-by-point definition (<= 1e-11 of the
largest force).

The matrices are checked at the scale of the matrix (max |dM| <= 1e-14 of the largest magnitude
sum: FP64 rounding) and element by element with the metric of tests/_metrics.py. Elements whose
magnitude sum is ~1e-10 of the largest are products of function tails within a few 1e-3 bohr of
their cutoffs, where the spline and its derivative keep only absolute accuracy (R ~ (rc - r)^3,
R' ~ (rc - r)^2; tests/_metrics.py): on the molecule below two such elements differ by ~1e-7 of
themselves, 5e-16 of the largest element. The element-wise bar is therefore 1e-6 for these
matrices (1e-12 holds on water, where no element is made of tails only).

The FP32 path (FP64 derivatives rounded once to FP32, products in FP32) is held to 1e-6 element
by element and at the matrix scale, and the forces to 1e-5 of the largest force (each force sums
n_ij M_ij over a row block, where FP32 rounding of the elements adds up)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(s, batch_points, seed, elementwise=1e-6, prec="fp64"):
    o = oracle.Oracle(s)
    v = s.potential()
    P = synth.density_matrix(s, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    X = rng.normal(size=(o.nb, o.nb))
    Q = (X + X.T) / 10
    Mref, Sref, AM, AS = o.pulay_matrices(s.pt_xyz, s.pt_w, v)
    Fref = o.pulay_forces(s.pt_xyz, s.pt_w, v, P, Q)
    with nao.Grid(s, device=0, max_batch_points=batch_points) as g:
        M0 = torch.full((3, g.nb, g.nb), float("nan"), dtype=torch.float64, device="cuda")
        S0 = torch.full((3, g.nb, g.nb), float("nan"), dtype=torch.float64, device="cuda")
        M, S = g.pulay_matrices(cuda(v), prec=prec, M=M0, S=S0)
        F = g.pulay_forces(cuda(P), cuda(Q), M, S)
        torch.cuda.synchronize()
        g.sync()
        M, S, F = M.cpu().numpy(), S.cpu().numpy(), F.cpu().numpy()
    eF = np.max(np.abs(F - Fref)) / np.abs(Fref).max()
    print(f"{prec} forces: {eF:.2e}")
    assert eF <= (1e-11 if prec == "fp64" else 1e-5)
    for c in range(3):
        em, es = rel_err(M[c], Mref[c], AM[c]), rel_err(S[c], Sref[c], AS[c])
        am = np.max(np.abs(M[c] - Mref[c])) / AM[c].max()
        a_s = np.max(np.abs(S[c] - Sref[c])) / AS[c].max()
        print(f"component {c}: e_M = {em:.2e}, e_S = {es:.2e}, at the matrix scale {am:.2e}, {a_s:.2e}")
        scale = 1e-14 if prec == "fp64" else 1e-6
        assert am <= scale and a_s <= scale
        assert em <= elementwise and es <= elementwise


def test_pulay_water():
    _check(synth.config_water(), 200, 3, elementwise=1e-12)


def test_pulay_molecule_with_f_functions():
    _check(synth.random_molecule(4, 5119, n_rad=12, n_theta=5, n_phi=6), 120, 4)


def test_pulay_fp32_water():
    _check(synth.config_water(), 200, 3, elementwise=1e-6, prec="fp32")


def test_pulay_fp32_molecule_with_f_functions():
    _check(synth.random_molecule(4, 5119, n_rad=12, n_theta=5, n_phi=6), 120, 4, prec="fp32")


def test_pulay_rejects_the_split_path():
    s = synth.config_water(n_rad=8, n_theta=4, n_phi=5)
    with nao.Grid(s, device=0) as g:
        with pytest.raises(Exception):
            g.pulay_matrices(None, prec="split")
