"""Density Hessian on the GPU (Sec. 2: d_a d_b n = 2 sum_ij P_ij (phi_i d_a d_b phi_j + d_a phi_i
d_b phi_j), six components) against the oracle's plain second derivative of Eq. Density:
e = max |dH| / max(D^h, 1e-10 max D^h) per component (D^h the sum of the term magnitudes,
tests/_metrics.py) <= 1e-12 in FP64, <= 1e-6 on the FP32 path (the FP64 derivatives rounded
once to FP32, products in FP32) and <= 1e-10 on the split path (the four products Phi P, (d_a Phi) P
as Ozaki slice products on the tensor cores); n, grad n and N_e from the same call meet the same
bars."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

NAMES = ["xx", "xy", "xz", "yy", "yz", "zz"]


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check_system(s, P, batch_points, tol=1e-12, prec="fp64"):
    o = oracle.Oracle(s)
    href, Dh = o.density_hessian(s.pt_xyz, P)
    gref, Dg = o.density_gradient(s.pt_xyz, P)
    nref, D, neref = o.density(s.pt_xyz, P, s.pt_w)
    with nao.Grid(s, device=0, max_batch_points=batch_points) as g:
        # outputs pre-filled with NaN: every point is written
        n0 = torch.full((g.n_points,), float("nan"), dtype=torch.float64, device="cuda")
        g0 = torch.full((3, g.n_points), float("nan"), dtype=torch.float64, device="cuda")
        h0 = torch.full((6, g.n_points), float("nan"), dtype=torch.float64, device="cuda")
        n, grad, hess, ne = g.density_hessian(cuda(P), prec=prec, n=n0, grad=g0, hess=h0)
        torch.cuda.synchronize()
        g.sync()
        hess = hess.cpu().numpy()
        grad = grad.cpu().numpy()
        for k in range(6):
            e = rel_err(hess[k], href[:, k], Dh[:, k])
            print(f"{prec} hessian {NAMES[k]}: e = {e:.2e}")
            assert e <= tol, NAMES[k]
        for c in range(3):
            assert rel_err(grad[c], gref[:, c], Dg[:, c]) <= tol
        assert rel_err(n.cpu().numpy(), nref, D) <= tol
        assert abs(ne.item() - neref) <= tol * abs(neref)
        # symmetric in (a, b) by construction, and the trace is the Laplacian of n
        assert np.all(np.isfinite(hess))


TOL = {"fp64": 1e-12, "fp32": 1e-6, "split": 1e-10}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split"])
def test_density_hessian_water(prec):
    s = synth.config_water()
    _check_system(s, synth.density_matrix(s, 0), 200, TOL[prec], prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split"])
def test_density_hessian_molecule_with_f_functions(prec):
    # species with d and f functions (l up to 3), several batches and atoms
    s = synth.random_molecule(5, 7311, n_rad=12, n_theta=5, n_phi=6)
    assert max(s.fn_l) >= 3
    _check_system(s, synth.density_matrix(s, 5), 120, TOL[prec], prec)


def test_density_hessian_rejects_grouped_handles():
    s = synth.config_water(n_rad=8, n_theta=4, n_phi=5)
    P = cuda(synth.density_matrix(s, 0))
    systems = [synth.config_water(n_rad=8, n_theta=4, n_phi=5), synth.random_molecule(3, 11, n_rad=8, n_theta=4, n_phi=5)]
    with nao.Grid(systems, device=0) as g:
        with pytest.raises(Exception):
            nao.nao_update_density_hessian(g.h, P, "fp64", torch.empty(10, device="cuda", dtype=torch.float64),
                                           torch.empty(30, device="cuda", dtype=torch.float64),
                                           torch.empty(60, device="cuda", dtype=torch.float64))
