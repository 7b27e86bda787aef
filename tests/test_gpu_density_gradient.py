"""Density gradient on the GPU (Sec. 2: grad n = 2 sum_ij grad phi_i P_ij phi_j) against the
oracle: e = max |d grad n| / max(D^g, 1e-10 max D^g) per component, D^g the sum of the term
magnitudes (tests/_metrics.py), <= 1e-12 (FP64), <= 1e-10 (split) and <= 1e-6 (FP32); n from
the same call meets the density bars."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-6, "split": 1e-10}


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def water():
    s = synth.config_water()
    o = oracle.Oracle(s)
    P = synth.density_matrix(s, 0)
    gref, Dg = o.density_gradient(s.pt_xyz, P)
    n, D, ne = o.density(s.pt_xyz, P, s.pt_w)
    g = nao.Grid(s, device=0, max_batch_points=200)
    yield dict(s=s, P=P, gref=gref, Dg=Dg, n=n, D=D, ne=ne, g=g)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split"])
def test_density_gradient_water(water, prec):
    g = water["g"]
    # outputs pre-filled with NaN: every point (also those of batches without functions) is written
    n0 = torch.full((g.n_points,), float("nan"), dtype=torch.float64, device="cuda")
    g0 = torch.full((3, g.n_points), float("nan"), dtype=torch.float64, device="cuda")
    n, grad, ne = g.density_gradient(cuda(water["P"]), prec=prec, n=n0, grad=g0)
    torch.cuda.synchronize()
    g.sync()
    grad = grad.cpu().numpy()
    for c in range(3):
        e = rel_err(grad[c], water["gref"][:, c], water["Dg"][:, c])
        print(f"{prec}: grad n component {c}: e = {e:.2e}")
        assert e <= TOL[prec]
    assert rel_err(n.cpu().numpy(), water["n"], water["D"]) <= TOL[prec]
    assert abs(ne.item() - water["ne"]) <= TOL[prec] * abs(water["ne"])


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_density_gradient_grouped(prec):
    systems, bs = synth.molecule_set(6, seed=3100, n_min=3, n_max=10, b_min=20, b_max=400, n_rad=14, n_theta=5, n_phi=6)
    Ps = [synth.density_matrix(s, 40 + k) for k, s in enumerate(systems)]
    with nao.Grid(systems, device=0, batch_points=bs) as g:
        ns = [torch.full((st["n_points"],), float("nan"), dtype=torch.float64, device="cuda") for st in g.systems]
        gs = [torch.full((3, st["n_points"]), float("nan"), dtype=torch.float64, device="cuda") for st in g.systems]
        nes = [torch.empty(1, dtype=torch.float64, device="cuda") for _ in g.systems]
        nao.nao_update_density_gradient_many(g.h, [cuda(P) for P in Ps], prec, ns, gs, nes)
        torch.cuda.synchronize()
        g.sync()
        for k, s in enumerate(systems):
            o = oracle.Oracle(s)
            gref, Dg = o.density_gradient(s.pt_xyz, Ps[k])
            gk = gs[k].cpu().numpy()
            for c in range(3):
                assert rel_err(gk[c], gref[:, c], Dg[:, c]) <= TOL[prec], (k, c)
