"""The meta-GGA term (nao_integrate_h_tau): H_ij += sum_p w_p vtau_p 1/2 grad phi_i . grad phi_j,
carried as a weight on the three gradient columns, against the oracle on every precision path
(e_H <= 1e-12 FP64, 1e-10 split, 1e-6 FP32); vtau = 1 with the tau term alone reproduces the
kinetic term of nao_integrate_h on the device."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-6, "split": 1e-10}
ALL = nao.NAO_TERM_POTENTIAL | nao.NAO_TERM_KINETIC | nao.NAO_TERM_TAU


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def water():
    s = synth.config_water()
    o = oracle.Oracle(s)
    v = s.potential()
    rng = np.random.Generator(np.random.PCG64(41))
    vtau = rng.uniform(-0.3, 1.2, s.n_points)  # either sign: the negative columns take the negate path
    H, A = o.hamiltonian_tau(s.pt_xyz, s.pt_w, v, vtau, ALL)
    Ht, At = o.hamiltonian_tau(s.pt_xyz, s.pt_w, None, vtau, nao.NAO_TERM_TAU)
    g = nao.Grid(s, device=0, max_batch_points=200)
    yield dict(s=s, v=v, vtau=vtau, H=H, A=A, Ht=Ht, At=At, g=g)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split"])
def test_tau_term(water, prec):
    g = water["g"]
    H = g.integrate_h_tau(cuda(water["v"]), cuda(water["vtau"]), ALL, prec=prec)
    Ht = g.integrate_h_tau(None, cuda(water["vtau"]), nao.NAO_TERM_TAU, prec=prec)
    torch.cuda.synchronize()
    g.sync()
    e = rel_err(H.cpu().numpy(), water["H"], water["A"])
    et = rel_err(Ht.cpu().numpy(), water["Ht"], water["At"])
    print(f"{prec}: e_H (all terms) = {e:.2e}, e_H (tau alone) = {et:.2e}")
    assert e <= TOL[prec] and et <= TOL[prec]


def test_tau_one_is_kinetic(water):
    g = water["g"]
    ones = torch.ones(g.n_points, dtype=torch.float64, device="cuda")
    Ht = g.integrate_h_tau(None, ones, nao.NAO_TERM_TAU, prec="fp64").cpu().numpy()
    Hk = g.integrate_h(None, nao.NAO_TERM_KINETIC, prec="fp64").cpu().numpy()
    assert np.max(np.abs(Ht - Hk)) <= 1e-14 * np.abs(Hk).max()


def test_tau_rejections(water):
    g = water["g"]
    with pytest.raises(Exception):
        g.integrate_h_tau(None, None, nao.NAO_TERM_TAU)  # the tau term needs vtau
    with pytest.raises(Exception):
        g.integrate_h_tau(None, None, 8)  # unknown term bit
