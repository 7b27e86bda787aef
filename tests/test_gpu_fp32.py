"""GPU parity of the FP32 path against the FP64 oracle: e_H, e_n <= 1e-6 (tests/_metrics.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import raw_rel_err, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-6


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def water():
    s = synth.config_water()
    o = oracle.Oracle(s)
    v = s.potential()
    P = synth.density_matrix(s, 0)
    H, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    n, D, ne = o.density(s.pt_xyz, P, s.pt_w)
    g = nao.Grid(s, device=0)
    yield dict(s=s, o=o, v=v, P=P, H=H, A=A, n=n, D=D, ne=ne, g=g)
    g.close()


def test_basis_functions_fp32(water):
    s, o, g = water["s"], water["o"], water["g"]
    bo, pp, ro, ri = g.batches()
    nonempty = np.nonzero(np.diff(ro))[0]
    for b in [int(nonempty[0]), int(nonempty[len(nonempty) // 2]), int(nonempty[-1])]:
        phi, grad = g.evaluate_batch(b, prec="fp32")
        pts = s.pt_xyz[pp[bo[b]:bo[b + 1]]]
        rphi, rgrad = o.eval_dense(pts)
        rel = ri[ro[b]:ro[b + 1]]
        rphi = rphi[:, rel].T
        rgrad = np.transpose(rgrad[:, rel, :], (2, 1, 0))
        scale = np.maximum(np.abs(rphi).max(axis=1, keepdims=True), 1e-300)
        assert np.all(np.abs(phi.cpu().numpy() - rphi) <= 2e-6 * scale)
        gscale = np.maximum(np.abs(rgrad).max(axis=(0, 2), keepdims=True), 1e-300)
        assert np.all(np.abs(grad.cpu().numpy() - rgrad) <= 2e-6 * gscale)


def test_hamiltonian_fp32(water):
    g = water["g"]
    H = g.integrate_h(cuda(water["v"]), prec="fp32").cpu().numpy()
    assert np.array_equal(H, H.T)
    e = rel_err(H, water["H"], water["A"])
    print(f"fp32 e_H={e:.2e} raw={raw_rel_err(H, water['H'], water['A']):.2e}")
    assert e <= TOL


def test_density_fp32(water):
    g = water["g"]
    n, ne = g.update_density(cuda(water["P"]), prec="fp32")
    e = rel_err(n.cpu().numpy(), water["n"], water["D"])
    print(f"fp32 e_n={e:.2e}")
    assert e <= TOL
    assert abs(float(ne.item()) - water["ne"]) <= TOL * abs(water["ne"])


@pytest.mark.parametrize("B", [1, 64, 1024])
def test_fp32_independent_of_batch_size(water, B):
    with nao.Grid(water["s"], device=0, max_batch_points=B) as g:
        H = g.integrate_h(cuda(water["v"]), prec="fp32").cpu().numpy()
        n, _ = g.update_density(cuda(water["P"]), prec="fp32")
        assert rel_err(H, water["H"], water["A"]) <= TOL
        assert rel_err(n.cpu().numpy(), water["n"], water["D"]) <= TOL
