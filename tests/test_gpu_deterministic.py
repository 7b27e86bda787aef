"""The deterministic option (nao_options.deterministic): H accumulated as 128-bit fixed-point
integers is bitwise the same from run to run, with and without CUDA graphs, on every precision
path, and agrees with the FP64-atomic H and with the oracle within each path's tolerance. The
grouped molecule set (many batches adding into the same H elements) and diamond8 make the
order of the FP64 atomic additions vary."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-6, "split": 1e-10}


@pytest.fixture(scope="module")
def cell():
    s = synth.config_diamond64(n_rad=30, n_theta=8, n_phi=9, cells=1)
    v = s.potential()
    H, A = oracle.Oracle(s).hamiltonian(s.pt_xyz, s.pt_w, v)
    return dict(s=s, v=torch.from_numpy(v).cuda(), H=H, A=A)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split"])
def test_bitwise_reproducible(cell, prec):
    runs = []
    for graph in (0, 1, 1, 0):
        with nao.Grid(cell["s"], device=0, max_batch_points=100, deterministic=1, capture_graph=graph) as g:
            H = g.integrate_h(cell["v"], prec=prec)
            H2 = g.integrate_h(cell["v"], prec=prec)  # a second call on the same handle (accumulators re-zeroed)
            torch.cuda.synchronize()
            g.sync()
            runs.append(H.cpu().numpy())
            assert torch.equal(H, H2)
    for r in runs[1:]:
        assert np.array_equal(r, runs[0])
    Hd = runs[0]
    assert np.array_equal(Hd, Hd.T)
    assert rel_err(Hd, cell["H"], cell["A"]) <= TOL[prec]
    with nao.Grid(cell["s"], device=0, max_batch_points=100) as g:
        Ha = g.integrate_h(cell["v"], prec=prec).cpu().numpy()
    # the same sums, added exactly instead of in FP64 in some order
    assert rel_err(Hd, Ha, cell["A"]) <= 1e-13


def test_grouped_reproducible():
    systems, bs = synth.molecule_set(6, seed=3300, n_min=3, n_max=10, b_min=20, b_max=400, n_rad=14, n_theta=5, n_phi=6)
    vs = [torch.from_numpy(s.potential()).cuda() for s in systems]
    out = []
    for _ in range(2):
        with nao.Grid(systems, device=0, batch_points=bs, deterministic=1) as g:
            Hs = g.integrate_h_many(vs, prec="split")
            torch.cuda.synchronize()
            g.sync()
            out.append([h.cpu().numpy() for h in Hs])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    for s, v, h in zip(systems, vs, out[0]):
        H, A = oracle.Oracle(s).hamiltonian(s.pt_xyz, s.pt_w, v.cpu().numpy())
        assert rel_err(h, H, A) <= TOL["split"]


def test_option_is_checked():
    s = synth.config_water(n_rad=6, n_theta=3, n_phi=4)
    with pytest.raises(nao.NaoError) as e:
        nao.Grid(s, device=0, deterministic=2)
    assert e.value.code == nao.NAO_ERR_INVALID_ARG
