"""Periodic Hamiltonian on the GPU (Eq. HamPeriodic): h^uc integrated by the finite-system code
over the unit cell's points with the cell's periodic images as atoms, then the Bloch sum
h_ij(k) = sum h^uc_{i'j'} e^{i k.(T_j' - T_i')} on the device, against the oracle's h(k) from
the Bloch functions themselves: e = max |dh| / max(A, 1e-10 max A) <= 1e-12 (FP64), 1e-10
(split), A the oracle's magnitude sums; the overlap s(k) likewise."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

LAT = np.diag([6.0, 6.5, 7.0]) + np.array([[0, 0, 0], [0.8, 0, 0], [0, 0.5, 0]])
SPECIES = [synth.Species(ls=[0, 1], alphas=[1.0, 0.8], rc=4.0, Z=1.0),
           synth.Species(ls=[0, 0, 1, 2], alphas=[2.0, 0.7, 1.1, 0.9], rc=4.5, Z=2.0)]
FRAC = [[0.11, 0.23, 0.31], [0.57, 0.61, 0.72]]
TOL = {"fp64": 1e-12, "split": 1e-10}


@pytest.fixture(scope="module")
def cell():
    s = synth.periodic_cell(LAT, FRAC, [0, 1], SPECIES, n_grid=10, max_batch_points=120)
    xyz, atom, cellidx = nao.nao_periodic_images(s.atom_xyz, LAT, float(np.max(s.fn_cutoff)))
    simg = synth.image_system(s, xyz, atom)
    fm, fi = nao.nao_periodic_basis_map(s, atom)
    B = 2 * np.pi * np.linalg.inv(LAT).T
    kpts = np.array([[0.0, 0.0, 0.0], [0.31, -0.17, 0.12], B[0] / 2 + B[2] / 3])
    v = synth.periodic_potential(s)
    o = oracle.Oracle(s)
    refs = [o.periodic_h(LAT, 2, s.pt_xyz, s.pt_w, k, v) for k in kpts]
    srefs = [o.periodic_h(LAT, 2, s.pt_xyz, s.pt_w, k, None, oracle.TERM_POTENTIAL) for k in kpts]
    return dict(s=s, simg=simg, fm=fm, fi=fi, cell=cellidx, kpts=kpts, v=v, refs=refs, srefs=srefs)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_bloch_hamiltonian_and_overlap(cell, prec):
    s = cell["s"]
    dev = "cuda"
    fm = torch.from_numpy(cell["fm"]).to(dev)
    fi = torch.from_numpy(cell["fi"]).to(dev)
    ci = torch.from_numpy(np.ascontiguousarray(cell["cell"], dtype=np.int32)).to(dev)
    k = torch.from_numpy(cell["kpts"]).to(dev)
    with nao.Grid(cell["simg"], device=0, max_batch_points=120) as g:
        assert g.nb == len(cell["fm"])
        Huc = g.integrate_h(torch.from_numpy(cell["v"]).to(dev), prec=prec)
        Suc = g.overlap(prec=prec)
        err = torch.full((1,), -1, dtype=torch.int32, device=dev)
        Hk = nao.nao_bloch_sum(Huc, fm, fi, ci, LAT, k, s.n_basis, err=err).cpu().numpy()
        assert int(err.item()) == 0  # no map entry was skipped
        Sk = nao.nao_bloch_sum(Suc, fm, fi, ci, LAT, k, s.n_basis).cpu().numpy()
        torch.cuda.synchronize()
        g.sync()
    for q in range(len(cell["kpts"])):
        Href, A = cell["refs"][q]
        Sref, AS = cell["srefs"][q]
        eh, es = rel_err(Hk[q], Href, A), rel_err(Sk[q], Sref, AS)
        print(f"{prec} k{q}: e_h = {eh:.2e}, e_s = {es:.2e}")
        assert eh <= TOL[prec] and es <= TOL[prec]
