"""The precision configuration at full size: a 375-atom two-species slab (15,000 basis
functions, 80 x 434 points per atom = 13,020,000 points, batches <= 200). Reported and checked
per precision: the maximum relative error of H over a sampled block of basis functions (all
points), and of n over sampled points, against the oracle, which computes them one by one
(tests/_metrics.py; FP64 1e-12, FP32 1e-6, split 1e-10), plus tr(PS) = N_e. P is
X X^T / 64 with X 15000 x 64 (low rank keeps the host generation short).
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = {"fp64": 1e-12, "fp32": 1e-6, "split": 1e-10}
# sampled basis functions: atoms of both species in several layers, every l
SAMPLE_F = np.array([0, 5, 17, 39, 40 * 12 + 3, 40 * 60 + 21, 40 * 130 + 30, 40 * 187 + 8, 40 * 188 + 36,
                     40 * 250 + 13, 40 * 301 + 27, 40 * 374 + 39])


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def slab():
    t0 = time.perf_counter()
    s = synth.config(2)
    v = s.potential()
    P = synth.density_matrix(s, 2, rank=64)
    t1 = time.perf_counter()
    o = oracle.Oracle(s)
    Hb, Ab = o.hamiltonian_block(SAMPLE_F, s.pt_xyz, s.pt_w, v)
    rng = np.random.Generator(np.random.PCG64(22))
    pidx = np.sort(rng.choice(s.n_points, 400, replace=False))
    n_s, D_s, _ = o.density(s.pt_xyz[pidx], P)
    t2 = time.perf_counter()
    print(f"slab: {s.n_atoms} atoms, {s.n_basis} basis functions, {s.n_points} points; "
          f"inputs {t1 - t0:.0f} s, oracle samples {t2 - t1:.0f} s")
    g = nao.Grid(s, device=0, max_batch_points=200)
    yield dict(s=s, v=v, P=P, Hb=Hb, Ab=Ab, pidx=pidx, n_s=n_s, D_s=D_s, g=g)
    g.close()


def test_slab_sizes(slab):
    g, s = slab["g"], slab["s"]
    assert s.n_atoms == 375 and g.nb == 15000 and g.n_points == 375 * 80 * 434
    assert g.info.n_batches == -(-g.n_points // 200)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split"])
def test_slab_sampled(slab, prec):
    g = slab["g"]
    t0 = time.perf_counter()
    H = g.integrate_h(cuda(slab["v"]), prec=prec)
    Pd = cuda(slab["P"])
    n, ne = g.update_density(Pd, prec=prec)
    torch.cuda.synchronize()
    g.sync()
    dt = time.perf_counter() - t0
    F = SAMPLE_F
    Hs = H[F][:, F].cpu().numpy()
    e_H = rel_err(Hs, slab["Hb"], slab["Ab"])
    e_n = rel_err(n.cpu().numpy()[slab["pidx"]], slab["n_s"], slab["D_s"])
    assert torch.equal(H, H.t())
    del H
    S = g.overlap(prec=prec)
    trPS = float(torch.sum(Pd * S).item())
    del S
    print(f"slab {prec}: e_H(sampled)={e_H:.2e} e_n(sampled)={e_n:.2e} N_e={float(ne.item()):.6f} tr(PS)={trPS:.6f} "
          f"({dt:.1f} s for H + n)")
    assert e_H <= TOL[prec] and e_n <= TOL[prec]
    assert abs(float(ne.item()) - trPS) <= 10 * TOL[prec] * abs(trPS)
