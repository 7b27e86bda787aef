"""Full-size parity on the benchmark workload (64-atom diamond-lattice cluster, 1600 basis
functions, 1,175,040 points, batches <= 300 points) in the launch configuration bench.py
times: partition and reduced bases bit-exact; H on a sampled block of basis functions and n
on sampled points against the oracle, which computes them one by one; plus properties that
hold at any size (symmetry, exact zeros, tr(PS) = sum_p w_p n_p)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-6, "split": 1e-10}
# the split path with the library's default slices, and with the 10 slices bench.py times
SPLIT_SLICES = {"split": None, "split10": 10}
# sampled basis functions: several atoms (neighbours and far-apart pairs), every l
SAMPLE_F = np.array([0, 3, 9, 18, 24, 25 * 1 + 2, 25 * 5 + 13, 25 * 8 + 21, 25 * 27 + 6, 25 * 40 + 11,
                     25 * 58 + 19, 25 * 63 + 24])


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def diamond():
    s = synth.config(1)
    v = s.potential()
    P = synth.density_matrix(s, 1)
    o = oracle.Oracle(s)
    Hb, Ab = o.hamiltonian_block(SAMPLE_F, s.pt_xyz, s.pt_w, v)
    rng = np.random.Generator(np.random.PCG64(77))
    pidx = np.sort(rng.choice(s.n_points, 3000, replace=False))
    n_s, D_s, _ = o.density(s.pt_xyz[pidx], P)
    g = nao.Grid(s, device=0, max_batch_points=s.max_batch_points)
    yield dict(s=s, v=v, P=P, o=o, Hb=Hb, Ab=Ab, pidx=pidx, n_s=n_s, D_s=D_s, g=g)
    g.close()


def test_partition_and_relevance_bit_exact_fullsize(diamond):
    s, o, g = diamond["s"], diamond["o"], diamond["g"]
    bo, pp, ro, ri = g.batches()
    obo, opp = oracle.Oracle.partition(s.pt_xyz, s.max_batch_points)
    assert np.array_equal(bo, obo) and np.array_equal(pp, opp)
    oro, ori = o.relevance(s.pt_xyz, obo, opp)
    assert np.array_equal(ro, oro) and np.array_equal(ri, ori)


@pytest.mark.parametrize("case", ["fp64", "fp32", "split", "split10"])
def test_fullsize_sampled(diamond, case):
    g, s = diamond["g"], diamond["s"]
    prec = "split" if case.startswith("split") else case
    own = None
    if SPLIT_SLICES.get(case) is not None:
        own = g = nao.Grid(s, device=0, max_batch_points=s.max_batch_points, split_slices=SPLIT_SLICES[case])
    H = g.integrate_h(cuda(diamond["v"]), prec=prec)
    n, ne = g.update_density(cuda(diamond["P"]), prec=prec)
    S = g.overlap(prec=prec)
    torch.cuda.synchronize()
    g.sync()
    if own is not None:
        own.close()
    Hc = H.cpu().numpy()
    assert np.array_equal(Hc, Hc.T)
    F = SAMPLE_F
    e_H = rel_err(Hc[np.ix_(F, F)], diamond["Hb"], diamond["Ab"])
    zero = diamond["Ab"] == 0
    assert np.all(Hc[np.ix_(F, F)][zero] == 0.0)
    nc = n.cpu().numpy()
    e_n = rel_err(nc[diamond["pidx"]], diamond["n_s"], diamond["D_s"])
    # tr(PS) = sum_p w_p n_p holds for the GPU's own S and n (same discrete sum)
    trPS = float(torch.sum(cuda(diamond["P"]) * S).item())
    print(f"{case}: e_H(sampled)={e_H:.2e} e_n(sampled)={e_n:.2e} N_e={float(ne.item()):.10f} tr(PS)={trPS:.10f}")
    assert e_H <= TOL[prec] and e_n <= TOL[prec]
    assert abs(float(ne.item()) - trPS) <= 10 * TOL[prec] * abs(trPS)
