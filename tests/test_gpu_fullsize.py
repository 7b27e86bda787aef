"""Full-size parity on the 64-atom diamond-lattice cluster (1600 basis functions, 1,175,040
points, batches <= 300 points), in the launch configuration bench.py times for it: partition
and reduced bases bit-exact; every element of H and n at every point against the oracle
(tests/_oracle_par.py spreads it over the host's cores), at every precision and at the split
slice counts the library defaults to and bench.py times; plus properties that hold at any size
(symmetry, exact zeros, tr(PS) = sum_p w_p n_p)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench
import oracle
from paper_1912_06636_gb300 import nao, synth
from tests import _oracle_par
from tests._metrics import raw_rel_err, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-6, "split": 1e-10}
# the split path at the library's default slice count and at the count bench.py times here
SPLIT_CASES = sorted({12, bench.BENCH_SLICES[1]})
# e4m3 digits (base 32) at the slice count bench.py uses with them
E4M3_CASES = [bench.BENCH_SLICES_E4M3[1]]


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def diamond():
    s = synth.config(1)
    v = s.potential()
    P = synth.density_matrix(s, 1)
    H_ref, A = _oracle_par.hamiltonian(s, s.pt_xyz, s.pt_w, v)
    n_ref, D = _oracle_par.density(s, s.pt_xyz, P)
    g = nao.Grid(s, device=0, max_batch_points=s.max_batch_points)
    yield dict(s=s, v=v, P=P, H=H_ref, A=A, n=n_ref, D=D, g=g)
    g.close()


def test_partition_and_relevance_bit_exact_fullsize(diamond):
    s, g = diamond["s"], diamond["g"]
    o = oracle.Oracle(s)
    bo, pp, ro, ri = g.batches()
    obo, opp = oracle.Oracle.partition(s.pt_xyz, s.max_batch_points)
    assert np.array_equal(bo, obo) and np.array_equal(pp, opp)
    oro, ori = o.relevance(s.pt_xyz, obo, opp)
    assert np.array_equal(ro, oro) and np.array_equal(ri, ori)


@pytest.mark.parametrize("case", ["fp64", "fp32"] + [f"split{S}" for S in SPLIT_CASES]
                         + [f"e4m3_{S}" for S in E4M3_CASES])
def test_fullsize_every_element(diamond, case):
    g, s = diamond["g"], diamond["s"]
    prec = "split" if case.startswith(("split", "e4m3")) else case
    own = None
    if case.startswith("split"):
        own = g = nao.Grid(s, device=0, max_batch_points=s.max_batch_points, split_slices=int(case[5:]))
    elif case.startswith("e4m3"):
        own = g = nao.Grid(s, device=0, max_batch_points=s.max_batch_points, split_slices=int(case[5:]), split_digits=1)
    H = g.integrate_h(cuda(diamond["v"]), prec=prec)
    n, ne = g.update_density(cuda(diamond["P"]), prec=prec)
    S = g.overlap(prec=prec)
    torch.cuda.synchronize()
    g.sync()
    if own is not None:
        own.close()
    Hc = H.cpu().numpy()
    assert np.array_equal(Hc, Hc.T)
    e_H = rel_err(Hc, diamond["H"], diamond["A"])
    assert np.all(Hc[diamond["A"] == 0] == 0.0)  # no pair of functions that never overlap picks up a value
    nc = n.cpu().numpy()
    e_n = rel_err(nc, diamond["n"], diamond["D"])
    # tr(PS) = sum_p w_p n_p holds for the GPU's own S and n (same discrete sum)
    trPS = float(torch.sum(cuda(diamond["P"]) * S).item())
    print(f"{case}: e_H={e_H:.2e} (raw {raw_rel_err(Hc, diamond['H'], diamond['A']):.2e}) over all "
          f"{Hc.size} elements, e_n={e_n:.2e} over all {nc.size} points, N_e={float(ne.item()):.10f} tr(PS)={trPS:.10f}")
    assert e_H <= TOL[prec] and e_n <= TOL[prec]
    assert abs(float(ne.item()) - trPS) <= 10 * TOL[prec] * abs(trPS)
