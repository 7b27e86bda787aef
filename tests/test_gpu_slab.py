"""The precision configuration at full size, which is also the workload bench.py times by
default: a 375-atom two-species slab (15,000 basis functions, 80 x 434 points per atom =
13,020,000 points, batches <= 200). Checked per precision, and on the split path at the
library's default slice count and at the count bench.py times: every element of H over a
block of 360 basis functions (nine whole atoms: both species, every l, in-layer and
between-layer neighbours and atoms far apart, so the block holds diagonal, neighbour and
exactly-zero pairs) over all points, and n at 50,000 sampled points, against the oracle
(tests/_oracle_par.py spreads it over the host's cores; tolerances of tests/_metrics.py: FP64
1e-12, FP32 1e-6, split 1e-10), plus tr(PS) = N_e. P is X X^T / 64 with X 15000 x 64 (low rank
keeps the host generation short).
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench
from paper_1912_06636_gb300 import nao, synth
from tests import _oracle_par
from tests._metrics import raw_rel_err, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = {"fp64": 1e-12, "fp32": 1e-6, "split": 1e-10}
SPLIT_CASES = sorted({12, bench.BENCH_SLICES[2]})
# e4m3 digits (base 32) at the slice count bench.py uses with them
E4M3_CASES = [bench.BENCH_SLICES_E4M3[2]]
# atoms of the block: 0 (B) with its in-layer neighbour 1 (B, 7.8 bohr) and 5, the layer above
# (25, 26: A, 5.7 bohr), a pair in the middle of the slab (187, 188) with the atom above one of
# them (212), and the far corner (374); 40 functions each (4s3p4d1f)
BLOCK_ATOMS = [0, 1, 5, 25, 26, 187, 188, 212, 374]
SAMPLE_F = np.concatenate([np.arange(40 * a, 40 * a + 40) for a in BLOCK_ATOMS])


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def slab():
    t0 = time.perf_counter()
    s = synth.config(2)
    v = s.potential()
    P = synth.density_matrix(s, 2, rank=64)
    t1 = time.perf_counter()
    Hb, Ab = _oracle_par.hamiltonian_block(s, SAMPLE_F, s.pt_xyz, s.pt_w, v)
    rng = np.random.Generator(np.random.PCG64(22))
    pidx = np.sort(rng.choice(s.n_points, 50000, replace=False))
    n_s, D_s = _oracle_par.density(s, s.pt_xyz[pidx], P)
    t2 = time.perf_counter()
    print(f"slab: {s.n_atoms} atoms, {s.n_basis} basis functions, {s.n_points} points; "
          f"inputs {t1 - t0:.0f} s, oracle block and samples {t2 - t1:.0f} s on {_oracle_par.workers()} threads")
    g = nao.Grid(s, device=0, max_batch_points=200)
    yield dict(s=s, v=v, P=P, Hb=Hb, Ab=Ab, pidx=pidx, n_s=n_s, D_s=D_s, g=g)
    g.close()


def test_slab_sizes(slab):
    g, s = slab["g"], slab["s"]
    assert s.n_atoms == 375 and g.nb == 15000 and g.n_points == 375 * 80 * 434
    assert g.info.n_batches == -(-g.n_points // 200)
    # the block holds pairs that overlap and pairs that never do
    assert np.count_nonzero(slab["Ab"]) > 0 and np.count_nonzero(slab["Ab"] == 0) > 0


@pytest.mark.parametrize("case", ["fp64", "fp32"] + [f"split{S}" for S in SPLIT_CASES]
                         + [f"e4m3_{S}" for S in E4M3_CASES])
def test_slab_block_and_samples(slab, case):
    g = slab["g"]
    prec = "split" if case.startswith(("split", "e4m3")) else case
    own = None
    if case.startswith("split"):
        own = g = nao.Grid(slab["s"], device=0, max_batch_points=200, split_slices=int(case[5:]))
    elif case.startswith("e4m3"):
        own = g = nao.Grid(slab["s"], device=0, max_batch_points=200, split_slices=int(case[5:]), split_digits=1)
    t0 = time.perf_counter()
    H = g.integrate_h(cuda(slab["v"]), prec=prec)
    Pd = cuda(slab["P"])
    n, ne = g.update_density(Pd, prec=prec)
    torch.cuda.synchronize()
    g.sync()
    dt = time.perf_counter() - t0
    F = torch.from_numpy(SAMPLE_F).cuda()
    Hs = H[F][:, F].cpu().numpy()
    e_H = rel_err(Hs, slab["Hb"], slab["Ab"])
    assert np.all(Hs[slab["Ab"] == 0] == 0.0)
    nc = n.cpu().numpy()[slab["pidx"]]
    e_n = rel_err(nc, slab["n_s"], slab["D_s"])
    assert torch.equal(H, H.t())
    del H
    S = g.overlap(prec=prec)
    trPS = float(torch.sum(Pd * S).item())
    del S
    if own is not None:
        own.close()
    print(f"slab {case}: e_H={e_H:.2e} (raw {raw_rel_err(Hs, slab['Hb'], slab['Ab']):.2e}) over {Hs.size} elements, "
          f"e_n={e_n:.2e} (raw {raw_rel_err(nc, slab['n_s'], slab['D_s']):.2e}) over {nc.size} points, "
          f"N_e={float(ne.item()):.6f} tr(PS)={trPS:.6f} ({dt:.1f} s for H + n)")
    assert e_H <= TOL[prec] and e_n <= TOL[prec]
    assert abs(float(ne.item()) - trPS) <= 10 * TOL[prec] * abs(trPS)
