"""Many independent molecules in one grouped handle (the batching configuration: molecules of
a few to a few dozen atoms, each with its own batch size, all batches in one launch per
kernel): every molecule's H, n and N_e against the oracle at each precision's bar (FP64 1e-12,
FP32 1e-6, split 1e-10; tests/_metrics.py).

Sizes are reduced so that the oracle finishes in seconds: 32 molecules of 3-16 atoms on a
16 x 42 points-per-atom grid, batch sizes log-uniform in [20, 400] as the batching
configuration states (the split path accumulates batches above 336 points in K segments).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-6, "split": 1e-10}


@pytest.fixture(scope="module")
def mols():
    systems, bs = synth.molecule_set(32, seed=3000, n_min=3, n_max=16, b_min=20, b_max=400,
                                     n_rad=16, n_theta=6, n_phi=7)
    refs = []
    for k, s in enumerate(systems):
        o = oracle.Oracle(s)
        v = s.potential()
        P = synth.density_matrix(s, 3000 + k)
        H, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
        n, D, ne = o.density(s.pt_xyz, P, s.pt_w)
        refs.append(dict(v=v, P=P, H=H, A=A, n=n, D=D, ne=ne))
    g = nao.Grid(systems, device=0, batch_points=bs)
    yield dict(systems=systems, bs=bs, refs=refs, g=g)
    g.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_partitions_follow_each_batch_size(mols):
    g, systems, bs = mols["g"], mols["systems"], mols["bs"]
    bo, pp, ro, ri = g.batches()
    assert len(set(bs)) > 8
    for m, (s, B) in enumerate(zip(systems, bs)):
        info = g.systems[m]
        b0, b1 = info["batch_begin"], info["batch_end"]
        obo, opp = oracle.Oracle.partition(s.pt_xyz, B)
        assert np.array_equal(bo[b0:b1 + 1] - info["point_offset"], obo)
        assert np.array_equal(pp[info["point_offset"]:info["point_offset"] + info["n_points"]] - info["point_offset"], opp)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split"])
def test_every_molecule_matches_oracle(mols, prec):
    g, refs = mols["g"], mols["refs"]
    Hs = g.integrate_h_many([cuda(r["v"]) for r in refs], prec=prec)
    ns, nes = g.update_density_many([cuda(r["P"]) for r in refs], prec=prec)
    torch.cuda.synchronize()
    g.sync()
    worst_h = worst_n = 0.0
    for m, r in enumerate(refs):
        H = Hs[m].cpu().numpy()
        assert np.array_equal(H, H.T)
        eh = rel_err(H, r["H"], r["A"])
        en = rel_err(ns[m].cpu().numpy(), r["n"], r["D"])
        worst_h, worst_n = max(worst_h, eh), max(worst_n, en)
        assert eh <= TOL[prec] and en <= TOL[prec], (m, eh, en)
        assert abs(nes[m].item() - r["ne"]) <= TOL[prec] * max(abs(r["ne"]), 1.0)
    print(f"{prec}: worst e_H {worst_h:.2e}, worst e_n {worst_n:.2e} over {len(refs)} molecules")


def test_twelve_slices_have_one_tile_width(mols):
    """12 slices need 12 x TN tensor-memory columns, so only the 32-wide tile exists."""
    g, refs = mols["g"], mols["refs"]
    g.integrate_h_many([cuda(r["v"]) for r in refs], prec="split")
    tw, timed = nao.nao_get_tuning(g.h)
    _, _, ro, _ = g.batches()
    N = np.diff(ro)
    assert timed == 0 and np.all(tw[N > 0] == 32)


def test_ten_slice_autotuner(mols):
    """With 10 slices both widths exist: the autotuner times them per histogram bucket; the
    tuned run and the fixed rule give the same H up to the order of the FP64 additions (every
    element's slice sums are exact integers whatever the tile) and the same n up to the rounding
    of each T element to a 64-bit integer in units of 2^(e_q + e_b - 50), whose grouping into
    tiles follows the width (at most 1e-13 of the magnitude sums D; the bar against the oracle is
    1e-10)."""
    systems, bs, refs = mols["systems"], mols["bs"], mols["refs"]
    sel = list(range(len(systems)))
    kw = dict(device=0, batch_points=[bs[k] for k in sel], split_slices=10)
    out = {}
    for auto in (1, 0):
        with nao.Grid([systems[k] for k in sel], autotune=auto, **kw) as g:
            Hs = g.integrate_h_many([cuda(refs[k]["v"]) for k in sel], prec="split")
            ns, _ = g.update_density_many([cuda(refs[k]["P"]) for k in sel], prec="split")
            torch.cuda.synchronize()
            g.sync()
            tw, timed = nao.nao_get_tuning(g.h)
            _, _, ro, _ = g.batches()
            out[auto] = ([h.cpu().numpy() for h in Hs], [n.cpu().numpy() for n in ns], tw, timed, np.diff(ro))
    Hs1, ns1, tw1, timed1, N = out[1]
    Hs0, ns0, tw0, timed0, _ = out[0]
    assert timed1 >= 1 and timed0 == 0
    assert set(np.unique(tw1[N > 0])) <= {32, 48}
    assert np.all(tw0[N > 0] == 48)
    print("autotuner:", timed1, "buckets timed;", int(np.sum(tw1[N > 0] == 48)), "batches at 48,",
          int(np.sum(tw1[N > 0] == 32)), "at 32")
    for m, k in enumerate(sel):
        assert rel_err(Hs1[m], Hs0[m], refs[k]["A"]) <= 1e-14
        assert rel_err(ns1[m], ns0[m], refs[k]["D"]) <= 1e-13


def test_graphs_recorded_before_tuning_are_replaced(mols):
    """A density graph recorded before the first split Hamiltonian call (which tunes and
    rebuilds the work lists) must not be replayed with the old lists."""
    systems, bs, refs = mols["systems"], mols["bs"], mols["refs"]
    sel = list(range(8))
    with nao.Grid([systems[k] for k in sel], device=0, batch_points=[bs[k] for k in sel], split_slices=10,
                  capture_graph=1) as g:
        Ps = [cuda(refs[k]["P"]) for k in sel]
        n1, _ = g.update_density_many(Ps, prec="split")
        g.integrate_h_many([cuda(refs[k]["v"]) for k in sel], prec="split")
        n2, ne2 = g.update_density_many(Ps, prec="split")
        torch.cuda.synchronize()
        g.sync()
        for i, k in enumerate(sel):
            r = refs[k]
            assert rel_err(n1[i].cpu().numpy(), r["n"], r["D"]) <= 1e-10
            assert rel_err(n2[i].cpu().numpy(), r["n"], r["D"]) <= 1e-10
            assert abs(ne2[i].item() - r["ne"]) <= 1e-10 * abs(r["ne"])


def test_every_molecule_matches_oracle_e4m3(mols):
    """The setting bench.py times the batching configuration with: 14 e4m3 slices (base-32
    digits, kind::f8f6f4), in a grouped handle of its own."""
    systems, bs, refs = mols["systems"], mols["bs"], mols["refs"]
    with nao.Grid(systems, device=0, batch_points=bs, split_slices=14, split_digits=1, capture_graph=1) as g:
        Hs = g.integrate_h_many([cuda(r["v"]) for r in refs], prec="split")
        ns, nes = g.update_density_many([cuda(r["P"]) for r in refs], prec="split")
        torch.cuda.synchronize()
        g.sync()
        worst = 0.0
        for m, r in enumerate(refs):
            eh = rel_err(Hs[m].cpu().numpy(), r["H"], r["A"])
            en = rel_err(ns[m].cpu().numpy(), r["n"], r["D"])
            worst = max(worst, eh, en)
            assert eh <= TOL["split"] and en <= TOL["split"], (m, eh, en)
    print(f"e4m3: worst error {worst:.2e} over {len(refs)} molecules")
