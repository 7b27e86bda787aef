"""Grouped handles: one handle over several molecules, one launch per kernel for all of them.

Each system's H, n and N_e from the grouped calls must meet the same bars against the
oracle as a handle of its own (FP64 1e-12, FP32 1e-6, split 1e-10; tests/_metrics.py), and
the FP64 results must agree with those of the single-system handles to rounding order
(both run the same per-batch kernels; only the order of the FP64 atomic additions into H
differs). Also: the graph-replay option gives the same results as plain launches with new
buffers on every call, and the single-system calls refuse a grouped handle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-6, "split": 1e-10}


def _systems():
    a = synth.config_water()
    # the same species in another geometry and a coarser grid
    heavy = synth.Species(ls=[0, 0, 1, 2], alphas=[10.0, 1.5, 0.4, 0.6], Z=8.0)
    light = synth.Species(ls=[0, 0, 1], alphas=[1.2, 0.3, 0.8], Z=1.0)
    b = synth.make_system([[0.3, -0.2, 0.1], [0.3, 1.5, 1.0], [1.9, -0.9, 0.1], [-1.1, -0.9, 0.4]], [0, 1, 1, 1],
                          [heavy, light], n_rad=30, n_theta=8, n_phi=9, name="ammonia4")
    # 8-atom diamond cell: 200 basis functions with l up to 3
    c = synth.config_diamond64(n_rad=20, n_theta=8, n_phi=9, cells=1)
    return [a, b, c]


@pytest.fixture(scope="module")
def group():
    systems = _systems()
    refs = []
    for k, s in enumerate(systems):
        o = oracle.Oracle(s)
        v = s.potential()
        P = synth.density_matrix(s, 10 + k)
        H, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
        n, D, ne = o.density(s.pt_xyz, P, s.pt_w)
        refs.append(dict(v=v, P=P, H=H, A=A, n=n, D=D, ne=ne))
    g = nao.Grid(systems, device=0, max_batch_points=200)
    yield dict(systems=systems, refs=refs, g=g)
    g.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_group_layout(group):
    g, systems = group["g"], group["systems"]
    assert g.n_systems == 3
    assert g.nb == sum(s.n_basis for s in systems)
    assert g.n_points == sum(len(s.pt_w) for s in systems)
    bo, pp, ro, ri = g.batches()
    b_prev, p_prev, nb_prev = 0, 0, 0
    for m, s in enumerate(systems):
        info = g.systems[m]
        assert info["n_basis"] == s.n_basis and info["n_points"] == len(s.pt_w)
        assert info["basis_offset"] == nb_prev and info["point_offset"] == p_prev
        assert info["batch_begin"] == b_prev
        b0, b1 = info["batch_begin"], info["batch_end"]
        # the system's own partition, shifted into the global numbering
        obo, opp = oracle.Oracle.partition(s.pt_xyz, 200)
        assert np.array_equal(bo[b0:b1 + 1] - p_prev, obo)
        assert np.array_equal(pp[p_prev:p_prev + len(s.pt_w)] - p_prev, opp)
        # reduced bases only hold the system's own functions
        rel = ri[ro[b0]:ro[b1]]
        assert rel.size == 0 or (rel.min() >= nb_prev and rel.max() < nb_prev + s.n_basis)
        b_prev, p_prev, nb_prev = b1, p_prev + len(s.pt_w), nb_prev + s.n_basis
    assert b_prev == len(bo) - 1


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split"])
def test_group_hamiltonian_and_density(group, prec):
    g, refs = group["g"], group["refs"]
    Hs = g.integrate_h_many([cuda(r["v"]) for r in refs], prec=prec)
    ns, nes = g.update_density_many([cuda(r["P"]) for r in refs], prec=prec)
    torch.cuda.synchronize()
    g.sync()
    for m, r in enumerate(refs):
        H = Hs[m].cpu().numpy()
        assert np.array_equal(H, H.T)
        assert rel_err(H, r["H"], r["A"]) <= TOL[prec], (m, prec)
        assert rel_err(ns[m].cpu().numpy(), r["n"], r["D"]) <= TOL[prec], (m, prec)
        assert abs(nes[m].item() - r["ne"]) <= TOL[prec] * max(abs(r["ne"]), 1.0), (m, prec)


def test_group_matches_single_handles(group):
    g, systems, refs = group["g"], group["systems"], group["refs"]
    Hs = g.integrate_h_many([cuda(r["v"]) for r in refs], prec="fp64")
    ns, nes = g.update_density_many([cuda(r["P"]) for r in refs], prec="fp64")
    for m, s in enumerate(systems):
        with nao.Grid(s, device=0, max_batch_points=200) as one:
            H1 = one.integrate_h(cuda(refs[m]["v"]), prec="fp64")
            n1, ne1 = one.update_density(cuda(refs[m]["P"]), prec="fp64")
            torch.cuda.synchronize()
            one.sync()
            assert rel_err(Hs[m].cpu().numpy(), H1.cpu().numpy(), refs[m]["A"]) <= 1e-14
            # density: no atomics, same per-tile order -> identical
            assert torch.equal(ns[m], n1)
            assert nes[m].item() == ne1.item()


def test_group_optional_entries(group):
    """v = 1 (NULL entries) gives the overlap matrix; N_e only where asked for."""
    g, systems, refs = group["g"], group["systems"], group["refs"]
    Ss = g.integrate_h_many([None, cuda(refs[1]["v"]), None], terms=nao.NAO_TERM_POTENTIAL, prec="fp64")
    nes = [torch.full((1,), -7.0, dtype=torch.float64, device="cuda") for _ in systems]
    ns, _ = g.update_density_many([cuda(r["P"]) for r in refs], prec="fp64", nes=[nes[0], None, nes[2]])
    torch.cuda.synchronize()
    g.sync()
    for m in (0, 2):
        o = oracle.Oracle(systems[m])
        S, SA = o.overlap(systems[m].pt_xyz, systems[m].pt_w)
        assert rel_err(Ss[m].cpu().numpy(), S, SA) <= 1e-12
        assert abs(nes[m].item() - refs[m]["ne"]) <= 1e-12 * abs(refs[m]["ne"])
    # potential-only term of system 1 with its v: compare with v . phi phi from the oracle
    o = oracle.Oracle(systems[1])
    Hp, Ap = o.hamiltonian(systems[1].pt_xyz, systems[1].pt_w, refs[1]["v"], terms=1)
    assert rel_err(Ss[1].cpu().numpy(), Hp, Ap) <= 1e-12
    assert nes[1].item() == -7.0


def test_single_calls_refuse_grouped_handle(group):
    g = group["g"]
    H = torch.empty((g.nb, g.nb), dtype=torch.float64, device="cuda")
    with pytest.raises(nao.NaoError) as e:
        nao.nao_integrate_h(g.h, None, 3, "fp64", H)
    assert e.value.code == nao.NAO_ERR_INVALID_ARG
    with pytest.raises(nao.NaoError):
        nao.nao_integrate_h_noalloc(g.h, None, 3, H)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_graph_replay_matches_plain_launches(prec):
    systems = _systems()[:2]
    refs = []
    for k, s in enumerate(systems):
        refs.append([(cuda(s.potential() * (1.0 + 0.25 * t)), cuda(synth.density_matrix(s, 20 + 3 * k + t)))
                     for t in range(3)])
    plain = nao.Grid(systems, device=0)
    graph = nao.Grid(systems, device=0, capture_graph=1)
    try:
        for t in range(3):  # new input and output buffers on every call
            vs = [refs[m][t][0] for m in range(2)]
            Ps = [refs[m][t][1] for m in range(2)]
            H0 = plain.integrate_h_many(vs, prec=prec)
            H1 = graph.integrate_h_many(vs, prec=prec)
            n0, ne0 = plain.update_density_many(Ps, prec=prec)
            n1, ne1 = graph.update_density_many(Ps, prec=prec)
            torch.cuda.synchronize()
            plain.sync()
            graph.sync()
            for m in range(2):
                scale = H0[m].abs().max().item()
                assert (H0[m] - H1[m]).abs().max().item() <= 1e-14 * scale
                if prec == "fp64":  # one tile writes each point: identical
                    assert torch.equal(n0[m], n1[m])
                    assert ne0[m].item() == ne1[m].item()
                else:  # split: per-point atomic additions over column tiles
                    nscale = n0[m].abs().max().item()
                    assert (n0[m] - n1[m]).abs().max().item() <= 1e-14 * nscale
                    assert abs(ne0[m].item() - ne1[m].item()) <= 1e-13 * abs(ne0[m].item())
    finally:
        plain.close()
        graph.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split"])
def test_every_output_element_is_written(group, prec):
    """H (both triangles) and n at every point, also points of batches without basis
    functions, are written by each call: outputs pre-filled with NaN come back finite."""
    g, refs = group["g"], group["refs"]
    Hs = [torch.full((s["n_basis"], s["n_basis"]), float("nan"), dtype=torch.float64, device="cuda") for s in g.systems]
    ns = [torch.full((s["n_points"],), float("nan"), dtype=torch.float64, device="cuda") for s in g.systems]
    nes = [torch.full((1,), float("nan"), dtype=torch.float64, device="cuda") for _ in g.systems]
    g.integrate_h_many([cuda(r["v"]) for r in refs], prec=prec, Hs=Hs)
    g.update_density_many([cuda(r["P"]) for r in refs], prec=prec, ns=ns, nes=nes)
    torch.cuda.synchronize()
    g.sync()
    bo, _, ro, _ = g.batches()
    assert np.any(np.diff(ro) == 0)  # there are batches without functions
    for m in range(len(refs)):
        assert torch.isfinite(Hs[m]).all() and torch.isfinite(ns[m]).all() and torch.isfinite(nes[m]).all()
