"""GPU parity of the FP64 path against the FP64 oracle (3-atom molecule and small edge cases).

Bars: batch partition and reduced bases bit-exact; phi/grad phi within 1e-13 of the
per-function magnitude in the batch; e_H, e_n <= 1e-12 (see tests/_metrics.py); N_e within
1e-12 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def water():
    s = synth.config_water()
    o = oracle.Oracle(s)
    v = s.potential()
    P = synth.density_matrix(s, 0)
    S, _ = o.overlap(s.pt_xyz, s.pt_w)
    P *= 10.0 / np.trace(P @ S)
    H, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    n, D, ne = o.density(s.pt_xyz, P, s.pt_w)
    g = nao.Grid(s, device=0, max_batch_points=200)
    yield dict(s=s, o=o, v=v, P=P, H=H, A=A, n=n, D=D, ne=ne, g=g)
    g.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_partition_and_relevance_bit_exact(water):
    s, o, g = water["s"], water["o"], water["g"]
    bo, pp, ro, ri = g.batches()
    obo, opp = oracle.Oracle.partition(s.pt_xyz, 200)
    assert np.array_equal(bo, obo) and np.array_equal(pp, opp)
    oro, ori = o.relevance(s.pt_xyz, obo, opp)
    assert np.array_equal(ro, oro) and np.array_equal(ri, ori)
    assert len(bo) == 67


def test_basis_functions_match_oracle(water):
    s, o, g = water["s"], water["o"], water["g"]
    bo, pp, ro, ri = g.batches()
    nonempty = np.nonzero(np.diff(ro))[0]
    empty = np.nonzero(np.diff(ro) == 0)[0]
    assert len(nonempty) > 4 and len(empty) > 0
    phi, grad = g.evaluate_batch(int(empty[0]))
    assert phi.numel() == 0
    for b in [int(nonempty[0]), int(nonempty[len(nonempty) // 2]), int(nonempty[-1])]:
        phi, grad = g.evaluate_batch(b)
        pts = s.pt_xyz[pp[bo[b]:bo[b + 1]]]
        rphi, rgrad = o.eval_dense(pts)
        rel = ri[ro[b]:ro[b + 1]]
        rphi = rphi[:, rel].T  # [N, P]
        rgrad = np.transpose(rgrad[:, rel, :], (2, 1, 0))  # [3, N, P]
        phi, grad = phi.cpu().numpy(), grad.cpu().numpy()
        scale = np.maximum(np.abs(rphi).max(axis=1, keepdims=True), 1e-300)
        assert np.all(np.abs(phi - rphi) <= 1e-13 * scale)
        gscale = np.maximum(np.abs(rgrad).max(axis=(0, 2), keepdims=True), 1e-300)
        assert np.all(np.abs(grad - rgrad) <= 1e-13 * gscale)


def test_hamiltonian_fp64(water):
    g = water["g"]
    H = g.integrate_h(cuda(water["v"]), prec="fp64")
    torch.cuda.synchronize()
    g.sync()
    H = H.cpu().numpy()
    assert np.array_equal(H, H.T)
    assert rel_err(H, water["H"], water["A"]) <= TOL


def test_overlap_and_kinetic_terms(water):
    s, o, g = water["s"], water["o"], water["g"]
    S_ref, SA = o.overlap(s.pt_xyz, s.pt_w)
    T_ref, TA = o.hamiltonian(s.pt_xyz, s.pt_w, None, oracle.TERM_KINETIC)
    S = g.overlap().cpu().numpy()
    T = g.integrate_h(None, nao.NAO_TERM_KINETIC).cpu().numpy()
    assert rel_err(S, S_ref, SA) <= TOL
    assert rel_err(T, T_ref, TA) <= TOL


def test_density_fp64(water):
    g = water["g"]
    n, ne = g.update_density(cuda(water["P"]), prec="fp64")
    torch.cuda.synchronize()
    assert rel_err(n.cpu().numpy(), water["n"], water["D"]) <= TOL
    assert abs(float(ne.item()) - water["ne"]) <= TOL * abs(water["ne"])
    assert abs(float(ne.item()) - 10.0) < 1e-10


def test_host_entry_points(water):
    g = water["g"]
    H = np.zeros((g.nb, g.nb))
    nao.nao_integrate_h_host(g.h, water["v"], 3, "fp64", H)
    assert rel_err(H, water["H"], water["A"]) <= TOL
    n = np.zeros(g.n_points)
    ne = nao.nao_update_density_host(g.h, water["P"], "fp64", n)
    assert rel_err(n, water["n"], water["D"]) <= TOL
    assert abs(ne - water["ne"]) <= TOL * abs(water["ne"])


@pytest.mark.parametrize("B", [1, 37, 64, 1024])
def test_result_independent_of_batch_size(water, B):
    """Eq. H_decomp: h is the sum of the batch contributions, whatever the batches."""
    s = water["s"]
    with nao.Grid(s, device=0, max_batch_points=B) as g:
        H = g.integrate_h(cuda(water["v"])).cpu().numpy()
        n, ne = g.update_density(cuda(water["P"]))
        assert rel_err(H, water["H"], water["A"]) <= TOL
        assert rel_err(n.cpu().numpy(), water["n"], water["D"]) <= TOL


def test_small_scratch_forces_many_chunks(water):
    s = water["s"]
    with nao.Grid(s, device=0, max_batch_points=200, scratch_bytes=1) as g:
        H = g.integrate_h(cuda(water["v"])).cpu().numpy()
        n, _ = g.update_density(cuda(water["P"]))
        assert rel_err(H, water["H"], water["A"]) <= TOL
        assert rel_err(n.cpu().numpy(), water["n"], water["D"]) <= TOL


def test_edge_cases_single_point_far_points_and_high_l():
    sp = synth.Species([0, 3, 6], [1.5, 0.9, 0.7], rc=4.0)
    atoms = [[0.1, -0.2, 0.3], [2.0, 1.0, -0.5]]
    s = synth.make_system(atoms, [0, 0], [sp], 6, 3, 4)
    rng = np.random.Generator(np.random.PCG64(9))
    # keep the generated grid, add far-away points (empty batches) and a ragged total
    far = rng.uniform(30.0, 40.0, (45, 3))
    s.pt_xyz = np.ascontiguousarray(np.concatenate([s.pt_xyz, far]))
    s.pt_w = np.ascontiguousarray(np.concatenate([s.pt_w, rng.uniform(0.1, 1.0, 45)]))
    o = oracle.Oracle(s)
    v = s.potential()
    P = synth.density_matrix(s, 1)
    Href, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    nref, D, ne = o.density(s.pt_xyz, P, s.pt_w)
    with nao.Grid(s, device=0, max_batch_points=17) as g:
        _, _, ro, _ = g.batches()
        assert np.any(np.diff(ro) == 0)
        H = g.integrate_h(cuda(v)).cpu().numpy()
        n, nev = g.update_density(cuda(P))
        n = n.cpu().numpy()
        assert rel_err(H, Href, A) <= TOL
        assert rel_err(n, nref, D) <= TOL
        assert np.all(n[-45:] == 0.0)
    one = synth.System(**{**s.__dict__})
    one.pt_xyz = np.ascontiguousarray(s.pt_xyz[5:6])
    one.pt_w = np.ascontiguousarray(s.pt_w[5:6])
    Href1, A1 = oracle.Oracle(one).hamiltonian(one.pt_xyz, one.pt_w, v[5:6])
    with nao.Grid(one, device=0) as g:
        H1 = g.integrate_h(cuda(v[5:6])).cpu().numpy()
        assert rel_err(H1, Href1, A1) <= TOL


def test_point_on_nucleus_is_rejected():
    s = synth.config_water(n_rad=4, n_theta=2, n_phi=3)
    s.pt_xyz = np.ascontiguousarray(np.concatenate([s.pt_xyz, s.atom_xyz[1:2]]))
    s.pt_w = np.ascontiguousarray(np.concatenate([s.pt_w, [1.0]]))
    with pytest.raises(nao.NaoError) as e:
        nao.Grid(s, device=0)
    assert e.value.code == 1


def test_profile_counts_launches(water):
    g = water["g"]
    nao.nao_profile_enable(g.h, True)
    g.integrate_h(cuda(water["v"]))
    g.update_density(cuda(water["P"]))
    prof = nao.nao_profile_read(g.h)
    nao.nao_profile_enable(g.h, False)
    assert prof["h_fp64"][0] >= 1 and prof["n_fp64"][0] >= 1 and prof["eval_grad"][0] >= 1
    assert all(ms >= 0.0 for _, ms in prof.values())
