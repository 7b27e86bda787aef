"""GPU parity of the split-precision (Ozaki slices on tcgen05 tensor cores) path against the
FP64 oracle: e_H, e_n <= 1e-10 (tests/_metrics.py); the error falls as slices are added."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import raw_rel_err, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


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
    return dict(s=s, o=o, v=v, P=P, H=H, A=A, n=n, D=D, ne=ne)


def run(water, **opts):
    with nao.Grid(water["s"], device=0, **opts) as g:
        H = g.integrate_h(cuda(water["v"]), prec="split")
        n, ne = g.update_density(cuda(water["P"]), prec="split")
        torch.cuda.synchronize()
        g.sync()
        return H.cpu().numpy(), n.cpu().numpy(), float(ne.item())


def test_split_hamiltonian_and_density(water):
    H, n, ne = run(water)
    assert np.array_equal(H, H.T)
    eH = rel_err(H, water["H"], water["A"])
    en = rel_err(n, water["n"], water["D"])
    print(f"split e_H={eH:.2e} (raw {raw_rel_err(H, water['H'], water['A']):.2e}) e_n={en:.2e}")
    assert eH <= TOL and en <= TOL
    assert abs(ne - water["ne"]) <= TOL * abs(water["ne"])


def test_split_overlap_and_kinetic(water):
    s, o = water["s"], water["o"]
    S_ref, SA = o.overlap(s.pt_xyz, s.pt_w)
    T_ref, TA = o.hamiltonian(s.pt_xyz, s.pt_w, None, oracle.TERM_KINETIC)
    with nao.Grid(s, device=0) as g:
        S = g.overlap(prec="split").cpu().numpy()
        T = g.integrate_h(None, nao.NAO_TERM_KINETIC, prec="split").cpu().numpy()
    assert rel_err(S, S_ref, SA) <= TOL
    assert rel_err(T, T_ref, TA) <= TOL


def test_split_error_falls_with_slices(water):
    errs = []
    for S in (4, 6, 8, 10, 11, 12):
        H, n, _ = run(water, split_slices=S)
        errs.append((rel_err(H, water["H"], water["A"]), rel_err(n, water["n"], water["D"])))
    print("split errors by slices 4,6,8,10,11,12:", errs)
    assert errs[0][0] > errs[2][0] and errs[0][1] > errs[2][1]
    for e in errs[3:]:
        assert e[0] <= TOL and e[1] <= TOL


# Exact slice sums need K S < 2^14 per accumulation: the H contraction (K = 4 Ppad, Ppad = batch
# points rounded up to 16) accumulates batches of more than 336 points at 12 slices (400 at 10)
# in K segments; (1024, 12) gives 4.3 segments' worth of K on the one-atom grid below.
@pytest.mark.parametrize("B,S", [(1, 12), (37, 12), (128, 12), (336, 12), (337, 12), (400, 12), (400, 10),
                                 (512, 12), (512, 10), (401, 10)])
def test_split_independent_of_batch_size(water, B, S):
    H, n, _ = run(water, max_batch_points=B, split_slices=S)
    assert rel_err(H, water["H"], water["A"]) <= TOL
    assert rel_err(n, water["n"], water["D"]) <= TOL


def test_split_segments_cover_every_k_chunk():
    """Batch sizes that put the segment boundary at every position of a chunk: one atom, so
    every batch has the same functions and H over the whole grid must not depend on B."""
    s = synth.make_system([[0.0, 0.0, 0.0]], [0], [synth.Species(ls=[0, 1, 2], alphas=[1.2, 0.7, 0.9], Z=2.0)],
                          n_rad=40, n_theta=8, n_phi=9)
    o = oracle.Oracle(s)
    v = s.potential()
    H_ref, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    for B in (321, 352, 368, 384, 448, 496, 512):
        with nao.Grid(s, device=0, max_batch_points=B, split_slices=12) as g:
            H = g.integrate_h(cuda(v), prec="split").cpu().numpy()
        assert rel_err(H, H_ref, A) <= TOL, B


@pytest.mark.parametrize("B,S", [(1024, 10), (600, 12)])
def test_split_rejects_batches_beyond_512_points(water, B, S):
    with nao.Grid(water["s"], device=0, max_batch_points=B, split_slices=S) as g:
        with pytest.raises(nao.NaoError) as e:
            g.integrate_h(cuda(water["v"]), prec="split")
        assert e.value.code == nao.NAO_ERR_UNSUPPORTED


# ---- e4m3 digits (options.split_digits = 1): balanced base-32 digits, |d| <= 16, exact in e4m3,
# kind::f8f6f4 MMAs; 5 bits per slice, so 14 slices carry 70 bits (11 bf16 slices carry 66).
def test_e4m3_hamiltonian_and_density(water):
    H, n, ne = run(water, split_digits=1, split_slices=14)
    assert np.array_equal(H, H.T)
    eH = rel_err(H, water["H"], water["A"])
    en = rel_err(n, water["n"], water["D"])
    print(f"e4m3 14 slices: e_H={eH:.2e} (raw {raw_rel_err(H, water['H'], water['A']):.2e}) e_n={en:.2e}")
    assert eH <= TOL and en <= TOL
    assert abs(ne - water["ne"]) <= TOL * abs(water["ne"])


def test_e4m3_error_falls_with_slices(water):
    errs = {}
    for S in (8, 10, 12, 14, 16):
        H, n, _ = run(water, split_digits=1, split_slices=S)
        errs[S] = (rel_err(H, water["H"], water["A"]), rel_err(n, water["n"], water["D"]))
    print("e4m3 errors by slices:", errs)
    # 8 slices carry 40 bits (about 6.7 bf16 slices): well above FP64 rounding on this molecule,
    # and about 32^2 more accurate two slices later
    assert errs[8][0] > 1e-12 and errs[8][0] / max(errs[10][0], 1e-300) > 300.0
    for S in (12, 14, 16):
        assert errs[S][0] <= TOL and errs[S][1] <= TOL


@pytest.mark.parametrize("B", [1, 37, 200, 400, 512])
def test_e4m3_independent_of_batch_size(water, B):
    H, n, _ = run(water, max_batch_points=B, split_digits=1, split_slices=14)
    assert rel_err(H, water["H"], water["A"]) <= TOL
    assert rel_err(n, water["n"], water["D"]) <= TOL


def test_e4m3_overlap_kinetic_and_gradient(water):
    s, o = water["s"], water["o"]
    S_ref, SA = o.overlap(s.pt_xyz, s.pt_w)
    T_ref, TA = o.hamiltonian(s.pt_xyz, s.pt_w, None, oracle.TERM_KINETIC)
    g_ref, Dg = o.density_gradient(s.pt_xyz, water["P"])
    with nao.Grid(s, device=0, split_digits=1, split_slices=14) as g:
        S = g.overlap(prec="split").cpu().numpy()
        T = g.integrate_h(None, nao.NAO_TERM_KINETIC, prec="split").cpu().numpy()
        n, grad, _ = g.density_gradient(cuda(water["P"]), prec="split")
        torch.cuda.synchronize()
        g.sync()
    assert rel_err(S, S_ref, SA) <= TOL
    assert rel_err(T, T_ref, TA) <= TOL
    assert rel_err(n.cpu().numpy(), water["n"], water["D"]) <= TOL
    gr = grad.cpu().numpy()
    for c in range(3):
        assert rel_err(gr[c], g_ref[:, c], Dg[:, c]) <= TOL


def test_digit_options_are_checked(water):
    for opts in (dict(split_digits=2), dict(split_digits=1, split_slices=7), dict(split_digits=1, split_slices=17),
                 dict(split_digits=0, split_slices=13)):
        with pytest.raises(nao.NaoError) as e:
            nao.Grid(water["s"], device=0, **opts)
        assert e.value.code == nao.NAO_ERR_INVALID_ARG


@pytest.mark.parametrize("case", ["water", "molecule_l3"])
def test_split_evaluation_matches_oracle(case):
    """The split path evaluates the basis in float-float arithmetic on the FP32 pipe (FP64 for the
    geometry, the radial coordinate and points within 0.1 bohr of a nucleus). Per basis function,
    with the function's largest magnitude over the whole grid as the scale (a spline keeps
    absolute accuracy, so where a function is tiny, near its cutoff or near its own nucleus for
    l > 0, only the error against that scale is meaningful), every value and gradient component
    of several batches is checked against the FP64 evaluation of the same batch on the GPU and
    against the oracle, both at 2e-13. Float-float keeps about 47 bits: a product loses up to ~3
    units of 2^-48 and the solid-harmonic recurrence chains ~10 of them at l = 3, so near a nodal
    surface of an f function (value ~0, terms of the order of the function's maximum) the
    difference reaches ~1.3e-13 of the maximum; the FP64 evaluation itself sits ~1.1e-13 from the
    oracle on water (the oracle's radial coordinate ln(r/r0)/Delta moves steep functions by that
    much). Both stay far below what the split path's H and n need (1e-10 of the magnitude sums)."""
    if case == "water":
        s, bp = synth.config_water(), 200
    else:
        s, bp = synth.random_molecule(5, 7311, n_rad=12, n_theta=5, n_phi=6), 120
        assert max(s.fn_l) >= 3
    o = oracle.Oracle(s)
    aphi, agrad = o.eval_dense(s.pt_xyz)
    fscale = np.maximum(np.abs(aphi).max(axis=0), 1e-300)[:, None]           # [nb, 1]
    gfscale = np.maximum(np.abs(agrad).max(axis=(0, 2)), 1e-300)[None, :, None]  # [1, nb, 1]
    with nao.Grid(s, device=0, max_batch_points=bp) as g:
        bo, pp, ro, ri = g.batches()
        nonempty = np.nonzero(np.diff(ro))[0]
        w_or = w_64 = 0.0
        for b in nonempty[:: max(1, len(nonempty) // 12)]:
            b = int(b)
            pts = s.pt_xyz[pp[bo[b]:bo[b + 1]]]
            rphi, rgrad = o.eval_dense(pts)
            rel = ri[ro[b]:ro[b + 1]]
            rphi = rphi[:, rel].T
            rgrad = np.transpose(rgrad[:, rel, :], (2, 1, 0))
            phi, grad = (t.cpu().numpy() for t in g.evaluate_batch(b, prec="split"))
            phi64, grad64 = (t.cpu().numpy() for t in g.evaluate_batch(b, prec="fp64"))
            scale, gscale = fscale[rel], gfscale[:, rel]
            w_or = max(w_or, float(np.max(np.abs(phi - rphi) / scale)), float(np.max(np.abs(grad - rgrad) / gscale)))
            w_64 = max(w_64, float(np.max(np.abs(phi - phi64) / scale)), float(np.max(np.abs(grad - grad64) / gscale)))
        print(f"{case}: split evaluation, worst {w_64:.2e} against the GPU's FP64 evaluation, {w_or:.2e} against the oracle")
        assert w_64 <= 2e-13 and w_or <= 2e-13
