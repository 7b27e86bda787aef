"""Failure handling without a GPU fault (host-side injection and a bounded device wait that is
made to run out).

Every device allocation, host<->device copy and kernel launch that creating a handle and
running H and n on the FP64 and split paths makes is made to fail in turn (nao_fault_inject):
the entry point that hits it returns an error that says the failure was injected, a failed
create leaves no handle, a failed call leaves its handle usable, and with the injection cleared
the same handle (or a new one) gives the oracle's results. A bounded mbarrier wait that nothing
completes gives up and nao_sync_status reports NAO_ERR_TIMEOUT once; later calls run normally.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "split": 1e-10}


@pytest.fixture(scope="module")
def water():
    s = synth.config_water(n_rad=14, n_theta=6, n_phi=7, max_batch_points=60)
    v = s.potential()
    P = synth.density_matrix(s, 0)
    o = oracle.Oracle(s)
    H, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    n, D, _ = o.density(s.pt_xyz, P)
    return dict(s=s, v=torch.from_numpy(v).cuda(), P=torch.from_numpy(P).cuda(), H=H, A=A, n=n, D=D)


def _run(g, w, prec):
    H = g.integrate_h(w["v"], prec=prec)
    n, _ = g.update_density(w["P"], prec=prec)
    torch.cuda.synchronize()
    g.sync()
    return H.cpu().numpy(), n.cpu().numpy()


def _good(g, w, prec):
    H, n = _run(g, w, prec)
    return rel_err(H, w["H"], w["A"]) <= TOL[prec] and rel_err(n, w["n"], w["D"]) <= TOL[prec]


@pytest.mark.parametrize("kind", ["alloc", "copy", "launch"])
def test_every_injected_failure_unwinds(water, kind):
    fired = 0
    for k in range(1, 400):
        nao.nao_fault_inject(f"{kind}:{k}")
        err = None
        g = None
        try:
            g = nao.Grid(water["s"], device=0, max_batch_points=60, capture_graph=1 if k % 2 else 0)
            for prec in ("fp64", "split"):
                _run(g, water, prec)
        except nao.NaoError as e:
            err = e
        finally:
            nao.nao_fault_inject(None)
        if err is None:
            if g is not None:
                g.close()
            break  # k is past the last operation of this kind: nothing fired
        fired += 1
        assert "injected failure" in str(err), str(err)
        assert err.code == (nao.NAO_ERR_OUT_OF_MEMORY if kind == "alloc" else nao.NAO_ERR_CUDA)
        if g is not None:  # the failure came from a call on a live handle: it is still usable
            assert _good(g, water, "fp64") and _good(g, water, "split"), (kind, k)
            g.close()
        else:  # a failed create: a fresh handle works
            with nao.Grid(water["s"], device=0, max_batch_points=60) as g2:
                assert _good(g2, water, "split"), (kind, k)
    assert fired >= 3, f"only {fired} {kind} operations were exercised"
    print(f"{kind}: {fired} injection points, every one unwound")


def test_bounded_wait_times_out_and_is_reported_once(water):
    with nao.Grid(water["s"], device=0, max_batch_points=60) as g:
        assert _good(g, water, "split")
        nao.nao_check_wait_timeout(g.h, 2_000_000)  # about a millisecond
        with pytest.raises(nao.NaoError) as e:
            g.sync()
        assert e.value.code == nao.NAO_ERR_TIMEOUT
        g.sync()  # reported once
        assert _good(g, water, "split") and _good(g, water, "fp64")
