"""The continuous-batching request loop (paper_1912_06636_gb300/serve.py) on the GPU.

Each request's results are the same alone and in the mix (requests admitted as slots free up,
overlapping on the device), within the stated tolerances (FP64 1e-12, split 1e-10); the
admission respects the HBM budget; and the last iteration of a request matches the oracle
for the same v and P.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import serve, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "split": 1e-10}
GRID = dict(n_rad=16, n_theta=6, n_phi=7)


def _requests(n_iter=4):
    sizes = [3, 9, 4, 12, 6, 5]
    out = []
    for i, na in enumerate(sizes):
        s = synth.random_molecule(na, 500 + i, **GRID)
        out.append(serve.Request(rid=i, system=s, v0=s.potential(), arrival_s=0.0, n_iter=n_iter, seed=70 + i))
    return out


@pytest.fixture(scope="module")
def reqs():
    return _requests()


def _last_inputs(q):
    """v and P of a request's last iteration, regenerated the way the server draws them."""
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(q.seed) * 1_000_003 + q.n_iter - 1)
    u = torch.rand(len(q.v0), generator=gen, dtype=torch.float64, device=dev)
    X = torch.randn((q.system.n_basis, 16), generator=gen, dtype=torch.float64, device=dev)
    v = (torch.from_numpy(q.v0).to(dev) * (u * 0.02 + 0.99)).cpu().numpy()
    P = (X @ X.t() / 16.0).cpu().numpy()
    return v, P


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_alone_equals_mix(reqs, prec):
    """Element by element, in the measure of every other parity test: |H_mix - H_alone| against
    the magnitude sums A of the oracle's H, |n_mix - n_alone| against D (tests/_metrics.py)."""
    mix_server = serve.Server(prec=prec, max_active=4, keep_results=True)
    mix = mix_server.run(reqs)
    assert [r.rid for r in mix] == list(range(len(reqs)))
    assert mix_server.stats["peak_active"] >= 2  # requests did overlap
    for q, m in zip(reqs, mix):
        alone = serve.Server(prec=prec, max_active=1, keep_results=True).run([q])[0]
        v, P = _last_inputs(q)
        o = oracle.Oracle(q.system)
        H_ref, A = o.hamiltonian(q.system.pt_xyz, q.system.pt_w, v)
        n_ref, D, _ = o.density(q.system.pt_xyz, P)
        assert rel_err(m.H, alone.H, A) <= TOL[prec], q.rid
        assert rel_err(m.n, alone.n, D) <= TOL[prec], q.rid
        # and both against the oracle
        assert rel_err(m.H, H_ref, A) <= TOL[prec] and rel_err(alone.n, n_ref, D) <= TOL[prec], q.rid
        assert np.allclose(m.n_electrons, alone.n_electrons, rtol=TOL[prec], atol=0.0)
        assert np.all(m.n_electrons > 0)


def test_admission_respects_budget(reqs):
    ests = [serve.estimate_bytes(len(q.v0), serve.n_basis_of(q.system), 200, 256 << 20, 16) for q in reqs]
    budget = int(max(ests) * 1.5)  # never room for two of the largest, sometimes for two small ones
    srv = serve.Server(prec="split", max_active=8, hbm_budget_bytes=budget)
    res = srv.run(reqs)
    assert len(res) == len(reqs)
    assert srv.stats["peak_reserved_bytes"] <= budget
    for r, e in zip(res, ests):  # the estimate bounds what a request actually held
        assert r.device_bytes <= e


def test_staggered_arrivals_and_oracle(reqs):
    qs = [serve.Request(rid=q.rid, system=q.system, v0=q.v0, arrival_s=0.02 * k, n_iter=3, seed=q.seed)
          for k, q in enumerate(reqs[:3])]
    srv = serve.Server(prec="fp64", max_active=2, keep_results=True)
    res = srv.run(qs)
    for r, q in zip(res, qs):
        assert r.admitted_s >= q.arrival_s and r.done_s > r.started_s >= r.admitted_s
    # the last iteration of request 1 against the oracle, with v and P regenerated the same way
    q, r = qs[1], res[1]
    s = q.system
    v, P = _last_inputs(q)
    o = oracle.Oracle(s)
    H, A = o.hamiltonian(s.pt_xyz, s.pt_w, v)
    n, D, ne = o.density(s.pt_xyz, P, s.pt_w)
    assert rel_err(r.H, H, A) <= 1e-12
    assert rel_err(r.n, n, D) <= 1e-12
    assert abs(r.n_electrons[-1] - ne) <= 1e-12 * abs(ne)


def test_summary(reqs):
    srv = serve.Server(prec="split", max_active=3)
    res = srv.run(reqs[:4])
    sm = serve.summarize(res, srv.stats)
    assert sm["requests"] == 4 and sm["p99_ms"] >= sm["p50_ms"] > 0
    assert sm["point_iterations_per_s"] > 0
