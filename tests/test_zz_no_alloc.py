"""nao_integrate_h_noalloc: the FP64 Hamiltonian computed with the library's fixed device
scratch array instead of allocated memory.

It serves callers that cannot allocate device memory where they integrate (an application
whose own memory manager owns all device memory, or a loop that must not call
cudaMalloc/cudaFree). Through the C ABI, two calls in a row must reproduce nao_integrate_h's
H within the FP64 parity bar used by the other tests, and a handle whose evaluation chunks do
not fit the array must be refused. The file name makes pytest collect it last; it also
passes alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1912_06636_gb300 import nao, synth
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-12


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_integrate_h_on_two_calls():
    s = synth.config_water()
    v = s.potential()
    _, A = oracle.Oracle(s).hamiltonian(s.pt_xyz, s.pt_w, v)
    with nao.Grid(s, device=0, scratch_bytes=16 << 20) as g:
        vv = cuda(v)
        H_ref = g.integrate_h(vv, prec="fp64").cpu().numpy()
        for _ in range(2):
            H = torch.full((g.nb, g.nb), float("nan"), dtype=torch.float64, device="cuda")
            nao.nao_integrate_h_noalloc(g.h, vv, nao.NAO_TERM_POTENTIAL | nao.NAO_TERM_KINETIC, H)
            torch.cuda.synchronize()
            g.sync()
            Hn = H.cpu().numpy()
            assert np.all(np.isfinite(Hn))
            assert np.array_equal(Hn, Hn.T)
            assert rel_err(Hn, H_ref, A) <= TOL


def test_noalloc_refuses_chunks_larger_than_its_array():
    s = synth.config_water(n_rad=80, n_theta=20, n_phi=21)  # ~64 MB of evaluated functions
    v = cuda(s.potential())
    with nao.Grid(s, device=0) as g:  # default chunk budget: one chunk holding everything
        H = torch.zeros((g.nb, g.nb), dtype=torch.float64, device="cuda")
        with pytest.raises(nao.NaoError) as e:
            nao.nao_integrate_h_noalloc(g.h, v, 3, H)
        assert e.value.code == nao.NAO_ERR_INVALID_ARG
        assert "NAO_NOALLOC_SCRATCH_BYTES" in str(e.value)
    with nao.Grid(s, device=0, scratch_bytes=nao.NAO_NOALLOC_SCRATCH_BYTES) as g:
        H_ref = g.integrate_h(v).cpu().numpy()
        H = torch.zeros((g.nb, g.nb), dtype=torch.float64, device="cuda")
        nao.nao_integrate_h_noalloc(g.h, v, 3, H)
        torch.cuda.synchronize()
        assert np.max(np.abs(H.cpu().numpy() - H_ref)) <= 1e-13 * np.max(np.abs(H_ref))
