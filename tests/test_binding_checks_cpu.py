"""The binding's buffer-size checks, on the CPU: the C ABI cannot see the size of a device
buffer, so every wrapper checks the caller's buffers against the handle's sizes (and a grouped
call's lists against its number of systems) before it calls the library. Here the library is a
stand-in that accepts every call, and the handle's sizes come from stand-ins for nao_get_info
and nao_get_system, so only the binding's own checks run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1912_06636_gb300 import nao

NB, NP, NA = 7, 11, 2
SYSTEMS = [(3, 5), (4, 6)]  # (n_basis, n_points) of a grouped handle's systems


class _Info:
    def __init__(self, nb, npts, n_sys, n_atoms=NA):
        self.n_basis, self.n_points, self.n_systems, self.n_atoms = nb, npts, n_sys, n_atoms


class _AcceptAll:
    def __getattr__(self, name):
        return lambda *a: 0


@pytest.fixture
def fake(monkeypatch):
    state = {"grouped": False}

    def info(h):
        if state["grouped"]:
            return _Info(sum(b for b, _ in SYSTEMS), sum(p for _, p in SYSTEMS), len(SYSTEMS))
        return _Info(NB, NP, 1)

    def system(h, m):
        b, p = SYSTEMS[m]
        return {"n_basis": b, "n_points": p}

    monkeypatch.setattr(nao, "load", lambda: _AcceptAll())
    monkeypatch.setattr(nao, "nao_get_info", info)
    monkeypatch.setattr(nao, "nao_get_system", system)
    monkeypatch.setattr(nao, "_dptr", lambda t: None if t is None else 1)
    return state


def z(*shape):
    return torch.zeros(shape, dtype=torch.float64)


def test_single_system_calls(fake):
    h, s = object(), 0
    nao.nao_integrate_h(h, z(NP), 3, "fp64", z(NB, NB), s)
    nao.nao_integrate_h(h, None, 3, "fp64", z(NB, NB), s)
    for bad in (lambda: nao.nao_integrate_h(h, z(NP - 1), 3, "fp64", z(NB, NB), s),
                lambda: nao.nao_integrate_h(h, z(NP), 3, "fp64", z(NB, NB - 1), s),
                lambda: nao.nao_integrate_h_tau(h, z(NP), z(NP - 1), 7, "fp64", z(NB, NB), s),
                lambda: nao.nao_update_density(h, z(NB, NB), "fp64", z(NP - 1), z(1), s),
                lambda: nao.nao_update_density(h, z(NB, NB), "fp64", z(NP), z(0), s),
                lambda: nao.nao_update_density_gradient(h, z(NB, NB), "fp64", z(NP), z(3, NP - 1), None, s),
                lambda: nao.nao_update_density_hessian(h, z(NB, NB), "fp64", z(NP), z(3, NP), z(5, NP), None, s),
                lambda: nao.nao_pulay_matrices(h, None, "fp64", z(3, NB, NB), z(2, NB, NB), s),
                lambda: nao.nao_pulay_forces(h, z(NB, NB), z(NB, NB), z(3, NB, NB), z(3, NB, NB - 1), z(6), s),
                lambda: nao.nao_pulay_forces(h, z(NB, NB), z(NB, NB), z(3, NB, NB), z(3, NB, NB), z(3 * NA - 1), s),
                lambda: nao.nao_integrate_h_noalloc(h, z(NP), 3, z(NB), s)):
        with pytest.raises(ValueError):
            bad()
    nao.nao_integrate_h_tau(h, z(NP), z(NP), 7, "fp64", z(NB, NB), s)
    nao.nao_update_density(h, z(NB, NB), "fp64", z(NP), None, s)
    nao.nao_update_density_gradient(h, z(NB, NB), "split", z(NP), z(3, NP), z(1), s)
    nao.nao_update_density_hessian(h, z(NB, NB), "fp64", z(NP), z(3, NP), z(6, NP), z(1), s)
    nao.nao_pulay_matrices(h, z(NP), "fp64", z(3, NB, NB), z(3, NB, NB), s)
    nao.nao_pulay_forces(h, z(NB, NB), z(NB, NB), z(3, NB, NB), z(3, NB, NB), z(3 * NA), s)
    nao.nao_integrate_h_noalloc(h, z(NP), 3, z(NB, NB), s)


def test_host_buffer_calls(fake):
    h = object()
    nao.nao_integrate_h_host(h, np.zeros(NP), 3, "fp64", np.zeros((NB, NB)), 0)
    assert nao.nao_update_density_host(h, np.zeros((NB, NB)), "fp64", np.zeros(NP), 0) == 0.0
    with pytest.raises(ValueError):
        nao.nao_integrate_h_host(h, np.zeros(NP - 1), 3, "fp64", np.zeros((NB, NB)), 0)
    with pytest.raises(ValueError):
        nao.nao_update_density_host(h, np.zeros((NB, NB)), "fp64", np.zeros(NP - 1), 0)


def test_grouped_calls(fake):
    fake["grouped"] = True
    h, s = object(), 0
    vs = [z(p) for _, p in SYSTEMS]
    Hs = [z(b, b) for b, _ in SYSTEMS]
    Ps = [z(b, b) for b, _ in SYSTEMS]
    ns = [z(p) for _, p in SYSTEMS]
    nes = [z(1) for _ in SYSTEMS]
    nao.nao_integrate_h_many(h, vs, 3, "split", Hs, s)
    nao.nao_integrate_h_many(h, None, 1, "fp64", Hs, s)
    nao.nao_integrate_h_many(h, [None, vs[1]], 1, "fp64", Hs, s)
    nao.nao_update_density_many(h, Ps, "fp64", ns, nes, s)
    nao.nao_update_density_many(h, Ps, "fp64", ns, [nes[0], None], s)
    nao.nao_update_density_gradient_many(h, Ps, "fp64", ns, [z(3, p) for _, p in SYSTEMS], None, s)
    for bad in (lambda: nao.nao_integrate_h_many(h, vs[:1], 3, "fp64", Hs, s),  # one entry per system
                lambda: nao.nao_integrate_h_many(h, vs, 3, "fp64", [Hs[0], z(3, 3)], s),
                lambda: nao.nao_update_density_many(h, Ps, "fp64", [ns[0], z(5)], nes, s),
                lambda: nao.nao_update_density_many(h, Ps + Ps, "fp64", ns, nes, s),
                lambda: nao.nao_update_density_gradient_many(h, Ps, "fp64", ns, [z(3, 5), z(3, 5)], None, s)):
        with pytest.raises(ValueError):
            bad()
