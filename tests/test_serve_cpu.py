"""Host-side pieces of the serving loop and of the workload generators (no GPU)."""
import numpy as np

from paper_1912_06636_gb300 import serve, synth


def test_serving_stream_shape():
    st = synth.serving_stream(4000, rate=200.0, seed=4, n_min=3, n_max=200)
    t = np.array([a for a, _, _ in st])
    n = np.array([b for _, b, _ in st])
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 200.0) < 200.0 * 0.05  # Poisson rate
    assert n.min() >= 3 and n.max() <= 200
    # log-uniform sizes: the median is near sqrt(3 * 201)
    assert 18 < np.median(n) < 30
    assert st == synth.serving_stream(4000, rate=200.0, seed=4, n_min=3, n_max=200)  # seeded


def test_random_molecule_rules():
    m = synth.random_molecule(25, 11, n_rad=4, n_theta=2, n_phi=3)
    d = np.linalg.norm(m.atom_xyz[:, None] - m.atom_xyz[None], axis=2)
    d[np.arange(25), np.arange(25)] = np.inf
    assert d.min() >= 2.0
    radius = (3 * 135.0 * 25 / (4 * np.pi)) ** (1 / 3)
    assert np.all(np.linalg.norm(m.atom_xyz, axis=1) <= radius)
    assert set(np.unique(m.atom_species)) <= {0, 1, 2}
    assert serve.n_basis_of(m) == m.n_basis
    assert m.n_points == 25 * 4 * 6


def test_slab_geometry():
    atoms, spec = synth.slab_geometry()
    assert atoms.shape == (375, 3)
    assert np.bincount(spec).tolist() == [150, 225]
    d = np.linalg.norm(atoms[:, None] - atoms[None], axis=2)
    d[np.arange(375), np.arange(375)] = np.inf
    assert d.min() > 3.4
    A, B = synth.slab_species("A"), synth.slab_species("B")
    nb = lambda sp: sum(2 * l + 1 for l in sp.ls)
    assert nb(A) == nb(B) == 40 and 150 * nb(A) + 225 * nb(B) == 15000


def test_estimate_bytes_grows_with_size():
    small = serve.estimate_bytes(10_000, 100, 200, 256 << 20, 16)
    big_pts = serve.estimate_bytes(1_000_000, 100, 200, 256 << 20, 16)
    big_nb = serve.estimate_bytes(10_000, 5000, 200, 256 << 20, 16)
    assert small < big_pts and small < big_nb
    assert big_nb >= 16 * 5000 * 5000  # H and P


def test_summarize():
    rs = [serve.Result(rid=i, arrival_s=0.01 * i, admitted_s=0.01 * i, started_s=0.01 * i + 0.001,
                       done_s=0.01 * i + 0.1 + 0.001 * i, n_points=1000, n_basis=10, n_iter=20, device_bytes=1,
                       n_electrons=np.ones(20)) for i in range(100)]
    sm = serve.summarize(rs, {"makespan_s": 2.0, "peak_active": 4, "peak_reserved_bytes": 10 ** 9})
    assert sm["requests"] == 100
    assert abs(sm["p50_ms"] - (100 + 0.5 * 99 * 1)) < 1.0
    assert sm["p99_ms"] > sm["p50_ms"]
    assert sm["point_iterations_per_s"] == 100 * 1000 * 20 / 2.0
