"""Seeded synthetic inputs for real-space grid integration with numeric atom-centred orbitals.

This module only *generates inputs*: atoms, per-species radial function tables, the
integration grid with its partition-of-unity weights, a local potential v and a
symmetric positive semi-definite density matrix P. It holds none of the integration
method's arithmetic (no spline, no spherical harmonics, no batch contraction), so both
the CUDA path and the FP64 oracle can consume the same arrays without sharing code.

Inputs follow the paper's statement of the problem:
  * points are atom-centred radial shells x angular points, weighted by a
    partition of unity (Sec. 3.2.1, Eq. H_int_aims);
  * radial functions are confined so that they reach zero at a cutoff radius and
    stay zero beyond it (Sec. 3.2.1, NAO basis paragraph);
  * the paper's Lebedev grids, Blum09 radial rule, Stratmann weights and NAO species
    files are not available, so the stand-ins are: Gauss-Chebyshev (2nd kind) radial
    shells with a Becke map, Gauss-Legendre(theta) x uniform(phi) angular product
    grids, plain Becke (1988) cell functions, and cutoff-smoothed Gaussian radial
    functions N r^l exp(-alpha r^2) c(r).

Seeds use numpy's PCG64 everywhere.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

try:  # scipy is present on both machines; keep the import local to what needs it
    from scipy.special import erf as _erf
except Exception:  # pragma: no cover
    _erf = np.vectorize(math.erf)

R0_DEFAULT = 1e-4
RLAST_DEFAULT = 8.0
NRGRID_DEFAULT = 1000
RCUT_DEFAULT = 6.0


# ----------------------------------------------------------------------------------------
# radial functions (inputs): N r^l exp(-alpha r^2) with a smooth cutoff
# ----------------------------------------------------------------------------------------
def gaussian_norm(l: int, alpha: float) -> float:
    """N with N^2 int_0^inf r^(2l) e^(-2 alpha r^2) r^2 dr = 1."""
    return math.sqrt(2.0 * (2.0 * alpha) ** (l + 1.5) / math.gamma(l + 1.5))


def cutoff_smoothing(r: np.ndarray, rc: float) -> np.ndarray:
    """1 inside rc-1, a C2 quintic step down to 0 on [rc-1, rc], 0 beyond."""
    r = np.asarray(r, dtype=np.float64)
    t = np.clip(r - (rc - 1.0), 0.0, 1.0)
    c = 1.0 - (10.0 * t**3 - 15.0 * t**4 + 6.0 * t**5)
    return np.where(r >= rc, 0.0, c)


def radial_function(r: np.ndarray, l: int, alpha: float, rc: float) -> np.ndarray:
    r = np.asarray(r, dtype=np.float64)
    return gaussian_norm(l, alpha) * r**l * np.exp(-alpha * r * r) * cutoff_smoothing(r, rc)


def log_grid(n: int, r0: float, r_last: float) -> np.ndarray:
    k = np.arange(n, dtype=np.float64)
    return r0 * (r_last / r0) ** (k / (n - 1))


# ----------------------------------------------------------------------------------------
# integration grid (inputs)
# ----------------------------------------------------------------------------------------
def radial_shells(n: int, rm: float = 1.0):
    """Gauss-Chebyshev (2nd kind) nodes mapped by r = rm (1+x)/(1-x); weights include r^2."""
    i = np.arange(1, n + 1, dtype=np.float64)
    th = i * math.pi / (n + 1)
    x = np.cos(th)
    r = rm * (1.0 + x) / (1.0 - x)
    w = math.pi / (n + 1) * np.sin(th) * (2.0 * rm / (1.0 - x) ** 2) * r * r
    return r, w


def angular_product_grid(n_theta: int, n_phi: int):
    """Gauss-Legendre in cos(theta) times a uniform phi grid (phi_0 = 0); weights sum to 4 pi."""
    u, wu = np.polynomial.legendre.leggauss(n_theta)
    phi = 2.0 * math.pi * np.arange(n_phi, dtype=np.float64) / n_phi
    ct = np.repeat(u, n_phi)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = np.tile(phi, n_theta)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    w = np.repeat(wu, n_phi) * (2.0 * math.pi / n_phi)
    return dirs, w


def becke_weights(pts: np.ndarray, owner: np.ndarray, atoms: np.ndarray, device: str | None = None,
                  chunk: int = 8192) -> np.ndarray:
    """Plain Becke (1988) partition weight of each point for the atom that owns it.

    Vectorised with torch (CPU threads, or a CUDA device when one is given or present):
    this is input generation, not part of the integration method.
    """
    import torch

    n_atoms = atoms.shape[0]
    if n_atoms == 1:
        return np.ones(pts.shape[0], dtype=np.float64)
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    A = torch.as_tensor(atoms, dtype=torch.float64, device=device)
    Rab = torch.cdist(A, A)
    Rab.fill_diagonal_(1.0)
    inv = 1.0 / Rab
    eye = torch.eye(n_atoms, dtype=torch.bool, device=device)
    P = torch.as_tensor(pts, dtype=torch.float64, device=device)
    own = torch.as_tensor(owner, dtype=torch.int64, device=device)
    out = torch.empty(pts.shape[0], dtype=torch.float64, device=device)
    if str(device).startswith("cuda"):
        chunk *= 8  # [c, A, A] temporaries of ~2 GB: fewer, larger steps on the GPU
    step = max(1, chunk * 64 * 64 // (n_atoms * n_atoms))
    for s in range(0, pts.shape[0], step):
        p = P[s : s + step]
        d = torch.sqrt(((p[:, None, :] - A[None, :, :]) ** 2).sum(-1))  # [c, A]
        mu = (d[:, :, None] - d[:, None, :]) * inv[None]  # [c, A, B]
        f = mu
        for _ in range(3):
            f = 1.5 * f - 0.5 * f * f * f
        sv = 0.5 * (1.0 - f)
        sv = torch.where(eye[None], torch.ones_like(sv), sv)
        cell = sv.prod(dim=2)  # [c, A]
        tot = cell.sum(dim=1)
        mine = cell.gather(1, own[s : s + step, None])[:, 0]
        out[s : s + step] = torch.where(tot > 0, mine / torch.where(tot > 0, tot, torch.ones_like(tot)), torch.zeros_like(tot))
    return out.cpu().numpy()


def build_grid(atoms: np.ndarray, n_rad, n_theta, n_phi, rm: float = 1.0):
    """Atom-major point list: for each atom, radial shell, theta, phi."""
    n_atoms = atoms.shape[0]
    n_rad = np.broadcast_to(np.asarray(n_rad), (n_atoms,))
    n_theta = np.broadcast_to(np.asarray(n_theta), (n_atoms,))
    n_phi = np.broadcast_to(np.asarray(n_phi), (n_atoms,))
    pts, wts, own = [], [], []
    for a in range(n_atoms):
        r, wr = radial_shells(int(n_rad[a]), rm)
        dirs, wa = angular_product_grid(int(n_theta[a]), int(n_phi[a]))
        p = atoms[a][None, None, :] + r[:, None, None] * dirs[None, :, :]
        pts.append(p.reshape(-1, 3))
        wts.append((wr[:, None] * wa[None, :]).reshape(-1))
        own.append(np.full(p.shape[0] * p.shape[1], a, dtype=np.int64))
    pts = np.concatenate(pts)
    wts = np.concatenate(wts)
    own = np.concatenate(own)
    wb = becke_weights(pts, own, atoms)
    return np.ascontiguousarray(pts), wts * wb


def model_potential(pts: np.ndarray, atoms: np.ndarray, Z: np.ndarray, on_device: bool = False) -> np.ndarray:
    """v(r) = sum_A [ -Z_A erf(r_A)/r_A + 0.3 exp(-r_A^2) ], with erf(r)/r -> 2/sqrt(pi) at r = 0.

    Inputs of more than 2M points (or any input, with on_device) are generated with torch on a
    CUDA device when one is present (input generation only; the caller passes the same array to
    every consumer)."""
    if pts.shape[0] > 2_000_000 or on_device:
        import torch

        if torch.cuda.is_available():
            P = torch.as_tensor(pts, dtype=torch.float64, device="cuda")
            v = torch.zeros(pts.shape[0], dtype=torch.float64, device="cuda")
            for a in range(atoms.shape[0]):
                r = torch.linalg.norm(P - torch.as_tensor(atoms[a], dtype=torch.float64, device="cuda")[None, :], dim=1)
                safe = torch.where(r > 0.0, r, torch.ones_like(r))
                ef = torch.where(r > 0.0, torch.erf(r) / safe, torch.full_like(r, 2.0 / math.sqrt(math.pi)))
                v += -float(Z[a]) * ef + 0.3 * torch.exp(-r * r)
            return v.cpu().numpy()
    v = np.zeros(pts.shape[0], dtype=np.float64)
    for a in range(atoms.shape[0]):
        r = np.linalg.norm(pts - atoms[a][None, :], axis=1)
        safe = np.where(r > 0.0, r, 1.0)
        ef = np.where(r > 0.0, _erf(r) / safe, 2.0 / math.sqrt(math.pi))
        v += -Z[a] * ef + 0.3 * np.exp(-r * r)
    return v


def random_psd(nb: int, seed: int, rank: int | None = None) -> np.ndarray:
    """P = X X^T / k with X ~ N(0,1) of shape nb x k (k = nb unless a rank is given)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = nb if rank is None else rank
    X = rng.standard_normal((nb, k))
    P = X @ X.T / k
    return np.ascontiguousarray(0.5 * (P + P.T))


# ----------------------------------------------------------------------------------------
# systems
# ----------------------------------------------------------------------------------------
@dataclass
class Species:
    ls: list  # angular momentum of each radial function
    alphas: list  # Gaussian exponent of each radial function
    rc: float = RCUT_DEFAULT
    Z: float = 1.0


@dataclass
class System:
    """Everything a grid handle is created from, plus generator metadata (alphas, Z)."""

    atom_xyz: np.ndarray
    atom_species: np.ndarray
    species_fn_offset: np.ndarray
    fn_l: np.ndarray
    fn_cutoff: np.ndarray
    fn_alpha: np.ndarray
    n_rgrid: int
    r0: float
    r_last: float
    fn_table: np.ndarray
    pt_xyz: np.ndarray
    pt_w: np.ndarray
    Z: np.ndarray
    max_batch_points: int = 200
    name: str = "custom"
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.atom_xyz.shape[0])

    @property
    def n_points(self) -> int:
        return int(self.pt_xyz.shape[0])

    @property
    def n_basis(self) -> int:
        per_species = [
            int(sum(2 * self.fn_l[f] + 1 for f in range(self.species_fn_offset[s], self.species_fn_offset[s + 1])))
            for s in range(len(self.species_fn_offset) - 1)
        ]
        return int(sum(per_species[s] for s in self.atom_species))

    def potential(self, on_device: bool = False) -> np.ndarray:
        return model_potential(self.pt_xyz, self.atom_xyz, self.Z, on_device)


def make_system(
    atoms,
    species_of_atom,
    species: list,
    n_rad=40,
    n_theta=10,
    n_phi=11,
    rm: float = 1.0,
    n_rgrid: int = NRGRID_DEFAULT,
    r0: float = R0_DEFAULT,
    r_last: float = RLAST_DEFAULT,
    max_batch_points: int = 200,
    name: str = "custom",
) -> System:
    atoms = np.ascontiguousarray(np.asarray(atoms, dtype=np.float64).reshape(-1, 3))
    species_of_atom = np.asarray(species_of_atom, dtype=np.int32)
    fn_l, fn_alpha, fn_rc, off = [], [], [], [0]
    for sp in species:
        fn_l += list(sp.ls)
        fn_alpha += list(sp.alphas)
        fn_rc += [sp.rc] * len(sp.ls)
        off.append(len(fn_l))
    rg = log_grid(n_rgrid, r0, r_last)
    table = np.stack([radial_function(rg, l, a, rc) for l, a, rc in zip(fn_l, fn_alpha, fn_rc)]) if fn_l else np.zeros((0, n_rgrid))
    pts, w = build_grid(atoms, n_rad, n_theta, n_phi, rm)
    Z = np.array([species[s].Z for s in species_of_atom], dtype=np.float64)
    return System(
        atom_xyz=atoms,
        atom_species=species_of_atom,
        species_fn_offset=np.asarray(off, dtype=np.int32),
        fn_l=np.asarray(fn_l, dtype=np.int32),
        fn_cutoff=np.asarray(fn_rc, dtype=np.float64),
        fn_alpha=np.asarray(fn_alpha, dtype=np.float64),
        n_rgrid=n_rgrid,
        r0=r0,
        r_last=r_last,
        fn_table=np.ascontiguousarray(table),
        pt_xyz=pts,
        pt_w=w,
        Z=Z,
        max_batch_points=max_batch_points,
        name=name,
    )


def _log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n))


def config_water(n_rad=40, n_theta=10, n_phi=11, max_batch_points=200) -> System:
    """3-atom molecule: heavy atom at the origin, light atoms at (+-1.43, 1.11, 0) bohr; 20 basis functions."""
    atoms = [[0.0, 0.0, 0.0], [1.43, 1.11, 0.0], [-1.43, 1.11, 0.0]]
    heavy = Species(ls=[0, 0, 1, 2], alphas=[10.0, 1.5, 0.4, 0.6], Z=8.0)
    light = Species(ls=[0, 0, 1], alphas=[1.2, 0.3, 0.8], Z=1.0)
    return make_system(atoms, [0, 1, 1], [heavy, light], n_rad, n_theta, n_phi, max_batch_points=max_batch_points, name="water3")


def diamond_cluster(a: float = 10.26, cells: int = 2) -> np.ndarray:
    base = np.array(
        [[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0],
         [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25]]
    )
    out = []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                out.append((base + np.array([i, j, k])) * a)
    return np.concatenate(out)


def silicon_species(seed: int = 1) -> Species:
    """2s,2p,2d,1f radial functions (25 basis functions), alpha log-uniform in [0.1, 20]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ls = [0, 0, 1, 1, 2, 2, 3]
    return Species(ls=ls, alphas=list(_log_uniform(rng, 0.1, 20.0, len(ls))), Z=14.0)


def config_diamond64(n_rad=60, n_theta=17, n_phi=18, max_batch_points=300, cells=2) -> System:
    """64-atom diamond-lattice cluster (cubic cell 10.26 bohr), 1600 basis functions, ~1.17M points."""
    atoms = diamond_cluster(10.26, cells)
    sp = silicon_species(1)
    return make_system(atoms, np.zeros(len(atoms), np.int32), [sp], n_rad, n_theta, n_phi,
                       max_batch_points=max_batch_points, name=f"diamond{len(atoms)}")


def slab_species(kind: str) -> Species:
    """Two-species slab basis: 4s,3p,4d,1f radial functions (40 basis functions per atom), alpha
    log-uniform in [0.1, 20]; species A (Z = 83, seed 2) and B (Z = 34, seed 3)."""
    seed, Z = {"A": (2, 83.0), "B": (3, 34.0)}[kind]
    rng = np.random.Generator(np.random.PCG64(seed))
    ls = [0, 0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 3]
    return Species(ls=ls, alphas=list(_log_uniform(rng, 0.1, 20.0, len(ls))), Z=Z)


def slab_geometry(layers: int = 15, n: int = 5, a: float = 7.8, pitch: float = 3.5):
    """Layered slab (finite cluster): `layers` layers of an n x n triangular lattice (spacing a),
    each layer shifted by (a/2, a/(2 sqrt 3)) from the one below (ABC stacking), layer pitch
    `pitch`; species pattern B A B A B in every five-layer unit (species index 0 = A, 1 = B)."""
    atoms, spec = [], []
    pattern = [1, 0, 1, 0, 1]
    for L in range(layers):
        sx, sy = (L % 3) * a / 2.0, (L % 3) * a / (2.0 * math.sqrt(3.0))
        for i in range(n):
            for j in range(n):
                atoms.append([i * a + j * a / 2.0 + sx, j * a * math.sqrt(3.0) / 2.0 + sy, L * pitch])
                spec.append(pattern[L % 5])
    return np.asarray(atoms, dtype=np.float64), np.asarray(spec, dtype=np.int32)


def config_slab375(n_rad=80, n_theta=14, n_phi=31, max_batch_points=200, layers=15, n=5) -> System:
    """375-atom layered slab of two species (150 A : 225 B), 15,000 basis functions, ~13M points."""
    atoms, spec = slab_geometry(layers, n)
    return make_system(atoms, spec, [slab_species("A"), slab_species("B")], n_rad, n_theta, n_phi,
                       max_batch_points=max_batch_points, name=f"slab{len(atoms)}")


# Per-atom grids of the species in their own configurations: Si as in the diamond cluster
# (60 shells x 17 x 18 directions), A and B as in the slab (80 shells x 14 x 31).
SPECIES_GRIDS = {"n_rad": (60, 80, 80), "n_theta": (17, 14, 14), "n_phi": (18, 31, 31)}


def random_molecule(n_atoms: int, seed: int, n_rad=40, n_theta=10, n_phi=11, max_batch_points=200,
                    min_dist: float = 2.0, species_grids: bool = False) -> System:
    """A random molecule: atoms placed one by one, uniformly in a sphere of volume 135 n_atoms
    bohr^3 (the atom density of silicon), rejecting any within min_dist of an earlier atom;
    each atom's species drawn uniformly from {Si (diamond cluster), A, B (slab)}. With
    species_grids, every atom gets its species' grid (SPECIES_GRIDS) instead of n_rad x
    (n_theta x n_phi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    radius = (3.0 * 135.0 * n_atoms / (4.0 * math.pi)) ** (1.0 / 3.0)
    atoms = []
    while len(atoms) < n_atoms:
        p = rng.uniform(-radius, radius, 3)
        if p @ p > radius * radius:
            continue
        if all(np.linalg.norm(p - q) >= min_dist for q in atoms):
            atoms.append(p)
    spec = rng.integers(0, 3, n_atoms).astype(np.int32)
    species = [silicon_species(1), slab_species("A"), slab_species("B")]
    if species_grids:
        n_rad, n_theta, n_phi = (np.asarray(SPECIES_GRIDS[k])[spec] for k in ("n_rad", "n_theta", "n_phi"))
    return make_system(np.asarray(atoms), spec, species, n_rad, n_theta, n_phi,
                       max_batch_points=max_batch_points, name=f"mol{n_atoms}-{seed}")


def molecule_set(n_mol: int, seed: int = 3000, n_min: int = 3, n_max: int = 60, b_min: int = 20, b_max: int = 400,
                 n_rad=60, n_theta=17, n_phi=18, species_grids: bool = False):
    """Independent molecules for one grouped handle: molecule k has a size log-uniform in
    [n_min, n_max] atoms and a batch size log-uniform in [b_min, b_max] points, both drawn
    with seed + k (random_molecule's rules for geometry, species and grids). Returns (systems, B)."""
    systems, bs = [], []
    for k in range(n_mol):
        rng = np.random.Generator(np.random.PCG64(seed + k))
        na = int(min(n_max, np.floor(_log_uniform(rng, n_min, n_max + 1, 1)[0])))
        b = int(min(b_max, np.floor(_log_uniform(rng, b_min, b_max + 1, 1)[0])))
        sysk = random_molecule(na, seed + k, n_rad, n_theta, n_phi, max_batch_points=b, species_grids=species_grids)
        systems.append(sysk)
        bs.append(b)
    return systems, bs


def serving_stream(n_requests: int, rate: float = 200.0, seed: int = 4, n_min: int = 3, n_max: int = 200):
    """Poisson arrivals at `rate` per second; molecule sizes log-uniform in [n_min, n_max] atoms.
    Returns a list of (arrival time in s, number of atoms, molecule seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    sizes = np.floor(_log_uniform(rng, n_min, n_max + 1, n_requests)).astype(int)
    return [(float(t[i]), int(min(sizes[i], n_max)), 4000 + i) for i in range(n_requests)]


def density_matrix(sys: System, seed: int, rank: int | None = None) -> np.ndarray:
    return random_psd(sys.n_basis, seed, rank)


def config(k: int, **kw) -> System:
    if k == 0:
        return config_water(**kw)
    if k == 1:
        return config_diamond64(**kw)
    if k == 2:
        return config_slab375(**kw)
    raise ValueError(f"unknown configuration {k}")


# ---------------------------------------------------------------------------------------
# Periodic cells (Eq. HamPeriodic): the unit cell's atoms and a uniform grid of its points.
# ---------------------------------------------------------------------------------------
def periodic_cell(lattice, frac_positions, species_of_atom, species: list, n_grid=12,
                  n_rgrid: int = NRGRID_DEFAULT, r0: float = R0_DEFAULT, r_last: float = RLAST_DEFAULT,
                  max_batch_points: int = 200) -> System:
    """Unit cell with lattice rows a1, a2, a3 (bohr) and atoms at fractional positions. The grid is
    the periodic trapezoid rule of the cell, fractional coordinates (i + 1/2) / n on each axis
    (n_grid: one n, or one per axis), weight V / (n1 n2 n3) (exact for trigonometric polynomials of degree < n_grid, so spectrally
    accurate for smooth periodic integrands); meta["lattice"] holds the lattice."""
    A = np.asarray(lattice, dtype=np.float64).reshape(3, 3)
    fr = np.asarray(frac_positions, dtype=np.float64).reshape(-1, 3)
    atoms = fr @ A
    sys0 = make_system(atoms, species_of_atom, species, n_rad=1, n_theta=1, n_phi=1, n_rgrid=n_rgrid, r0=r0,
                       r_last=r_last, max_batch_points=max_batch_points, name="periodic-cell")
    ng = (n_grid,) * 3 if np.isscalar(n_grid) else tuple(int(x) for x in n_grid)
    u = [(np.arange(n) + 0.5) / n for n in ng]
    f = np.stack(np.meshgrid(*u, indexing="ij"), axis=-1).reshape(-1, 3)
    sys0.pt_xyz = np.ascontiguousarray(f @ A)
    sys0.pt_w = np.full(f.shape[0], abs(np.linalg.det(A)) / float(np.prod(ng)))
    sys0.meta["lattice"] = A
    return sys0


def periodic_potential(sys0: System, pts=None) -> np.ndarray:
    """A smooth lattice-periodic potential: v = -1 + 0.3 cos(2 pi f1) + 0.2 sin(2 pi f2) + 0.1 cos(2 pi (f1 + f3))
    with f the fractional coordinates of the points."""
    A = sys0.meta["lattice"]
    f = np.asarray(sys0.pt_xyz if pts is None else pts) @ np.linalg.inv(A)
    t = 2 * np.pi * f
    return -1.0 + 0.3 * np.cos(t[:, 0]) + 0.2 * np.sin(t[:, 1]) + 0.1 * np.cos(t[:, 0] + t[:, 2])


def image_system(sys0: System, img_xyz, img_atom) -> System:
    """The unit cell's grid with the periodic images of its atoms as the atoms (the real-space
    system whose Hamiltonian is h^uc): img_atom[k] is the unit-cell atom of image k."""
    import copy

    s = copy.copy(sys0)
    s.atom_xyz = np.ascontiguousarray(np.asarray(img_xyz, dtype=np.float64).reshape(-1, 3))
    s.atom_species = np.ascontiguousarray(np.asarray(sys0.atom_species)[np.asarray(img_atom)], dtype=np.int32)
    s.Z = np.asarray(sys0.Z)[np.asarray(img_atom)]
    s.name = sys0.name + "-images"
    return s
