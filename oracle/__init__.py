"""FP64 CPU oracle (test infrastructure).

Only the tests, the package's smoke check and the benchmark's CPU-baseline leg may import
this module. It wraps ``oracle.c`` (plain C, FP64, ``-ffp-contract=off``) through ctypes
and shares no code with the CUDA library. See ``oracle.c`` for what each function computes
and which equation of the paper it follows.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, library routines, invariants, brute force), and
``tests/test_mutants_oracle.py`` checks that those pins catch plausible mistakes planted in copies
of ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_LIBDIR = _HERE / "lib"
_LIB = _LIBDIR / "liboracle.so"
_SRC = _HERE / "oracle.c"
_lib = None


def build(force: bool = False) -> Path:
    """Compile liboracle.so with gcc (no FMA contraction, no fast-math)."""
    _LIBDIR.mkdir(exist_ok=True)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-D_DEFAULT_SOURCE", str(_SRC), "-o", str(_LIB) + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(str(_LIB) + ".tmp", _LIB)
    return _LIB


class _Sys(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int32),
        ("atom_xyz", C.c_void_p),
        ("atom_species", C.c_void_p),
        ("n_species", C.c_int32),
        ("species_fn_offset", C.c_void_p),
        ("fn_l", C.c_void_p),
        ("fn_cutoff", C.c_void_p),
        ("n_rgrid", C.c_int32),
        ("r0", C.c_double),
        ("r_last", C.c_double),
        ("fn_table", C.c_void_p),
        ("spline_M", C.c_void_p),
    ]


def _load():
    """Load the oracle library: liboracle.so built from oracle.c, or the prebuilt library that
    the environment variable NAO_ORACLE_LIB names (the mutation tests load copies of oracle.c
    with one planted mistake each this way)."""
    global _lib
    if _lib is None:
        override = os.environ.get("NAO_ORACLE_LIB")
        lib = C.CDLL(override if override else str(build()))
        P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        lib.or_spline_M.argtypes = [P, I32, P]
        lib.or_spline_M.restype = C.c_int
        lib.or_radial.argtypes = [P, I32, D, P, P]
        lib.or_radial.restype = None
        lib.or_ylm.argtypes = [I32, D, D, D, P]
        lib.or_ylm.restype = C.c_int
        lib.or_n_basis.argtypes = [P]
        lib.or_n_basis.restype = I64
        lib.or_eval_dense.argtypes = [P, I64, P, P, P, P]
        lib.or_eval_dense.restype = C.c_int
        lib.or_hamiltonian.argtypes = [P, I64, P, P, P, C.c_uint32, P, P, P]
        lib.or_hamiltonian.restype = C.c_int
        lib.or_hamiltonian_tau.argtypes = [P, I64, P, P, P, P, C.c_uint32, P, P, P]
        lib.or_hamiltonian_tau.restype = C.c_int
        lib.or_hamiltonian_block.argtypes = [P, I64, P, P, P, C.c_uint32, I32, P, P, P, P]
        lib.or_hamiltonian_block.restype = C.c_int
        lib.or_density.argtypes = [P, I64, P, P, P, P, P, P, P]
        lib.or_density.restype = C.c_int
        lib.or_density_gradient.argtypes = [P, I64, P, P, P, P, P]
        lib.or_density_gradient.restype = C.c_int
        lib.or_radial2.argtypes = [P, I32, D, P, P, P]
        lib.or_radial2.restype = None
        lib.or_solid.argtypes = [I32, D, D, D, P, P, P]
        lib.or_solid.restype = C.c_int
        lib.or_eval_dense2.argtypes = [P, I64, P, P, P, P]
        lib.or_eval_dense2.restype = C.c_int
        lib.or_density_hessian.argtypes = [P, I64, P, P, P, P]
        lib.or_density_hessian.restype = C.c_int
        lib.or_pulay_matrices.argtypes = [P, I64, P, P, P, P, P, P, P]
        lib.or_pulay_matrices.restype = C.c_int
        lib.or_pulay_forces.argtypes = [P, I64, P, P, P, P, P, P]
        lib.or_pulay_forces.restype = C.c_int
        lib.or_periodic_h.argtypes = [P, P, I32, I64, P, P, P, P, C.c_uint32, P, P]
        lib.or_periodic_h.restype = C.c_int
        lib.or_bruteforce.argtypes = [P, I64, P, P, P, P, P, P, P]
        lib.or_bruteforce.restype = C.c_int
        lib.or_partition.argtypes = [I64, P, I64, P, P]
        lib.or_partition.restype = I64
        lib.or_relevance.argtypes = [P, P, I64, P, P, P, P]
        lib.or_relevance.restype = I64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st == -2:
        raise OracleError(f"{what}: a grid point coincides with a nucleus")
    if st == -3:
        raise OracleError(f"{what}: a grid point lies on an atom's polar axis")
    if st != 0:
        raise OracleError(f"{what}: status {st}")


TERM_POTENTIAL = 1
TERM_KINETIC = 2
TERM_TAU = 4  # meta-GGA: w vtau 1/2 grad phi_i . grad phi_j


class Oracle:
    """The oracle bound to one system (atoms, species radial tables)."""

    def __init__(self, sys):
        self.lib = _load()
        self._keep = {}
        k = self._keep
        k["atom_xyz"] = np.ascontiguousarray(sys.atom_xyz, dtype=np.float64)
        k["atom_species"] = np.ascontiguousarray(sys.atom_species, dtype=np.int32)
        k["species_fn_offset"] = np.ascontiguousarray(sys.species_fn_offset, dtype=np.int32)
        k["fn_l"] = np.ascontiguousarray(sys.fn_l, dtype=np.int32)
        k["fn_cutoff"] = np.ascontiguousarray(sys.fn_cutoff, dtype=np.float64)
        k["fn_table"] = np.ascontiguousarray(sys.fn_table, dtype=np.float64)
        n_fn, n_r = k["fn_table"].shape if k["fn_table"].ndim == 2 else (len(k["fn_l"]), int(sys.n_rgrid))
        k["fn_table"] = k["fn_table"].reshape(n_fn, int(sys.n_rgrid))
        M = np.zeros_like(k["fn_table"])
        for f in range(n_fn):
            st = self.lib.or_spline_M(k["fn_table"][f].ctypes.data, int(sys.n_rgrid), M[f].ctypes.data)
            if st:
                raise OracleError("spline")
        k["spline_M"] = M
        self.s = _Sys(
            int(k["atom_xyz"].shape[0]), _ptr(k["atom_xyz"]), _ptr(k["atom_species"]),
            int(len(k["species_fn_offset"]) - 1), _ptr(k["species_fn_offset"]), _ptr(k["fn_l"]),
            _ptr(k["fn_cutoff"]), int(sys.n_rgrid), float(sys.r0), float(sys.r_last), _ptr(k["fn_table"]),
            _ptr(k["spline_M"]),
        )
        self.sp = C.addressof(self.s)
        self.nb = int(self.lib.or_n_basis(self.sp))
        self.pole_count = C.c_int64(0)

    # -- radial / angular pieces ----------------------------------------------------------
    @property
    def spline_M(self) -> np.ndarray:
        return self._keep["spline_M"]

    def radial(self, f: int, r: float):
        R, dR = C.c_double(), C.c_double()
        self.lib.or_radial(self.sp, int(f), float(r), C.byref(R), C.byref(dR))
        return R.value, dR.value

    def radial2(self, f: int, r: float):
        """R_f(r), dR/dr, d^2R/dr^2."""
        R, dR, d2R = C.c_double(), C.c_double(), C.c_double()
        self.lib.or_radial2(self.sp, int(f), float(r), C.byref(R), C.byref(dR), C.byref(d2R))
        return R.value, dR.value, d2R.value

    @staticmethod
    def solid(l: int, x: float, y: float, z: float):
        """Real solid harmonics S_lm = r^l Y_lm (m = -l..l) from their monomial expansion, with
        gradients [2l+1, 3] and Hessians [2l+1, 6] (xx, xy, xz, yy, yz, zz)."""
        lib = _load()
        S = np.zeros(2 * l + 1)
        G = np.zeros((2 * l + 1, 3))
        Hs = np.zeros((2 * l + 1, 6))
        st = lib.or_solid(int(l), float(x), float(y), float(z), S.ctypes.data, G.ctypes.data, Hs.ctypes.data)
        if st != 0:
            raise OracleError(f"solid: status {st}")
        return S, G, Hs

    @staticmethod
    def ylm(l: int, x: float, y: float, z: float) -> np.ndarray:
        lib = _load()
        out = np.zeros(2 * l + 1)
        st = lib.or_ylm(int(l), float(x), float(y), float(z), out.ctypes.data)
        _check(st, "ylm")
        return out

    # -- basis functions ------------------------------------------------------------------
    def eval_dense(self, pts: np.ndarray):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        n = pts.shape[0]
        phi = np.zeros((n, self.nb))
        grad = np.zeros((n, self.nb, 3))
        _check(self.lib.or_eval_dense(self.sp, n, _ptr(pts), _ptr(phi), _ptr(grad), C.byref(self.pole_count)), "eval")
        return phi, grad

    def eval_dense2(self, pts: np.ndarray):
        """phi [n, nb], grad [n, nb, 3] and Hessian [n, nb, 6] through the Cartesian form."""
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        n = pts.shape[0]
        phi = np.zeros((n, self.nb))
        grad = np.zeros((n, self.nb, 3))
        hess = np.zeros((n, self.nb, 6))
        _check(self.lib.or_eval_dense2(self.sp, n, _ptr(pts), _ptr(phi), _ptr(grad), _ptr(hess)), "eval2")
        return phi, grad, hess

    # -- integrals ------------------------------------------------------------------------
    def hamiltonian(self, pts, w, v=None, terms=TERM_POTENTIAL | TERM_KINETIC):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, dtype=np.float64)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        H = np.zeros((self.nb, self.nb))
        A = np.zeros((self.nb, self.nb))
        st = self.lib.or_hamiltonian(self.sp, pts.shape[0], _ptr(pts), _ptr(w), _ptr(v), int(terms), _ptr(H), _ptr(A),
                                     C.byref(self.pole_count))
        _check(st, "hamiltonian")
        return H, A

    def hamiltonian_tau(self, pts, w, v, vtau, terms=TERM_POTENTIAL | TERM_KINETIC | TERM_TAU):
        """H with the meta-GGA term w vtau 1/2 grad phi_i . grad phi_j (terms bit 4)."""
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, dtype=np.float64)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        vtau = np.ascontiguousarray(vtau, dtype=np.float64)
        H = np.zeros((self.nb, self.nb))
        A = np.zeros((self.nb, self.nb))
        st = self.lib.or_hamiltonian_tau(self.sp, pts.shape[0], _ptr(pts), _ptr(w), _ptr(v), _ptr(vtau), int(terms),
                                         _ptr(H), _ptr(A), C.byref(self.pole_count))
        _check(st, "hamiltonian_tau")
        return H, A

    def hamiltonian_block(self, F, pts, w, v=None, terms=TERM_POTENTIAL | TERM_KINETIC):
        F = np.ascontiguousarray(F, dtype=np.int64)
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, dtype=np.float64)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        H = np.zeros((len(F), len(F)))
        A = np.zeros((len(F), len(F)))
        st = self.lib.or_hamiltonian_block(self.sp, pts.shape[0], _ptr(pts), _ptr(w), _ptr(v), int(terms), len(F),
                                           _ptr(F), _ptr(H), _ptr(A), C.byref(self.pole_count))
        _check(st, "hamiltonian_block")
        return H, A

    def overlap(self, pts, w):
        return self.hamiltonian(pts, w, None, TERM_POTENTIAL)

    def density(self, pts, P, w=None):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        P = np.ascontiguousarray(P, dtype=np.float64)
        assert P.shape == (self.nb, self.nb)
        w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        n = np.zeros(pts.shape[0])
        D = np.zeros(pts.shape[0])
        Ne = C.c_double(0.0)
        st = self.lib.or_density(self.sp, pts.shape[0], _ptr(pts), _ptr(w), _ptr(P), _ptr(n), _ptr(D), C.byref(Ne),
                                 C.byref(self.pole_count))
        _check(st, "density")
        return n, D, (Ne.value if w is not None else None)

    def density_gradient(self, pts, P):
        """grad n at each point ([n, 3]) and the magnitude sums 2 sum_ij |d_c phi_i P_ij phi_j| ([n, 3])."""
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        P = np.ascontiguousarray(P, dtype=np.float64)
        assert P.shape == (self.nb, self.nb)
        g = np.zeros((pts.shape[0], 3))
        Dg = np.zeros((pts.shape[0], 3))
        st = self.lib.or_density_gradient(self.sp, pts.shape[0], _ptr(pts), _ptr(P), _ptr(g), _ptr(Dg),
                                          C.byref(self.pole_count))
        _check(st, "density_gradient")
        return g, Dg

    def density_hessian(self, pts, P):
        """The density Hessian at each point ([n, 6]: xx, xy, xz, yy, yz, zz) and the magnitude sums
        of its four terms ([n, 6])."""
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        P = np.ascontiguousarray(P, dtype=np.float64)
        assert P.shape == (self.nb, self.nb)
        h = np.zeros((pts.shape[0], 6))
        Dh = np.zeros((pts.shape[0], 6))
        _check(self.lib.or_density_hessian(self.sp, pts.shape[0], _ptr(pts), _ptr(P), _ptr(h), _ptr(Dh)),
               "density_hessian")
        return h, Dh

    def pulay_matrices(self, pts, w, v=None):
        """M [3, nb, nb] (sum_p w d_c phi_i (-1/2 lap + v) phi_j), S [3, nb, nb] (sum_p w d_c phi_i phi_j)
        and their magnitude sums."""
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, dtype=np.float64)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        M = np.zeros((3, self.nb, self.nb)); S = np.zeros((3, self.nb, self.nb))
        AM = np.zeros((3, self.nb, self.nb)); AS = np.zeros((3, self.nb, self.nb))
        _check(self.lib.or_pulay_matrices(self.sp, pts.shape[0], _ptr(pts), _ptr(w), _ptr(v), _ptr(M), _ptr(S), _ptr(AM),
                                          _ptr(AS)), "pulay_matrices")
        return M, S, AM, AS

    def pulay_forces(self, pts, w, v, nmat, qmat):
        """Local Pulay forces [n_atoms, 3] point by point from their definition."""
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, dtype=np.float64)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        nmat = np.ascontiguousarray(nmat, dtype=np.float64); qmat = np.ascontiguousarray(qmat, dtype=np.float64)
        F = np.zeros((int(self._keep["atom_xyz"].shape[0]), 3))
        _check(self.lib.or_pulay_forces(self.sp, pts.shape[0], _ptr(pts), _ptr(w), _ptr(v), _ptr(nmat), _ptr(qmat),
                                        _ptr(F)), "pulay_forces")
        return F

    def periodic_h(self, lattice, nrange, pts, w, k, v=None, terms=TERM_POTENTIAL | TERM_KINETIC):
        """h(k) [nb, nb] complex of the unit cell described by this oracle's system (Bloch basis
        summed over the translations |n_c| <= nrange) and the magnitude sums [nb, nb]."""
        lattice = np.ascontiguousarray(lattice, dtype=np.float64).reshape(3, 3)
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, dtype=np.float64)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        k = np.ascontiguousarray(k, dtype=np.float64).reshape(3)
        H = np.zeros((self.nb, self.nb, 2))
        A = np.zeros((self.nb, self.nb))
        _check(self.lib.or_periodic_h(self.sp, _ptr(lattice), int(nrange), pts.shape[0], _ptr(pts), _ptr(w), _ptr(v),
                                      _ptr(k), int(terms), _ptr(H), _ptr(A)), "periodic_h")
        return H[..., 0] + 1j * H[..., 1], A

    def bruteforce(self, pts, w, v, P):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        P = np.ascontiguousarray(P, dtype=np.float64)
        H = np.zeros((self.nb, self.nb))
        n = np.zeros(pts.shape[0])
        st = self.lib.or_bruteforce(self.sp, pts.shape[0], _ptr(pts), _ptr(w), _ptr(v), _ptr(P), _ptr(H), _ptr(n),
                                    C.byref(self.pole_count))
        _check(st, "bruteforce")
        return H, n

    # -- partition and reduced basis --------------------------------------------------------
    @staticmethod
    def partition(pts, B: int):
        lib = _load()
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        n = pts.shape[0]
        kmax = (n + B - 1) // B
        offsets = np.zeros(kmax + 1, dtype=np.int64)
        perm = np.zeros(n, dtype=np.int64)
        nbat = lib.or_partition(n, _ptr(pts), int(B), _ptr(offsets), _ptr(perm))
        if nbat < 0:
            raise OracleError("partition")
        return offsets[: nbat + 1].copy(), perm

    def relevance(self, pts, offsets, perm):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        perm = np.ascontiguousarray(perm, dtype=np.int64)
        nbat = len(offsets) - 1
        rel_off = np.zeros(nbat + 1, dtype=np.int64)
        total = self.lib.or_relevance(self.sp, _ptr(pts), nbat, _ptr(offsets), _ptr(perm), _ptr(rel_off), None)
        rel = np.zeros(max(total, 1), dtype=np.int32)
        self.lib.or_relevance(self.sp, _ptr(pts), nbat, _ptr(offsets), _ptr(perm), _ptr(rel_off), _ptr(rel))
        return rel_off, rel[:total].copy()
