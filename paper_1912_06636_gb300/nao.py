"""Thin ctypes binding of libnao (include/nao.h): argument marshalling only.

Every numeric step runs in the CUDA library; this module only turns torch tensors into
device pointers and streams, numpy arrays into host pointers, and status codes into
exceptions. The functions keep the C names; ``Grid`` is a small owner object around a
handle. There is no fallback: if libnao.so is missing or cannot be loaded, importing the
library raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "lib" / "libnao.so"
_lib = None

NAO_FP64, NAO_FP32, NAO_SPLIT = 0, 1, 2
NAO_TERM_POTENTIAL, NAO_TERM_KINETIC, NAO_TERM_TAU = 1, 2, 4
NAO_OK, NAO_ERR_INVALID_ARG, NAO_ERR_OUT_OF_MEMORY, NAO_ERR_CUDA = 0, 1, 2, 3
NAO_ERR_TIMEOUT, NAO_ERR_INTERNAL, NAO_ERR_UNSUPPORTED = 4, 5, 6
PRECISIONS = {"fp64": NAO_FP64, "fp32": NAO_FP32, "split": NAO_SPLIT}

STATUS = {0: "NAO_OK", 1: "NAO_ERR_INVALID_ARG", 2: "NAO_ERR_OUT_OF_MEMORY", 3: "NAO_ERR_CUDA",
          4: "NAO_ERR_TIMEOUT", 5: "NAO_ERR_INTERNAL", 6: "NAO_ERR_UNSUPPORTED"}

# exported symbols declared in include/nao.h
SYMBOLS = [
    "nao_default_options", "nao_grid_create", "nao_destroy", "nao_get_info", "nao_export_batches",
    "nao_integrate_h", "nao_update_density", "nao_integrate_h_host", "nao_update_density_host",
    "nao_evaluate_batch", "nao_sync_status", "nao_status_string", "nao_last_error",
    "nao_profile_enable", "nao_profile_read", "nao_integrate_h_noalloc",
    "nao_grid_create_many", "nao_get_system", "nao_integrate_h_many", "nao_update_density_many",
    "nao_get_tuning", "nao_update_density_gradient", "nao_update_density_gradient_many",
    "nao_update_density_hessian", "nao_integrate_h_tau", "nao_pulay_matrices", "nao_pulay_forces",
    "nao_periodic_images", "nao_periodic_basis_map", "nao_bloch_sum", "nao_partition_points",
    "nao_radial_spline", "nao_fault_inject", "nao_check_wait_timeout",
]
NAO_NOALLOC_SCRATCH_BYTES = 32 << 20
KERNELS = ["eval_grad", "eval_phi", "h_fp64", "h_fp32", "h_split", "slice_h", "mirror", "n_fp64", "n_fp32",
           "n_split", "reduce", "slice_n"]


class NaoError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code


class SystemDesc(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int32), ("atom_xyz", C.c_void_p), ("atom_species", C.c_void_p),
        ("n_species", C.c_int32), ("species_fn_offset", C.c_void_p), ("fn_l", C.c_void_p),
        ("fn_cutoff", C.c_void_p), ("n_rgrid", C.c_int32), ("r0", C.c_double), ("r_last", C.c_double),
        ("fn_table", C.c_void_p), ("n_points", C.c_int64), ("pt_xyz", C.c_void_p), ("pt_w", C.c_void_p),
    ]


class Options(C.Structure):
    _fields_ = [
        ("max_batch_points", C.c_int32), ("split_slices", C.c_int32), ("deterministic", C.c_int32),
        ("device", C.c_int32), ("scratch_bytes", C.c_int64), ("capture_graph", C.c_int32),
        ("autotune", C.c_int32), ("split_digits", C.c_int32),
    ]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * 12), ("ms", C.c_double * 12)]


class GridInfo(C.Structure):
    _fields_ = [
        ("n_basis", C.c_int64), ("n_points", C.c_int64), ("n_batches", C.c_int64), ("rel_total", C.c_int64),
        ("max_batch_points", C.c_int32), ("max_batch_basis", C.c_int32), ("device_bytes", C.c_int64),
        ("flops_h", C.c_int64), ("flops_n", C.c_int64), ("n_systems", C.c_int32), ("n_atoms", C.c_int32),
    ]


def lib_path() -> Path:
    return _LIB_PATH


def load():
    """Load libnao.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise ImportError(f"libnao.so not built at {_LIB_PATH}; run __graft_entry__.build()")
    lib = C.CDLL(str(_LIB_PATH))
    P, I32, I64, U32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
    sig = {
        "nao_default_options": ([P], C.c_int),
        "nao_grid_create": ([P, P, P], C.c_int),
        "nao_destroy": ([P], C.c_int),
        "nao_get_info": ([P, P], C.c_int),
        "nao_export_batches": ([P, P, P, P, P], C.c_int),
        "nao_integrate_h": ([P, P, U32, C.c_int, P, P], C.c_int),
        "nao_update_density": ([P, P, C.c_int, P, P, P], C.c_int),
        "nao_integrate_h_host": ([P, P, U32, C.c_int, P, P], C.c_int),
        "nao_update_density_host": ([P, P, C.c_int, P, P, P], C.c_int),
        "nao_evaluate_batch": ([P, I64, C.c_int, P, P, P], C.c_int),
        "nao_sync_status": ([P], C.c_int),
        "nao_status_string": ([C.c_int], C.c_char_p),
        "nao_last_error": ([], C.c_char_p),
        "nao_profile_enable": ([P, I32], C.c_int),
        "nao_profile_read": ([P, P, I32], C.c_int),
        "nao_integrate_h_noalloc": ([P, P, U32, P, P], C.c_int),
        "nao_grid_create_many": ([P, I32, P, P, P], C.c_int),
        "nao_get_system": ([P, I32, P, P, P, P, P, P], C.c_int),
        "nao_integrate_h_many": ([P, P, U32, C.c_int, P, P], C.c_int),
        "nao_update_density_many": ([P, P, C.c_int, P, P, P], C.c_int),
        "nao_get_tuning": ([P, P, P], C.c_int),
        "nao_update_density_gradient": ([P, P, C.c_int, P, P, P, P], C.c_int),
        "nao_update_density_hessian": ([P, P, C.c_int, P, P, P, P, P], C.c_int),
        "nao_integrate_h_tau": ([P, P, P, C.c_uint32, C.c_int, P, P], C.c_int),
        "nao_pulay_matrices": ([P, P, C.c_int, P, P, P], C.c_int),
        "nao_pulay_forces": ([P, P, P, P, P, P, P], C.c_int),
        "nao_update_density_gradient_many": ([P, P, C.c_int, P, P, P, P], C.c_int),
        "nao_periodic_images": ([P, I32, P, C.c_double, I32, P, P, P, P], C.c_int),
        "nao_periodic_basis_map": ([P, I32, P, I32, P, P, I32, I64, P, P, P], C.c_int),
        "nao_bloch_sum": ([P, I64, P, P, P, I32, P, P, I32, I64, P, P, P], C.c_int),
        "nao_partition_points": ([P, I64, I64, I64, P, P, P], C.c_int),
        "nao_radial_spline": ([P, I32, P], C.c_int),
        "nao_fault_inject": ([C.c_char_p], C.c_int),
        "nao_check_wait_timeout": ([P, I64, P], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != 0:
        msg = load().nao_last_error().decode(errors="replace")
        raise NaoError(code, where, msg)


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _dptr(t) -> int | None:
    """Device pointer of a CUDA tensor (None stays None)."""
    if t is None:
        return None
    import torch

    if not t.is_cuda or not t.is_contiguous() or t.dtype != torch.float64:
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _count(t) -> int:
    return int(t.numel()) if hasattr(t, "numel") else int(np.size(t))


def _need(t, n: int, what: str) -> None:
    """A caller's buffer (tensor or array; None is checked by the library) must hold n elements:
    the C ABI cannot see the size of a device buffer, so the binding checks it before the call."""
    if t is not None and _count(t) < n:
        raise ValueError(f"{what}: needs {n} elements, the buffer holds {_count(t)}")


def _handle_sizes(h):
    """(n_basis, n_points, [(n_basis_m, n_points_m) per system], n_atoms) of a handle, queried from
    the library (host-side queries) and kept on the handle object itself when it can hold them, so
    that no size outlives its handle."""
    got = getattr(h, "_nao_sizes", None)
    if got is None:
        info = nao_get_info(h)
        per = []
        for m in range(int(info.n_systems)):
            sysm = nao_get_system(h, m)
            per.append((sysm["n_basis"], sysm["n_points"]))
        got = (int(info.n_basis), int(info.n_points), per, int(info.n_atoms))
        try:
            h._nao_sizes = got
        except AttributeError:  # a plain integer address: queried again on every call
            pass
    return got


def _sizes(h):
    """(n_basis, n_points) of a handle (for a grouped handle, the totals)."""
    nb, npts, _, _ = _handle_sizes(h)
    return nb, npts


def _need_each(h, ts, per_system, what: str) -> None:
    """Per-system buffers of a grouped call: one entry per system (the library reads that many
    pointers), ts[m] holding per_system(n_basis_m, n_points_m) elements."""
    if ts is None:
        return
    per = _handle_sizes(h)[2]
    if len(ts) != len(per):
        raise ValueError(f"{what}: {len(per)} entries required (one per system), got {len(ts)}")
    for m, (t, (nb_m, np_m)) in enumerate(zip(ts, per)):
        _need(t, per_system(nb_m, np_m), f"{what}[{m}]")


# ---- C-named functions --------------------------------------------------------------------
def nao_default_options() -> Options:
    o = Options()
    _check(load().nao_default_options(C.byref(o)), "nao_default_options")
    return o


def _desc(system, keep: list) -> SystemDesc:
    """nao_system_desc of a system (any object with its fields); arrays kept alive in keep."""
    a = {
        "atom_xyz": np.ascontiguousarray(system.atom_xyz, dtype=np.float64),
        "atom_species": np.ascontiguousarray(system.atom_species, dtype=np.int32),
        "species_fn_offset": np.ascontiguousarray(system.species_fn_offset, dtype=np.int32),
        "fn_l": np.ascontiguousarray(system.fn_l, dtype=np.int32),
        "fn_cutoff": np.ascontiguousarray(system.fn_cutoff, dtype=np.float64),
        "fn_table": np.ascontiguousarray(system.fn_table, dtype=np.float64),
        "pt_xyz": np.ascontiguousarray(system.pt_xyz, dtype=np.float64),
        "pt_w": np.ascontiguousarray(system.pt_w, dtype=np.float64),
    }
    keep.append(a)
    return SystemDesc(
        int(a["atom_xyz"].size // 3), a["atom_xyz"].ctypes.data, a["atom_species"].ctypes.data,
        int(a["species_fn_offset"].size - 1), a["species_fn_offset"].ctypes.data, a["fn_l"].ctypes.data,
        a["fn_cutoff"].ctypes.data, int(system.n_rgrid), float(system.r0), float(system.r_last),
        a["fn_table"].ctypes.data, int(a["pt_w"].size), a["pt_xyz"].ctypes.data, a["pt_w"].ctypes.data,
    )


def _options(options: Options | None, opts: dict) -> Options:
    o = options if options is not None else nao_default_options()
    for k, v in opts.items():
        setattr(o, k, v)
    return o


def nao_grid_create(system, options: Options | None = None, **opts) -> C.c_void_p:
    """Create a handle from a system (any object with the fields of nao_system_desc)."""
    keep: list = []
    d = _desc(system, keep)
    o = _options(options, opts)
    h = C.c_void_p()
    _check(load().nao_grid_create(C.byref(d), C.byref(o), C.byref(h)), "nao_grid_create")
    return h


def nao_grid_create_many(systems, options: Options | None = None, batch_points=None, **opts) -> C.c_void_p:
    """One handle over several systems that share the radial grid (optional per-system B)."""
    keep: list = []
    arr = (SystemDesc * len(systems))(*[_desc(s, keep) for s in systems])
    bp = None if batch_points is None else np.ascontiguousarray(batch_points, dtype=np.int32)
    o = _options(options, opts)
    h = C.c_void_p()
    _check(load().nao_grid_create_many(arr, len(systems), None if bp is None else bp.ctypes.data, C.byref(o),
                                       C.byref(h)), "nao_grid_create_many")
    return h


def nao_get_system(h, m: int) -> dict:
    v = [C.c_int64() for _ in range(6)]
    _check(load().nao_get_system(h, int(m), *[C.byref(x) for x in v]), "nao_get_system")
    keys = ("basis_offset", "n_basis", "point_offset", "n_points", "batch_begin", "batch_end")
    return {k: int(x.value) for k, x in zip(keys, v)}


def nao_get_tuning(h):
    """(per-batch split tile width, number of histogram buckets the autotuner timed)."""
    info = nao_get_info(h)
    tw = np.zeros(max(int(info.n_batches), 1), np.int32)
    nb = C.c_int32()
    _check(load().nao_get_tuning(h, tw.ctypes.data, C.byref(nb)), "nao_get_tuning")
    return tw[: int(info.n_batches)], int(nb.value)


def _ptr_array(ts, allow_none: bool):
    """Host array of device pointers (None entries allowed where the call allows them)."""
    if ts is None:
        return None
    vals = []
    for t in ts:
        if t is None and not allow_none:
            raise ValueError("a required tensor is None")
        vals.append(_dptr(t))
    return (C.c_void_p * len(vals))(*vals)


def nao_destroy(h) -> None:
    if getattr(h, "_nao_sizes", None) is not None:
        h._nao_sizes = None
    _check(load().nao_destroy(h), "nao_destroy")


def nao_get_info(h) -> GridInfo:
    info = GridInfo()
    _check(load().nao_get_info(h, C.byref(info)), "nao_get_info")
    return info


def nao_export_batches(h):
    info = nao_get_info(h)
    bo = np.zeros(info.n_batches + 1, np.int64)
    pp = np.zeros(info.n_points, np.int64)
    ro = np.zeros(info.n_batches + 1, np.int64)
    ri = np.zeros(max(info.rel_total, 1), np.int32)
    _check(load().nao_export_batches(h, bo.ctypes.data, pp.ctypes.data, ro.ctypes.data, ri.ctypes.data),
           "nao_export_batches")
    return bo, pp, ro, ri[: info.rel_total]


def nao_integrate_h(h, v, terms: int, prec, H, stream=None) -> None:
    nb, npts = _sizes(h)
    _need(v, npts, "v")
    _need(H, nb * nb, "H")
    _check(load().nao_integrate_h(h, _dptr(v), int(terms), _prec(prec), _dptr(H), _stream(stream)), "nao_integrate_h")


def nao_integrate_h_tau(h, v, vtau, terms: int, prec, H, stream=None) -> None:
    nb, npts = _sizes(h)
    _need(v, npts, "v")
    _need(vtau, npts, "vtau")
    _need(H, nb * nb, "H")
    _check(load().nao_integrate_h_tau(h, _dptr(v), _dptr(vtau), int(terms), _prec(prec), _dptr(H), _stream(stream)),
           "nao_integrate_h_tau")


def nao_pulay_matrices(h, v, prec, M, S, stream=None) -> None:
    nb, npts = _sizes(h)
    _need(v, npts, "v")
    _need(M, 3 * nb * nb, "M")
    _need(S, 3 * nb * nb, "S")
    _check(load().nao_pulay_matrices(h, _dptr(v), _prec(prec), _dptr(M), _dptr(S), _stream(stream)),
           "nao_pulay_matrices")


def nao_pulay_forces(h, n, q, M, S, F, stream=None) -> None:
    nb, _, _, n_atoms = _handle_sizes(h)
    for t, k, what in ((n, 1, "n"), (q, 1, "q"), (M, 3, "M"), (S, 3, "S")):
        _need(t, k * nb * nb, what)
    _need(F, 3 * n_atoms, "F")
    _check(load().nao_pulay_forces(h, _dptr(n), _dptr(q), _dptr(M), _dptr(S), _dptr(F), _stream(stream)),
           "nao_pulay_forces")


def nao_fault_inject(spec: str | None) -> None:
    """Make the n-th device allocation, copy or launch of the library fail once ("alloc:<n>",
    "copy:<n>", "launch:<n>"); None or "" clears it (host-side; no GPU fault is involved)."""
    _check(load().nao_fault_inject(None if spec is None else spec.encode()), "nao_fault_inject")


def nao_check_wait_timeout(h, max_cycles: int, stream=None) -> None:
    """Enqueue one bounded device wait that runs out after max_cycles SM cycles and records
    NAO_ERR_TIMEOUT for nao_sync_status to report."""
    _check(load().nao_check_wait_timeout(h, int(max_cycles), _stream(stream)), "nao_check_wait_timeout")


def nao_partition_points(pt_xyz, max_batch_points: int):
    """The batch partition of the points (host, no GPU): (batch_offsets [n_batches + 1],
    point_perm [n_points]), int64."""
    lib = load()
    x = np.ascontiguousarray(pt_xyz, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    B = int(max_batch_points)
    max_b = -(-n // B) if B > 0 else 0
    off = np.zeros(max_b + 1, np.int64)
    perm = np.zeros(max(n, 1), np.int64)
    nbat = C.c_int64(0)
    _check(lib.nao_partition_points(x.ctypes.data, n, B, max_b, off.ctypes.data, perm.ctypes.data, C.byref(nbat)),
           "nao_partition_points")
    return off[: nbat.value + 1], perm[:n]


def nao_radial_spline(fn_table):
    """Cubic coefficients [(n_rgrid - 1), 4] of the natural spline through one radial table (host)."""
    lib = load()
    y = np.ascontiguousarray(fn_table, dtype=np.float64).reshape(-1)
    coef = np.zeros((max(y.size - 1, 1), 4))
    _check(lib.nao_radial_spline(y.ctypes.data, y.size, coef.ctypes.data), "nao_radial_spline")
    return coef


def nao_periodic_images(atom_xyz, lattice, reach: float):
    """Periodic images of the cell's atoms that can reach the cell (host): (xyz [n, 3], unit-cell
    atom [n], cell [n, 3]), the atoms themselves first."""
    lib = load()
    x = np.ascontiguousarray(atom_xyz, dtype=np.float64).reshape(-1, 3)
    A = np.ascontiguousarray(lattice, dtype=np.float64).reshape(9)
    n = C.c_int32(0)
    lib.nao_periodic_images(x.ctypes.data, x.shape[0], A.ctypes.data, float(reach), 0, None, None, None, C.byref(n))
    xyz = np.zeros((max(n.value, 1), 3))
    atom = np.zeros(max(n.value, 1), dtype=np.int32)
    cell = np.zeros((max(n.value, 1), 3), dtype=np.int32)
    _check(lib.nao_periodic_images(x.ctypes.data, x.shape[0], A.ctypes.data, float(reach), n.value, xyz.ctypes.data,
                                   atom.ctypes.data, cell.ctypes.data, C.byref(n)), "nao_periodic_images")
    return xyz[:n.value], atom[:n.value], cell[:n.value]


def nao_periodic_basis_map(system, img_atom):
    """(fn_map, fn_image) of the image system's N_rs functions (host int32 arrays)."""
    lib = load()
    sp = np.ascontiguousarray(system.atom_species, dtype=np.int32)
    off = np.ascontiguousarray(system.species_fn_offset, dtype=np.int32)
    fl = np.ascontiguousarray(system.fn_l, dtype=np.int32)
    ia = np.ascontiguousarray(img_atom, dtype=np.int32)
    n = C.c_int64(0)
    lib.nao_periodic_basis_map(sp.ctypes.data, len(sp), off.ctypes.data, len(off) - 1, fl.ctypes.data, ia.ctypes.data,
                               len(ia), 0, None, None, C.byref(n))
    fm = np.zeros(max(n.value, 1), dtype=np.int32)
    fi = np.zeros(max(n.value, 1), dtype=np.int32)
    _check(lib.nao_periodic_basis_map(sp.ctypes.data, len(sp), off.ctypes.data, len(off) - 1, fl.ctypes.data,
                                      ia.ctypes.data, len(ia), n.value, fm.ctypes.data, fi.ctypes.data, C.byref(n)),
           "nao_periodic_basis_map")
    return fm[:n.value], fi[:n.value]


def check_bloch_maps(fn_map, fn_image, img_cell, nb: int) -> int:
    """The Bloch sum's index arrays against the sizes they index (tensors on any device; a
    device tensor costs one synchronising read of its extremes): every fn_map entry in [0, nb),
    every fn_image entry in [0, n_images) with n_images = img_cell's length / 3. Returns n_images."""
    if img_cell.numel() % 3 != 0 or img_cell.numel() == 0:
        raise ValueError("img_cell must hold 3 integers per image")
    n_images = int(img_cell.numel() // 3)
    if fn_map.numel() and (int(fn_map.min()) < 0 or int(fn_map.max()) >= nb):
        raise ValueError(f"fn_map entries must lie in [0, {nb})")
    if fn_image.numel() and (int(fn_image.min()) < 0 or int(fn_image.max()) >= n_images):
        raise ValueError(f"fn_image entries must lie in [0, {n_images})")
    return n_images


def nao_bloch_sum(h_uc, fn_map, fn_image, img_cell, lattice, kpts, nb: int, stream=None, out=None, err=None):
    """h(k) [n_k, nb, nb] complex from h^uc [n_rs, n_rs] (CUDA tensors; the index arrays int32).
    out: optional FP64 CUDA tensor [n_k, nb, nb, 2] to write into. err: optional int32 CUDA
    tensor of one element that receives the kernel's count of skipped out-of-range map entries
    (0 after a valid call; the maps are also checked here before the call)."""
    import torch

    A = np.ascontiguousarray(lattice, dtype=np.float64).reshape(9)
    k = kpts.contiguous()
    hk = out if out is not None else torch.empty((k.shape[0], nb, nb, 2), dtype=torch.float64, device=h_uc.device)
    if hk.dtype != torch.float64 or tuple(hk.shape) != (k.shape[0], nb, nb, 2) or not hk.is_contiguous():
        raise ValueError("out must be a contiguous float64 tensor [n_k, nb, nb, 2]")
    for t in (fn_map, fn_image, img_cell):
        if not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous():
            raise ValueError("index arrays must be contiguous int32 CUDA tensors")
    n_rs = int(h_uc.shape[0])
    if h_uc.dim() != 2 or int(h_uc.shape[1]) != n_rs:
        raise ValueError("h_uc must be a square [n_rs, n_rs] tensor")
    _need(fn_map, n_rs, "fn_map")
    _need(fn_image, n_rs, "fn_image")
    if k.dim() != 2 or int(k.shape[1]) != 3:
        raise ValueError("kpts must be [n_k, 3]")
    n_images = check_bloch_maps(fn_map[:n_rs], fn_image[:n_rs], img_cell, int(nb))
    if err is not None and (not err.is_cuda or err.dtype != torch.int32 or err.numel() < 1):
        raise ValueError("err must be an int32 CUDA tensor of at least one element")
    _check(load().nao_bloch_sum(_dptr(h_uc), h_uc.shape[0], fn_map.data_ptr(), fn_image.data_ptr(), img_cell.data_ptr(),
                                n_images, A.ctypes.data, _dptr(k), k.shape[0], int(nb), _dptr(hk),
                                None if err is None else err.data_ptr(), _stream(stream)), "nao_bloch_sum")
    return torch.view_as_complex(hk)


def nao_update_density(h, P, prec, n, ne=None, stream=None) -> None:
    nb, npts = _sizes(h)
    _need(P, nb * nb, "P")
    _need(n, npts, "n")
    _need(ne, 1, "ne")
    _check(load().nao_update_density(h, _dptr(P), _prec(prec), _dptr(n), _dptr(ne), _stream(stream)),
           "nao_update_density")


def nao_integrate_h_many(h, vs, terms: int, prec, Hs, stream=None) -> None:
    _need_each(h, vs, lambda nb, npts: npts, "vs")
    _need_each(h, Hs, lambda nb, npts: nb * nb, "Hs")
    _check(load().nao_integrate_h_many(h, _ptr_array(vs, True), int(terms), _prec(prec), _ptr_array(Hs, False),
                                       _stream(stream)), "nao_integrate_h_many")


def nao_update_density_many(h, Ps, prec, ns, nes=None, stream=None) -> None:
    _need_each(h, Ps, lambda nb, npts: nb * nb, "Ps")
    _need_each(h, ns, lambda nb, npts: npts, "ns")
    _need_each(h, nes, lambda nb, npts: 1, "nes")
    _check(load().nao_update_density_many(h, _ptr_array(Ps, False), _prec(prec), _ptr_array(ns, False),
                                          _ptr_array(nes, True), _stream(stream)), "nao_update_density_many")


def nao_update_density_gradient(h, P, prec, n, grad, ne=None, stream=None) -> None:
    nb, npts = _sizes(h)
    _need(P, nb * nb, "P")
    _need(n, npts, "n")
    _need(grad, 3 * npts, "grad")
    _need(ne, 1, "ne")
    _check(load().nao_update_density_gradient(h, _dptr(P), _prec(prec), _dptr(n), _dptr(grad), _dptr(ne),
                                              _stream(stream)), "nao_update_density_gradient")


def nao_update_density_hessian(h, P, prec, n, grad, hess, ne=None, stream=None) -> None:
    nb, npts = _sizes(h)
    _need(P, nb * nb, "P")
    _need(n, npts, "n")
    _need(grad, 3 * npts, "grad")
    _need(hess, 6 * npts, "hess")
    _need(ne, 1, "ne")
    _check(load().nao_update_density_hessian(h, _dptr(P), _prec(prec), _dptr(n), _dptr(grad), _dptr(hess), _dptr(ne),
                                             _stream(stream)), "nao_update_density_hessian")


def nao_update_density_gradient_many(h, Ps, prec, ns, grads, nes=None, stream=None) -> None:
    _need_each(h, Ps, lambda nb, npts: nb * nb, "Ps")
    _need_each(h, ns, lambda nb, npts: npts, "ns")
    _need_each(h, grads, lambda nb, npts: 3 * npts, "grads")
    _need_each(h, nes, lambda nb, npts: 1, "nes")
    _check(load().nao_update_density_gradient_many(h, _ptr_array(Ps, False), _prec(prec), _ptr_array(ns, False),
                                                   _ptr_array(grads, False), _ptr_array(nes, True), _stream(stream)),
           "nao_update_density_gradient_many")


def nao_integrate_h_host(h, v: np.ndarray | None, terms: int, prec, H: np.ndarray, stream=None) -> None:
    nb, npts = _sizes(h)
    v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    _need(v, npts, "v")
    _need(H, nb * nb, "H")
    vp = None if v is None else v.ctypes.data
    assert H.dtype == np.float64 and H.flags.c_contiguous
    _check(load().nao_integrate_h_host(h, vp, int(terms), _prec(prec), H.ctypes.data, _stream(stream)),
           "nao_integrate_h_host")


def nao_update_density_host(h, P: np.ndarray, prec, n: np.ndarray, stream=None) -> float:
    nb, npts = _sizes(h)
    P = np.ascontiguousarray(P, dtype=np.float64)
    _need(P, nb * nb, "P")
    _need(n, npts, "n")
    assert n.dtype == np.float64 and n.flags.c_contiguous
    ne = C.c_double(0.0)
    _check(load().nao_update_density_host(h, P.ctypes.data, _prec(prec), n.ctypes.data, C.byref(ne), _stream(stream)),
           "nao_update_density_host")
    return ne.value


def nao_evaluate_batch(h, batch: int, prec, phi, grad=None, stream=None) -> None:
    _check(load().nao_evaluate_batch(h, int(batch), _prec(prec), _dptr(phi), _dptr(grad), _stream(stream)),
           "nao_evaluate_batch")


def nao_sync_status(h) -> None:
    _check(load().nao_sync_status(h), "nao_sync_status")


def nao_integrate_h_noalloc(h, v, terms: int, H, stream=None) -> None:
    """FP64 Hamiltonian with the library's fixed device scratch (no allocation of any kind)."""
    nb, npts = _sizes(h)
    _need(v, npts, "v")
    _need(H, nb * nb, "H")
    _check(load().nao_integrate_h_noalloc(h, _dptr(v), int(terms), _dptr(H), _stream(stream)),
           "nao_integrate_h_noalloc")


def nao_profile_enable(h, enable: bool = True) -> None:
    _check(load().nao_profile_enable(h, 1 if enable else 0), "nao_profile_enable")


def nao_profile_read(h, reset: bool = True) -> dict:
    p = Profile()
    _check(load().nao_profile_read(h, C.byref(p), 1 if reset else 0), "nao_profile_read")
    return {k: (int(p.launches[i]), float(p.ms[i])) for i, k in enumerate(KERNELS)}


def nao_status_string(code: int) -> str:
    return load().nao_status_string(int(code)).decode()


# ---- owner object -------------------------------------------------------------------------
@dataclass
class _Sizes:
    nb: int
    n_points: int
    n_batches: int


class Grid:
    """Owns one nao_grid handle; allocates outputs as torch tensors on the handle's device.

    ``system`` is one system, or a list of systems for a grouped handle (nao_grid_create_many);
    the grouped handle's per-system calls are integrate_h_many / update_density_many."""

    def __init__(self, system, device: int | None = None, batch_points=None, **opts):
        import torch

        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", device)
        with torch.cuda.device(self.device):
            if isinstance(system, (list, tuple)):
                self.h = nao_grid_create_many(list(system), batch_points=batch_points, device=device, **opts)
            else:
                self.h = nao_grid_create(system, device=device, **opts)
        self.info = nao_get_info(self.h)
        self.split_slices = int(opts.get("split_slices", nao_default_options().split_slices))
        self.split_digits = int(opts.get("split_digits", 0))
        self.nb = int(self.info.n_basis)
        self.n_points = int(self.info.n_points)
        self.n_systems = int(self.info.n_systems)
        self.systems = [nao_get_system(self.h, m) for m in range(self.n_systems)]
        sys_list = list(system) if isinstance(system, (list, tuple)) else [system]
        self.n_atoms = sum(len(np.asarray(sy.atom_xyz).reshape(-1, 3)) for sy in sys_list)

    def close(self):
        if getattr(self, "h", None):
            nao_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def integrate_h(self, v=None, terms=NAO_TERM_POTENTIAL | NAO_TERM_KINETIC, prec="fp64", H=None, stream=None):
        import torch

        if H is None:
            H = torch.empty((self.nb, self.nb), dtype=torch.float64, device=self.device)
        nao_integrate_h(self.h, v, terms, prec, H, stream)
        return H

    def integrate_h_tau(self, v, vtau, terms=NAO_TERM_POTENTIAL | NAO_TERM_KINETIC | NAO_TERM_TAU, prec="fp64", H=None,
                        stream=None):
        """H with the meta-GGA term sum_p w_p vtau_p 1/2 grad phi_i . grad phi_j (single system)."""
        import torch

        if H is None:
            H = torch.empty((self.nb, self.nb), dtype=torch.float64, device=self.device)
        nao_integrate_h_tau(self.h, v, vtau, terms, prec, H, stream)
        return H

    def pulay_matrices(self, v=None, prec="fp64", M=None, S=None, stream=None):
        """M [3, nb, nb] = sum_p w d_c phi_i (-1/2 lap + v) phi_j and S [3, nb, nb] = sum_p w d_c phi_i phi_j."""
        import torch

        if M is None:
            M = torch.empty((3, self.nb, self.nb), dtype=torch.float64, device=self.device)
        if S is None:
            S = torch.empty((3, self.nb, self.nb), dtype=torch.float64, device=self.device)
        nao_pulay_matrices(self.h, v, prec, M, S, stream)
        return M, S

    def pulay_forces(self, n, q, M, S, F=None, stream=None):
        """Local Pulay forces [n_atoms, 3] from the matrix elements and the (energy-weighted) density matrices."""
        import torch

        if F is None:
            F = torch.empty((self.n_atoms, 3), dtype=torch.float64, device=self.device)
        nao_pulay_forces(self.h, n, q, M, S, F, stream)
        return F

    def overlap(self, prec="fp64", S=None, stream=None):
        return self.integrate_h(None, NAO_TERM_POTENTIAL, prec, S, stream)

    def update_density(self, P, prec="fp64", n=None, ne=None, stream=None, want_ne=True):
        import torch

        if n is None:
            n = torch.empty(self.n_points, dtype=torch.float64, device=self.device)
        if ne is None and want_ne:
            ne = torch.empty(1, dtype=torch.float64, device=self.device)
        nao_update_density(self.h, P, prec, n, ne, stream)
        return n, ne

    def integrate_h_many(self, vs=None, terms=NAO_TERM_POTENTIAL | NAO_TERM_KINETIC, prec="fp64", Hs=None,
                         stream=None):
        import torch

        if Hs is None:
            Hs = [torch.empty((s["n_basis"], s["n_basis"]), dtype=torch.float64, device=self.device)
                  for s in self.systems]
        nao_integrate_h_many(self.h, vs, terms, prec, Hs, stream)
        return Hs

    def update_density_many(self, Ps, prec="fp64", ns=None, nes=None, stream=None, want_ne=True):
        import torch

        if ns is None:
            ns = [torch.empty(s["n_points"], dtype=torch.float64, device=self.device) for s in self.systems]
        if nes is None and want_ne:
            nes = [torch.empty(1, dtype=torch.float64, device=self.device) for _ in self.systems]
        nao_update_density_many(self.h, Ps, prec, ns, nes, stream)
        return ns, nes

    def density_gradient(self, P, prec="fp64", n=None, grad=None, ne=None, stream=None, want_ne=True):
        """n, grad n ([3, n_points]) and N_e of a single-system handle."""
        import torch

        if n is None:
            n = torch.empty(self.n_points, dtype=torch.float64, device=self.device)
        if grad is None:
            grad = torch.empty((3, self.n_points), dtype=torch.float64, device=self.device)
        if ne is None and want_ne:
            ne = torch.empty(1, dtype=torch.float64, device=self.device)
        nao_update_density_gradient(self.h, P, prec, n, grad, ne, stream)
        return n, grad, ne

    def density_hessian(self, P, prec="fp64", n=None, grad=None, hess=None, ne=None, stream=None, want_ne=True):
        """n, grad n ([3, n_points]), the density Hessian ([6, n_points]: xx, xy, xz, yy, yz, zz)
        and N_e of a single-system handle ("fp64", "fp32" or "split")."""
        import torch

        if n is None:
            n = torch.empty(self.n_points, dtype=torch.float64, device=self.device)
        if grad is None:
            grad = torch.empty((3, self.n_points), dtype=torch.float64, device=self.device)
        if hess is None:
            hess = torch.empty((6, self.n_points), dtype=torch.float64, device=self.device)
        if ne is None and want_ne:
            ne = torch.empty(1, dtype=torch.float64, device=self.device)
        nao_update_density_hessian(self.h, P, prec, n, grad, hess, ne, stream)
        return n, grad, hess, ne

    def density_gradient_many(self, Ps, prec="fp64", stream=None):
        import torch

        ns = [torch.empty(s["n_points"], dtype=torch.float64, device=self.device) for s in self.systems]
        gs = [torch.empty((3, s["n_points"]), dtype=torch.float64, device=self.device) for s in self.systems]
        nes = [torch.empty(1, dtype=torch.float64, device=self.device) for _ in self.systems]
        nao_update_density_gradient_many(self.h, Ps, prec, ns, gs, nes, stream)
        return ns, gs, nes

    def evaluate_batch(self, b: int, prec="fp64", grad=True, stream=None):
        import torch

        bo, _, ro, _ = self.batches()
        P, N = int(bo[b + 1] - bo[b]), int(ro[b + 1] - ro[b])
        phi = torch.zeros((N, P), dtype=torch.float64, device=self.device)
        g = torch.zeros((3, N, P), dtype=torch.float64, device=self.device) if grad else None
        nao_evaluate_batch(self.h, b, prec, phi, g, stream)
        return phi, g

    def batches(self):
        if not hasattr(self, "_batches"):
            self._batches = nao_export_batches(self.h)
        return self._batches

    def sync(self):
        nao_sync_status(self.h)
