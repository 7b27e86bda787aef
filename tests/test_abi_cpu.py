"""The C-ABI library loads, exports every symbol include/nao.h declares, and rejects bad
input before touching a GPU (these tests make no compute call)."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

from paper_1912_06636_gb300 import nao, synth

HEADER = Path(__file__).resolve().parents[1] / "include" / "nao.h"


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nao_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = nao.load()
    decl = declared_functions()
    assert len(decl) >= 13
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(nao.SYMBOLS) == sorted(set(nao.SYMBOLS) & set(decl))


def test_status_strings_and_defaults():
    assert nao.nao_status_string(0) == "ok"
    assert nao.nao_status_string(1) == "invalid argument"
    o = nao.nao_default_options()
    assert o.max_batch_points == 200 and o.split_slices == 12 and o.device == -1
    assert o.capture_graph == 0 and o.autotune == 1


def _bad(sys_, **opts):
    with pytest.raises(nao.NaoError) as e:
        nao.nao_grid_create(sys_, **opts)
    return e.value.code


def test_invalid_input_is_rejected_without_gpu():
    s = synth.config_water(n_rad=4, n_theta=2, n_phi=3)
    bad = synth.System(**{**s.__dict__})
    bad.fn_l = s.fn_l.copy()
    bad.fn_l[0] = 7
    assert _bad(bad) == 1
    bad = synth.System(**{**s.__dict__})
    bad.fn_cutoff = s.fn_cutoff.copy()
    bad.fn_cutoff[1] = 9.0  # beyond r_last
    assert _bad(bad) == 1
    bad = synth.System(**{**s.__dict__})
    bad.pt_xyz = s.pt_xyz.copy()
    bad.pt_xyz[3, 1] = np.nan
    assert _bad(bad) == 1
    bad = synth.System(**{**s.__dict__})
    bad.atom_species = np.array([0, 1, 5], np.int32)
    assert _bad(bad) == 1
    assert _bad(s, max_batch_points=0) == 1
    assert _bad(s, max_batch_points=5000) == 1
    assert _bad(s, split_slices=2) == 1
    assert _bad(s, split_slices=13) == 1
    assert _bad(s, capture_graph=2) == 1
    assert _bad(s, autotune=2) == 1


def test_grouped_create_rejects_bad_input_without_gpu():
    s = synth.config_water(n_rad=4, n_theta=2, n_phi=3)
    bad = synth.System(**{**s.__dict__})
    bad.fn_l = s.fn_l.copy()
    bad.fn_l[0] = 7
    with pytest.raises(nao.NaoError) as e:
        nao.nao_grid_create_many([s, bad])
    assert e.value.code == 1 and "system 1" in str(e.value)
    lib = nao.load()
    out = C.c_void_p(123)
    assert lib.nao_grid_create_many(None, 2, None, None, C.byref(out)) == 1 and out.value is None
    arr = (nao.SystemDesc * 1)()
    assert lib.nao_grid_create_many(arr, 0, None, None, C.byref(out)) == 1
    with pytest.raises(nao.NaoError) as e:
        nao.nao_grid_create_many([s, s], batch_points=[200, 0])
    assert e.value.code == 1 and "max_batch_points[1]" in str(e.value)


def test_null_handle_calls_fail_cleanly():
    lib = nao.load()
    assert lib.nao_destroy(None) == 0
    assert lib.nao_integrate_h(None, None, 3, 0, None, None) == 1
    assert lib.nao_update_density(None, None, 0, None, None, None) == 1
    assert lib.nao_integrate_h_many(None, None, 3, 0, None, None) == 1
    assert lib.nao_update_density_many(None, None, 0, None, None, None) == 1
    assert lib.nao_get_system(None, 0, None, None, None, None, None, None) == 1
    assert lib.nao_get_tuning(None, None, None) == 1
    assert lib.nao_update_density_gradient(None, None, 0, None, None, None, None) == 1
    assert lib.nao_update_density_gradient_many(None, None, 0, None, None, None, None) == 1
    assert lib.nao_update_density_hessian(None, None, 0, None, None, None, None, None) == 1
    assert lib.nao_integrate_h_tau(None, None, None, 7, 0, None, None) == 1
    assert lib.nao_pulay_matrices(None, None, 0, None, None, None) == 1
    assert lib.nao_pulay_forces(None, None, None, None, None, None, None) == 1
    assert lib.nao_bloch_sum(None, 0, None, None, None, 0, None, None, 0, 0, None, None, None) == 1
    info = nao.GridInfo()
    assert lib.nao_get_info(None, C.byref(info)) == 1
    out = C.c_void_p(123)
    assert lib.nao_grid_create(None, None, C.byref(out)) == 1 and out.value is None


def test_fault_injection_spec_is_checked_without_gpu():
    """nao_fault_inject accepts alloc/copy/launch:<n>, n >= 1, and clears with "" or None."""
    for good in ("alloc:1", "copy:17", "launch:3", "", None):
        nao.nao_fault_inject(good)
    for bad in ("alloc", "alloc:0", "launch:-2", "copy:x", "free:3", "alloc:3junk", ":4"):
        with pytest.raises(nao.NaoError) as e:
            nao.nao_fault_inject(bad)
        assert e.value.code == nao.NAO_ERR_INVALID_ARG
    nao.nao_fault_inject(None)
