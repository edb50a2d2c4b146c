"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/bttb.h declares; argument validation that
needs no device returns the documented codes; host-side recipes are stable."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_20350_gb300 import build
    build.build()
    import paper_2506_20350_gb300 as bt
    return bt.load_library()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "bttb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(bttb_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ["bttb_plan_create", "bttb_set_generators", "bttb_matvec", "bttb_gmres_solve",
              "bttb_plan_destroy", "bttb_last_error", "bttb_plan_workspace_bytes"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_names_match_header():
    import paper_2506_20350_gb300 as bt
    for n in _declared_functions():
        assert hasattr(bt, n), n
        assert n in bt.EXPORTS


def test_invalid_sizes_rejected_without_device(lib):
    import paper_2506_20350_gb300 as bt
    h = ctypes.c_void_p()
    for args in [(0, 4, 12, 1), (4, 0, 12, 1), (4, 4, 0, 1), (4, 4, 12, 0), (2000, 4, 12, 1), (4, 4, 300, 1),
                 (4, 4, 12, 5000)]:
        rc = lib.bttb_plan_create(ctypes.byref(h), *args, 0, None)
        assert rc == bt.BTTB_ERR_INVALID_ARG
        assert h.value is None
        assert "sizes" in bt.bttb_last_error()
    rc = lib.bttb_plan_create(ctypes.byref(h), 4, 4, 12, 1, 1 << 7, None)
    assert rc == bt.BTTB_ERR_INVALID_ARG
    assert lib.bttb_plan_create(None, 4, 4, 12, 1, 0, None) == bt.BTTB_ERR_INVALID_ARG


def test_null_plan_calls_are_errors(lib):
    import paper_2506_20350_gb300 as bt
    assert lib.bttb_matvec(None, None, None, 1, 10, 1, 0) == bt.BTTB_ERR_INVALID_ARG
    assert lib.bttb_set_generators(None, None, 1, 1) == bt.BTTB_ERR_INVALID_ARG
    assert lib.bttb_gmres_solve(None, None, None, 1, 1, None, None) == bt.BTTB_ERR_INVALID_ARG
    assert lib.bttb_plan_destroy(None) == bt.BTTB_OK
    assert lib.bttb_plan_workspace_bytes(None) == 0
    assert isinstance(bt.bttb_last_error(), str)


def test_struct_layouts_match_c():
    import paper_2506_20350_gb300 as bt
    # double, 6 ints, pointer, int -> 48 bytes with natural alignment on LP64
    assert ctypes.sizeof(bt.GmresOpts) == 48
    assert bt.GmresOpts.history.offset == 32
    assert ctypes.sizeof(bt.ColResult) == 24
    assert bt.ColResult.relres_true.offset == 16


def test_uneven_batch_recipe_is_stable():
    from workloads import arrays
    specs = arrays.uneven_batch_specs()
    assert len(specs) == 64
    assert all(8 <= s.nx <= 40 and 8 <= s.ny <= 40 and s.b in (24, 60, 96) and 1 <= s.nrhs <= 16 for s in specs)
    assert specs[5].seed == 3005
    again = arrays.uneven_batch_specs()
    assert [(s.nx, s.ny, s.b, s.nrhs) for s in specs] == [(s.nx, s.ny, s.b, s.nrhs) for s in again]


def test_excitations():
    from workloads import arrays
    v = arrays.port_excitations(4, 4, 12, [(1, 1)])
    assert v.shape == (192, 1) and v[(1 * 4 + 1) * 12, 0] == 1 and np.count_nonzero(v) == 1
    c = arrays.centre_excitation(30, 30, 60)
    assert c[(15 * 30 + 15) * 60] == 1 and np.count_nonzero(c) == 1


def test_bounds_check_entry_points_in_the_normal_build(lib):
    """The normal library reports that it is not the bounds-checked build (no hits, no device call) and
    refuses the probe without launching anything."""
    import paper_2506_20350_gb300 as bt
    h, f = ctypes.c_ulonglong(7), ctypes.c_ulonglong(7)
    assert lib.bttb_check_report(ctypes.byref(h), ctypes.byref(f)) == 0
    assert h.value == 0 and f.value == 0
    assert lib.bttb_check_report(None, None) == 0
    n = ctypes.c_ulonglong(7)
    assert lib.bttb_check_probe(ctypes.byref(n)) == bt.BTTB_ERR_INVALID_ARG
    assert n.value == 0 and "checked" in bt.bttb_last_error()
