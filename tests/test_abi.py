"""The C-ABI library builds, loads and exports every function include/npb.h declares.

These tests make no compute call: they run on a machine without a GPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "npb.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(npb_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_1410_2788_gb300 as npb
    from paper_1410_2788_gb300 import build

    build.build()
    return npb.load_library()


def test_header_declares_the_boundary_calls():
    names = _declared_functions()
    for required in ["npb_grid_create", "npb_lod_solve", "npb_energy", "npb_submit", "npb_poll",
                     "npb_ctx_create", "npb_potential", "npb_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    import paper_1410_2788_gb300 as npb

    assert sorted(npb.SIGNATURES) == _declared_functions()


def test_exports_are_c_symbols(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (npb_\w+)$", out, flags=re.M))
    assert set(_declared_functions()) <= exported


def test_struct_layouts_match_header():
    import paper_1410_2788_gb300 as npb

    # int32 n_atoms, 3 pointers, 4 doubles, int32[3], double[3]
    assert ctypes.sizeof(npb.npb_problem) == 8 + 3 * 8 + 4 * 8 + 16 + 3 * 8
    assert ctypes.sizeof(npb.npb_opts) == 2 * 8 + 6 * 4
    assert ctypes.sizeof(npb.npb_result) == 3 * 8 + 8 + 4 + 12


def test_no_device_is_reported_not_crashed(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1410_2788_gb300 as npb

    with pytest.raises(npb.NpbError):
        npb.npb_ctx_create(0, 0)
    assert npb.npb_version().startswith("npb-lod-gb300")


def test_binding_constants_match_header():
    """Every NPB_* integer constant the header defines has the same value in the binding."""
    import paper_1410_2788_gb300 as npb

    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    defs = dict(re.findall(r"^#define\s+(NPB_\w+)\s+\(?(-?\d+)\)?\s*$", text, flags=re.M))
    assert len(defs) > 30
    missing = [k for k in defs if not hasattr(npb, k)]
    assert not missing, missing
    wrong = {k: (getattr(npb, k), int(v)) for k, v in defs.items() if getattr(npb, k) != int(v)}
    assert not wrong, wrong
