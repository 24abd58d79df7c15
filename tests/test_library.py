"""The C-ABI library loads and exports every entry point declared in include/*.h (no GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1802_07525_gb300 import build
    return build.build()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        with open(h) as fh:
            txt = fh.read()
        names |= set(re.findall(r"MFC_API\s+[\w\s\*]+?\b(mfc_\w+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary_calls():
    names = declared_symbols()
    for required in ["mfc_create_lattice", "mfc_set_geometry", "mfc_step_flow", "mfc_step_ade",
                     "mfc_solve_steady", "mfc_read_fields"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(mfc_\w+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_1802_07525_gb300 import mfc
    assert set(declared_symbols()) <= set(mfc.EXPORTED)
    L = mfc.lib()
    for n in declared_symbols():
        assert getattr(L, n) is not None


def test_host_only_calls(libpath):
    from paper_1802_07525_gb300 import mfc
    assert mfc.status_string(mfc.MFC_NOT_CONVERGED).startswith("not converged")
    assert mfc.lib().mfc_version().decode().startswith("mfc ")
    b2 = mfc.lattice_bytes((2048, 1024))
    # two FP32 buffers of 9 + 5 planes dominate: 2 * 14 * 4 B per node
    assert 2 * 14 * 4 * 2048 * 1024 <= b2 <= 2 * 14 * 4 * 2048 * 1024 * 1.3
    b16 = mfc.lattice_bytes((2048, 1024), precision=mfc.MFC_FP16_DEV)
    assert b16 < b2
    b3 = mfc.lattice_bytes((64, 32, 48))
    assert b3 >= 2 * 26 * 4 * 64 * 32 * 48
    # FP64 storage: populations at 8 B and fields at 8 B.  The FP32 - FP16 difference gives the
    # plane size P (2 buffers x 14 planes x 2 B per element), from which the FP64 - FP32
    # difference is fixed: 2 x 14 planes x 4 B more, and 2 + dim fields x 4 B more.
    b64 = mfc.lattice_bytes((2048, 1024), precision=mfc.MFC_FP64)
    P = (b2 - b16) // (2 * 14 * 2)
    assert (b2 - b16) % (2 * 14 * 2) == 0 and P >= 2048 * 1024
    assert b64 - b2 == 2 * 14 * P * 4 + (2 + 2) * P * 4
    assert mfc.lattice_bytes((2048, 1024), precision=3) == 0
    # batches take FP32 or FP16 storage only; refused before any device call
    import pytest
    with pytest.raises(mfc.MfcError) as e:
        mfc.Batch(precision=mfc.MFC_FP64)
    assert e.value.status == mfc.MFC_ERR_ARG
    # invalid descriptors are refused without touching a device
    assert mfc.lattice_bytes((0, 4)) == 0
    assert mfc.lattice_bytes((8, 8), bc=(mfc.MFC_BC_WALL, mfc.MFC_BC_INOUT)) == 0


def test_create_rejects_bad_arguments_before_any_allocation(libpath):
    from paper_1802_07525_gb300 import mfc
    L = mfc.lib()
    h = ctypes.c_void_p()
    d = mfc.make_desc((8, 8))
    p = mfc.make_params(tau=0.5)
    assert L.mfc_create_lattice(ctypes.byref(d), ctypes.byref(p), ctypes.byref(h)) == mfc.MFC_ERR_ARG
    assert b"tau" in L.mfc_last_error(None)
    p = mfc.make_params(k_sink=1.5)
    assert L.mfc_create_lattice(ctypes.byref(d), ctypes.byref(p), ctypes.byref(h)) == mfc.MFC_ERR_ARG
    p = mfc.make_params(k_half=-0.1)
    assert L.mfc_create_lattice(ctypes.byref(d), ctypes.byref(p), ctypes.byref(h)) == mfc.MFC_ERR_ARG
    assert b"k_half" in L.mfc_last_error(None)
    d = mfc.make_desc((8, 8), bc=(mfc.MFC_BC_WALL, mfc.MFC_BC_INOUT))
    p = mfc.make_params()
    assert L.mfc_create_lattice(ctypes.byref(d), ctypes.byref(p), ctypes.byref(h)) == mfc.MFC_ERR_ARG
    assert not h.value


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1802_07525_gb300 import mfc
    monkeypatch.setattr(mfc, "_lib", None)
    monkeypatch.setattr(mfc, "LIB_PATH", str(tmp_path / "libmfc.so"))
    with pytest.raises(RuntimeError, match="not built"):
        mfc.lib()
