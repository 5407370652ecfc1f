"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point include/gridcorr.h declares."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libso():
    from paper_2005_03060_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"GC_API\s+[\w\s\*]+?\b(gc_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("gc_create", "gc_destroy", "gc_correlate", "gc_last_error", "gc_device_status"):
        assert n in names


def test_library_exports_every_declared_symbol(libso):
    missing = [n for n in declared_symbols() if not hasattr(libso, n)]
    assert not missing, missing


def test_every_exported_entry_point_is_declared(libso):
    """The reverse direction: no gc_* symbol leaves the library undocumented
    (the dynamic symbol table as nm lists it)."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    from paper_2005_03060_gb300 import _build
    out = subprocess.run([nm, "-D", "--defined-only", _build.build()], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-1].startswith("gc_")}
    assert exported, "no gc_* symbols exported"
    assert sorted(exported - set(declared_symbols())) == []


def test_fft_size(libso):
    libso.gc_fft_size.argtypes = [ctypes.c_int]
    expect = {1: 2, 2: 4, 3: 8, 8: 16, 9: 32, 16: 32, 17: 64, 32: 64, 33: 128, 64: 128, 128: 256}
    for L, M in expect.items():
        assert libso.gc_fft_size(L) == M
        assert M >= 2 * L - 1
    assert libso.gc_fft_size(0) == 0 and libso.gc_fft_size(129) == 0


def test_null_context_is_rejected(libso):
    libso.gc_correlate.argtypes = [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int] * 4 + \
        [ctypes.c_void_p] * 3
    assert libso.gc_correlate(None, None, 0, 8, 1, 1, None, None, None) == 1  # GC_EINVAL
    libso.gc_last_error.restype = ctypes.c_char_p
    libso.gc_last_error.argtypes = [ctypes.c_void_p]
    assert libso.gc_last_error(None) == b"null context"


def test_host_entry_points_validate_arguments(libso):
    """The host-only calls reject what the header says they reject, without a
    GPU: NULL outputs, sizes out of range, p <= 0, log base 1, a NULL mask or
    an unknown lattice (GC_EINVAL = 1), and L = 2 (GC_EDEGEN = 6)."""
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    out = vp()
    ref = ctypes.byref(out)
    sub, low = libso.gc_selection_subset, libso.gc_selection_lowcad
    subm, lowm = libso.gc_selection_subset_masked, libso.gc_selection_lowcad_masked
    for f in (sub, low):
        f.argtypes = [i, i, d, d, vp]
    for f in (subm, lowm):
        f.argtypes = [i, i, d, d, vp, i, vp]
    assert sub(8, 64, 1.0, 2.0, None) == 1
    for args in ((1, 64, 1.0, 2.0), (257, 64, 1.0, 2.0), (8, 0, 1.0, 2.0), (8, 64, 0.0, 2.0),
                 (8, 64, 1.0, 1.0), (8, 64, -1.0, 2.0)):
        assert sub(*args, ref) == 1, args
        assert out.value is None
        assert low(*args, ref) == 1, args
    assert sub(2, 64, 1.0, 2.0, ref) == 6
    mask = (ctypes.c_uint8 * 64)(*([1] * 64))
    assert subm(8, 64, 1.0, 2.0, None, 0, ref) == 1
    assert lowm(8, 64, 1.0, 2.0, None, 0, ref) == 1
    assert subm(8, 64, 1.0, 2.0, ctypes.cast(mask, vp), 7, ref) == 1
    assert subm(8, 64, 1.0, 2.0, ctypes.cast(mask, vp), 0, ref) == 0 and out.value
    libso.gc_sel_free.argtypes = [vp]
    libso.gc_sel_info.argtypes = [vp, vp]
    info = (ctypes.c_int32 * 11)()
    assert libso.gc_sel_info(out, ctypes.cast(info, vp)) == 0 and info[0] == 8 and info[10] == 64
    assert libso.gc_sel_info(None, ctypes.cast(info, vp)) == 1
    assert libso.gc_sel_info(out, None) == 1
    libso.gc_sel_free(out)
    libso.gc_sel_free(None)


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    """The binding raises when the compiled library is absent (no fallback)."""
    import importlib.util
    src = os.path.join(ROOT, "paper_2005_03060_gb300", "gridcorr.py")
    fake = tmp_path / "gridcorr.py"
    fake.write_text(open(src).read())
    spec = importlib.util.spec_from_file_location("gridcorr_nolib", fake)
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)
