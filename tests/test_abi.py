"""Host-side checks of the C ABI and of the oracle/CUDA separation (no GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(dhr_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    import paper_2406_06963_b300 as dhrs
    from paper_2406_06963_b300 import build
    build.build()
    L = ctypes.CDLL(dhrs.LIB_PATH)
    names = _declared_symbols()
    assert len(names) >= 17
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    # the binding wraps every declared entry point
    assert names <= set(dhrs._SIGNATURES), sorted(names - set(dhrs._SIGNATURES))


def test_debug_library_exports_every_declared_symbol():
    """The bounds-checked build (DHR_DEBUG) has the same ABI."""
    from paper_2406_06963_b300 import build
    L = ctypes.CDLL(build.build(debug=True))
    missing = [n for n in sorted(_declared_symbols()) if not hasattr(L, n)]
    assert not missing, missing


def test_release_build_reports_itself():
    """The release library says it is not the debug build and refuses the
    self test, without touching a device."""
    from paper_2406_06963_b300 import build
    L = ctypes.CDLL(build.build())
    err, dbg = ctypes.c_uint64(7), ctypes.c_int32(7)
    assert L.dhr_debug_status(ctypes.byref(err), ctypes.byref(dbg)) == 0
    assert (err.value, dbg.value) == (0, 0)
    assert L.dhr_debug_selftest(None) == 6   # DHR_ERR_STATE
    assert L.dhr_debug_status(ctypes.byref(err), ctypes.byref(dbg)) == 0   # clears the error text


def test_binding_constants_match_header():
    """The binding's integer constants are the header's #defines."""
    import paper_2406_06963_b300 as dhrs
    text = open(os.path.join(ROOT, "include", "dhrs.h")).read()
    defs = dict(re.findall(r"#define\s+DHR_([A-Z0-9_]+)\s+(\w+)", text))
    as_int = lambda v: int(v.rstrip("uU"), 0)
    assert as_int(defs["PRIMARY_RASTER"]) == dhrs.PRIMARY_RASTER
    assert as_int(defs["PRIMARY_TRAVERSE"]) == dhrs.PRIMARY_TRAVERSE
    assert as_int(defs["TAPE_RECOMPUTE"]) == dhrs.TAPE_RECOMPUTE
    assert as_int(defs["TAPE_STORE"]) == dhrs.TAPE_STORE
    assert as_int(defs["MAX_LIGHTS"]) == dhrs.MAX_LIGHTS
    assert as_int(defs["BACKGROUND"]) == dhrs.BACKGROUND


def test_binding_loads_without_gpu():
    import paper_2406_06963_b300 as dhrs
    L = dhrs.lib()
    assert L.dhr_last_error() == b""


def test_oracle_and_cuda_share_no_code():
    """The oracle and the CUDA library include nothing from each other and
    the product package never imports the oracle."""
    csrc = glob.glob(os.path.join(ROOT, "paper_2406_06963_b300", "csrc", "*"))
    for f in csrc:
        t = open(f).read()
        for inc in re.findall(r"#include\s*[<\"]([^>\"]+)", t):
            assert "oracle" not in inc and "orc_" not in inc, (f, inc)
        assert "orc_" not in t, f
    for f in glob.glob(os.path.join(ROOT, "paper_2406_06963_b300", "*.py")):
        t = open(f).read()
        assert not re.search(r"^\s*(from|import)\s+oracle", t, re.M), f
    oc = open(os.path.join(ROOT, "oracle", "dhrs_oracle.c")).read()
    for inc in re.findall(r"#include\s*[<\"]([^>\"]+)", oc):
        assert inc in ("math.h", "stdint.h", "stdlib.h", "string.h", "omp.h"), inc
