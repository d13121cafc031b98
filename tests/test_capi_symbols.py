"""The C-ABI library builds, loads without a GPU and exports every entry
point declared in include/agf2.h (no compute calls here)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def declared_symbols():
    names = set()
    for hdr in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", hdr.read_text(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char\s*\*|double|long\s+long)\s*\*?\s*(agf2_\w+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("agf2_build_moments", "agf2_compress", "agf2_fock_loop", "agf2_run"):
        assert n in names


def test_library_exports_declared_symbols(agf2_lib):
    lib = ctypes.CDLL(str(agf2_lib.LIB_PATH))
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(agf2_lib.EXPORTED) <= declared_symbols()


def test_create_without_gpu_fails_cleanly(agf2_lib):
    import torch
    if torch.cuda.is_available():
        return
    h = ctypes.c_void_p()
    lib = ctypes.CDLL(str(agf2_lib.LIB_PATH))
    rc = lib.agf2_create(ctypes.byref(h), 0)
    assert rc != 0 and not h.value
