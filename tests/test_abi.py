"""CPU checks of the boundary: the C-ABI library loads and exports every symbol
include/napg.h declares (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "napg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(napg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("napg_create", "napg_load_cohort", "napg_run", "napg_run_batch", "napg_debug_integers",
                 "napg_serve_start", "napg_serve_submit", "napg_serve_poll", "napg_serve_stop"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2505_00448_gb300 import build
    lib_path = build.build()
    L = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(L, name), f"{name} declared in napg.h but not exported"
    from paper_2505_00448_gb300 import napg
    assert set(napg.EXPORTS) <= set(declared_functions())
    assert napg.version().startswith("napg")
