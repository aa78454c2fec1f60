"""The C-ABI library loads on a machine without a GPU and exports every
function that include/*.h declares; the Python binding wraps each of them.
No compute call is made here."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(spdz_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("spdz_load_preproc", "spdz_linear", "spdz_mul_batch", "spdz_open",
                     "spdz_mac_check", "spdz_run_dag", "spdz_innerprod_batch", "spdz_matmul",
                     "spdz_serve_start", "spdz_serve_submit", "spdz_serve_poll", "spdz_serve_stop"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2512_11112_b300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_2512_11112_b300 import spdz as S
    missing = [n for n in sorted(declared_functions()) if not callable(getattr(S, n, None))]
    assert not missing, missing
