"""CPU tests of the C-ABI boundary: the library builds, loads, and exports
every entry point that include/sht.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for f in os.listdir(HEADER_DIR):
        if f.endswith(".h"):
            src = open(os.path.join(HEADER_DIR, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names.update(re.findall(r"\b(sht_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("sht_plan_create", "sht_plan_destroy", "sht_workspace_bytes", "sht_alm2map",
              "sht_map2alm", "sht_alm2map_adjoint", "sht_map2alm_adjoint", "sht_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2208_10154_b300 import build, sht
    build.build()
    lib = ctypes.CDLL(sht.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_without_gpu():
    from paper_2208_10154_b300 import build, sht
    build.build()
    lib = sht.load()
    assert b"sm_103a" in lib.sht_version()


def test_plan_create_rejects_bad_arguments_without_gpu():
    from paper_2208_10154_b300 import build, sht
    build.build()
    lib = sht.load()
    h = ctypes.c_void_p()
    assert lib.sht_plan_create(0, 10, -1, 0, 0, 0, ctypes.byref(h)) == sht.SHT_EINVAL
    assert lib.sht_plan_create(4, 10, 20, 0, 0, 0, ctypes.byref(h)) == sht.SHT_EINVAL
    assert lib.sht_plan_create(4, 10, -1, 1, 0, 0, ctypes.byref(h)) == sht.SHT_EINVAL
    assert "spin" in sht.sht_last_error()
    assert lib.sht_workspace_bytes(None, 4) == 0


def test_oracle_and_product_share_no_code():
    """The oracle and the CUDA path never import or include each other."""
    pkg = os.path.join(ROOT, "paper_2208_10154_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f), errors="replace").read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "sht_oracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "import paper_2208_10154_b300" not in txt, f
            assert "from paper_2208_10154_b300" not in txt, f
            assert "#include" not in txt or "sht.h" not in txt, f
