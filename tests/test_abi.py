"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/ifem.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

from paper_1807_08219_gb300 import build, ifem

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ifem.h")


def declared_functions():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|int64_t|int)\s*\**\s*(ifem_\w+)\s*\(", src, re.M)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for required in ("ifem_compute_forces", "ifem_spread", "ifem_interpolate", "ifem_step_coupling",
                     "ifem_force_hvp"):
        assert required in names
    assert set(names) == set(ifem.EXPORTS), set(names) ^ set(ifem.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_config_default_without_gpu():
    lib = ifem.load()
    cfg = ifem.ifem_config()
    assert lib.ifem_config_default(ctypes.byref(cfg)) == 0
    assert (cfg.precision, cfg.kernel, cfg.scatter, cfg.tile) == (0, 0, 0, 0)
    assert lib.ifem_config_default(None) == -1
