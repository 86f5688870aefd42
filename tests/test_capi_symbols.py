"""The C-ABI library builds, loads without a GPU, and exports every function
declared in include/cutmg.h (no compute calls)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cutmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cf_setup", "cf_solve", "cf_vcycle", "cf_apply", "cf_level_colour_step",
                 "cf_coarse_solve_noalloc", "cf_batch_solve", "cf_server_run"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2508_11608_gb300.build import build
    lib = ctypes.CDLL(build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
