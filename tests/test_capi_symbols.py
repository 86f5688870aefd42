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
    for must in ("cf_setup", "cf_footprint", "cf_solve", "cf_vcycle", "cf_apply", "cf_level_colour_step",
                 "cf_coarse_solve_noalloc", "cf_batch_solve", "cf_server_run"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2508_11608_gb300.build import build
    lib = ctypes.CDLL(build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_bad_arguments_return_einval_without_a_device():
    """The documented error behaviour of the boundary: device calls on a
    host-only handle, bad levels and indices and null outputs all return
    CF_EINVAL with a message, before any CUDA call (so this runs on a host
    without a GPU)."""
    import ctypes
    import numpy as np
    import paper_2508_11608_gb300 as cm
    from paper_2508_11608_gb300 import _lib
    lib = _lib.load()
    pb = cm.Problem(2, 16, 2, 2, center=[0.031, 0.017], radius=0.7, host_only=True)
    h = pb._h
    dummy = ctypes.c_void_p(256)  # never dereferenced: the handle check comes first
    info = _lib.cf_info()
    calls = {
        "cf_apply": lambda: lib.cf_apply(h, dummy, dummy, None),
        "cf_vcycle": lambda: lib.cf_vcycle(h, dummy, dummy, None),
        "cf_solve": lambda: lib.cf_solve(h, dummy, dummy, 1e-8, 10, ctypes.byref(info), None),
        "cf_level_colour_step": lambda: lib.cf_level_colour_step(h, 1, 0, 0, _lib.CF_FP64, dummy, dummy, None),
        "cf_coarse_solve": lambda: lib.cf_coarse_solve(h, _lib.CF_FP64, dummy, dummy, None),
        "cf_coarse_solve_noalloc": lambda: lib.cf_coarse_solve_noalloc(h, dummy, dummy, None),
        "cf_batch_create": lambda: lib.cf_batch_create(ctypes.byref(ctypes.c_void_p(h.value)), 1,
                                                       ctypes.byref(ctypes.c_void_p())),
        "cf_footprint(null)": lambda: lib.cf_footprint(None, None, 2, None, ctypes.byref(ctypes.c_size_t())),
        "cf_problem_footprint(null)": lambda: lib.cf_problem_footprint(None, ctypes.byref(ctypes.c_size_t())),
        "cf_set_kernel_variant(host-only)": lambda: lib.cf_set_kernel_variant(h, 1, 1),
        "cf_set_wait_limit(host-only)": lambda: lib.cf_set_wait_limit(h, 5),
        "cf_dof_coords(bad level)": lambda: lib.cf_dof_coords(h, pb.n_levels, dummy),
        "cf_host_cell_matrix(bad level)": lambda: lib.cf_host_cell_matrix(h, -1, 0, dummy),
        "cf_host_cell_matrix(inactive cell)": lambda: lib.cf_host_cell_matrix(h, 1, 0, dummy),
        "cf_host_cut_patch(bad index)": lambda: lib.cf_host_cut_patch(h, 1, 10 ** 9, dummy, dummy, dummy, None),
        "cf_host_coarse_inverse(null)": lambda: lib.cf_host_coarse_inverse(h, None),
        "cf_host_diagonal(level 0)": lambda: lib.cf_host_diagonal(h, 0, dummy),
    }
    for name, call in calls.items():
        st = call()
        assert st == _lib.CF_EINVAL, (name, st)
        assert lib.cf_last_error(), name
    # the handle still answers afterwards
    assert pb.n_dofs() > 0 and np.isfinite(pb.host_rhs()).all()


def test_setup_and_footprint_signatures_follow_the_boundary():
    """cf_setup takes (mesh, level set, degree, params, stream, out) and
    cf_footprint (mesh, level set, degree, params, bytes): the estimate needs
    no built problem."""
    import re
    src = open(os.path.join(ROOT, "include", "cutmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    setup = re.search(r"cf_status cf_setup\(([^)]*)\)", src).group(1)
    assert [a.split()[-1].lstrip("*") for a in setup.split(",")] == ["mesh", "ls", "degree", "params", "stream", "out"]
    fp = re.search(r"cf_status cf_footprint\(([^)]*)\)", src).group(1)
    assert [a.split()[-1].lstrip("*") for a in fp.split(",")] == ["mesh", "ls", "degree", "params", "bytes"]
