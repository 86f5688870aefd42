"""GB300-native CutFEM multigrid (arXiv 2508.11608): Python handle over the
C ABI of libcutmg.so.

Device vectors are torch CUDA tensors of dtype float64 in the library's DoF
order; torch is used for device memory and streams only.
"""

import ctypes

import numpy as np

from . import _lib
from ._lib import CF_FP64, CF_MIXED, CF_SMOOTHER_CHEBYSHEV, CF_SMOOTHER_MVS, CutmgError, check  # noqa: F401


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def footprint(dim, n_cells, n_levels, degree, levelset, lo=-1.0, hi=1.0, n_c=0, setup_threads=0):
    """Device bytes a cf_setup of this problem would hold, estimated before
    any setup (cf_footprint: classification and index lists only)."""
    lib = _lib.load()
    mesh = _lib.cf_mesh(dim, n_cells, lo, hi, n_levels)
    ls = _lib.make_levelset(levelset)
    prm = _lib.cf_params()
    prm.n_c = n_c
    prm.setup_threads = setup_threads
    out = ctypes.c_size_t()
    check(lib.cf_footprint(ctypes.byref(mesh), ctypes.byref(ls), degree, ctypes.byref(prm), ctypes.byref(out)))
    return out.value


class Problem:
    """A resident multigrid hierarchy (cf_setup .. cf_destroy)."""

    def __init__(self, dim, n_cells, n_levels, degree, center=None, radius=None, plane=None,
                 levelset=None, lo=-1.0, hi=1.0, gamma_D=0.0, gamma_ghost=(0.0,) * 4, n_c=0,
                 quad_q=0, precision=CF_FP64, host_only=False, smoother=0, smoother_degree=0, setup_threads=None,
                 stream=None):
        lib = _lib.load()
        self._lib = lib
        mesh = _lib.cf_mesh(dim, n_cells, lo, hi, n_levels)
        if levelset is not None:
            spec = levelset
        elif plane is not None:
            spec = {"kind": "plane", "normal": plane[0], "offset": plane[1]}
        else:
            spec = {"kind": "sphere", "center": center, "radius": radius}
        ls = _lib.make_levelset(spec)
        self._ls = ls  # level-set callbacks are called again by rhs_user
        prm = _lib.cf_params()
        prm.gamma_D = gamma_D
        for k, v in enumerate(gamma_ghost):
            prm.gamma_ghost[k] = v
        prm.n_c = n_c
        prm.quad_q = quad_q
        prm.precision = precision
        prm.smoother = smoother
        prm.smoother_degree = smoother_degree
        if setup_threads is None:  # Python callbacks serialise on the interpreter lock
            setup_threads = 1 if spec.get("kind") == "callback" else 0
        prm.setup_threads = setup_threads
        h = ctypes.c_void_p()
        if host_only:
            check(lib.cf_setup_host(ctypes.byref(mesh), ctypes.byref(ls), degree, ctypes.byref(prm),
                                    ctypes.byref(h)))
        else:
            check(lib.cf_setup(ctypes.byref(mesh), ctypes.byref(ls), degree, ctypes.byref(prm),
                               _stream(stream), ctypes.byref(h)))
        self._h = h
        self.dim = dim
        self.degree = degree

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- sizes and maps ---------------------------------------------------------
    @property
    def n_levels(self):
        return self._lib.cf_n_levels(self._h)

    def n_dofs(self, level=None):
        if level is None:
            return self._lib.cf_n_dofs(self._h)
        return self._lib.cf_level_n_dofs(self._h, level)

    def dof_lattice(self, level=None):
        level = self.n_levels - 1 if level is None else level
        out = np.empty(self.n_dofs(level), dtype=np.int64)
        check(self._lib.cf_dof_lattice(self._h, level, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def dof_coords(self, level=None):
        level = self.n_levels - 1 if level is None else level
        out = np.empty((self.n_dofs(level), self.dim), dtype=np.float64)
        check(self._lib.cf_dof_coords(self._h, level, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def stats(self, level=None):
        level = self.n_levels - 1 if level is None else level
        out = np.empty(6, dtype=np.int64)
        check(self._lib.cf_stats(self._h, level, out.ctypes.data_as(ctypes.c_void_p)))
        keys = ["active_cells", "cut_cells", "ghost_faces", "patches", "cut_patches", "inverse_entries"]
        return dict(zip(keys, out.tolist()))

    def footprint(self):
        """Estimated device bytes of this problem's device handle."""
        out = ctypes.c_size_t()
        check(self._lib.cf_problem_footprint(self._h, ctypes.byref(out)))
        return out.value

    def work_model(self, level, kind, colour):
        """Algorithmic work of one colour step: kind 0 interior, 1 cut patches.
        Returns (flops, scalars moved, index bytes moved)."""
        out = np.empty(3, dtype=np.float64)
        check(self._lib.cf_work_model(self._h, level, kind, colour, out.ctypes.data_as(ctypes.c_void_p)))
        return tuple(out.tolist())

    def set_precision(self, precision):
        check(self._lib.cf_set_precision(self._h, precision))

    def set_kernel_variant(self, family, variant):
        """Force a launch variant (family _lib.CF_VAR_INTERIOR / CF_VAR_CUT;
        0 = automatic)."""
        check(self._lib.cf_set_kernel_variant(self._h, family, variant))

    def set_wait_limit(self, polls):
        """Polls of the tensor-core interior kernel's wait on its product
        (default 2^22)."""
        check(self._lib.cf_set_wait_limit(self._h, int(polls)))

    # ---- finest-level calls ----------------------------------------------------------
    def rhs(self, b, stream=None):
        check(self._lib.cf_rhs(self._h, _ptr(b), _stream(stream)))

    @staticmethod
    def _data_fn(fn, dim):
        if fn is None:
            return ctypes.cast(None, _lib.DATA_FN)
        return _lib.DATA_FN(lambda xp, user: float(fn(tuple(xp[k] for k in range(dim)))))

    def rhs_user(self, f, g, b=None, stream=None):
        """Right-hand side for source f(x) and Dirichlet data g(x) (Python
        callables of a coordinate tuple; None = zero).  With a device tensor b
        it is filled in place (cf_rhs_user); without, the host array is
        returned (cf_host_rhs_user)."""
        cf, cg = self._data_fn(f, self.dim), self._data_fn(g, self.dim)
        if b is None:
            out = np.empty(self.n_dofs(), dtype=np.float64)
            check(self._lib.cf_host_rhs_user(self._h, cf, cg, None, out.ctypes.data_as(ctypes.c_void_p)))
            return out
        check(self._lib.cf_rhs_user(self._h, cf, cg, None, _ptr(b), _stream(stream)))
        return b

    def apply(self, x, y, stream=None):
        check(self._lib.cf_apply(self._h, _ptr(x), _ptr(y), _stream(stream)))

    def vcycle(self, r, z, stream=None):
        check(self._lib.cf_vcycle(self._h, _ptr(r), _ptr(z), _stream(stream)))

    def solve(self, b, x, rtol=1e-8, maxit=500, stream=None, allow_noconv=False):
        info = _lib.cf_info()
        st = self._lib.cf_solve(self._h, _ptr(b), _ptr(x), rtol, maxit, ctypes.byref(info),
                                _stream(stream))
        if not (allow_noconv and st == _lib.CF_ENOCONV):
            check(st)
        return {"iterations": info.iterations, "rel_residual": info.rel_residual,
                "true_rel_residual": info.true_rel_residual, "solve_ms": info.solve_ms}

    def solve_vcycle(self, b, x, rtol=1e-9, maxit=500, stream=None, allow_noconv=False):
        """The V-cycle iteration as the solver (cf_solve_vcycle)."""
        info = _lib.cf_info()
        st = self._lib.cf_solve_vcycle(self._h, _ptr(b), _ptr(x), rtol, maxit, ctypes.byref(info),
                                       _stream(stream))
        if not (allow_noconv and st == _lib.CF_ENOCONV):
            check(st)
        return {"iterations": info.iterations, "rel_residual": info.rel_residual,
                "true_rel_residual": info.true_rel_residual, "solve_ms": info.solve_ms}

    def solve_gmres(self, b, x, rtol=1e-9, restart=30, maxit=500, stream=None, allow_noconv=False):
        """GMRES(restart) preconditioned by the V-cycle (cf_solve_gmres)."""
        info = _lib.cf_info()
        st = self._lib.cf_solve_gmres(self._h, _ptr(b), _ptr(x), rtol, restart, maxit, ctypes.byref(info),
                                      _stream(stream))
        if not (allow_noconv and st == _lib.CF_ENOCONV):
            check(st)
        return {"iterations": info.iterations, "rel_residual": info.rel_residual,
                "true_rel_residual": info.true_rel_residual, "solve_ms": info.solve_ms}

    # ---- single steps on one level ---------------------------------------------------
    def level_apply(self, level, x, y, precision=CF_FP64, stream=None):
        check(self._lib.cf_level_apply(self._h, level, precision, _ptr(x), _ptr(y), _stream(stream)))

    def colour_step(self, level, cut, colour, x, b, precision=CF_FP64, stream=None):
        check(self._lib.cf_level_colour_step(self._h, level, precision, int(cut), colour, _ptr(x),
                                             _ptr(b), _stream(stream)))

    def smooth(self, level, x, b, post=False, precision=CF_FP64, stream=None):
        check(self._lib.cf_level_smooth(self._h, level, precision, int(post), _ptr(x), _ptr(b),
                                        _stream(stream)))

    def restrict(self, level, r_fine, b_coarse, precision=CF_FP64, stream=None):
        check(self._lib.cf_level_restrict(self._h, level, precision, _ptr(r_fine), _ptr(b_coarse),
                                          _stream(stream)))

    def prolongate(self, level, x_coarse, x_fine, precision=CF_FP64, stream=None):
        check(self._lib.cf_level_prolongate(self._h, level, precision, _ptr(x_coarse), _ptr(x_fine),
                                            _stream(stream)))

    def coarse_solve(self, b0, x0, precision=CF_FP64, stream=None):
        check(self._lib.cf_coarse_solve(self._h, precision, _ptr(b0), _ptr(x0), _stream(stream)))

    def coarse_solve_noalloc(self, b0, x0, stream=None):
        """cf_coarse_solve_noalloc: the FP64 coarse solve without any device
        allocation in the call (fixed static staging array, see cutmg.h)."""
        check(self._lib.cf_coarse_solve_noalloc(self._h, _ptr(b0), _ptr(x0), _stream(stream)))

    # ---- instrumentation --------------------------------------------------------------
    def launch_count(self):
        return self._lib.cf_launch_count(self._h)

    def profile_start(self, kernel, level=-1):
        check(self._lib.cf_profile_start_level(self._h, kernel, level))

    def profile_read(self):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        fl = ctypes.c_double()
        by = ctypes.c_double()
        check(self._lib.cf_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl),
                                        ctypes.byref(by)))
        return {"ms": ms.value, "launches": n.value, "flops": fl.value, "bytes": by.value}

    # ---- host-side views of the setup (work on host-only handles too) -------------
    def host_rhs(self):
        out = np.empty(self.n_dofs(), dtype=np.float64)
        check(self._lib.cf_host_rhs(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def host_cell_matrix(self, level, cell):
        nb = (self.degree + 1) ** self.dim
        out = np.empty((nb, nb), dtype=np.float64)
        check(self._lib.cf_host_cell_matrix(self._h, level, cell, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def host_diagonal(self, level):
        """Diagonal of A_level in DoF order (levels >= 1)."""
        out = np.empty(self.n_dofs(level), dtype=np.float64)
        check(self._lib.cf_host_diagonal(self._h, level, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def host_coarse_inverse(self):
        """A_0^{-1} of the coarsest level (n_0 x n_0, DoF order)."""
        n0 = self.n_dofs(0)
        out = np.empty((n0, n0), dtype=np.float64)
        check(self._lib.cf_host_coarse_inverse(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def host_interior_update(self, level):
        """The level's dense interior-patch map W ((2p-1)^d x (2p+1)^d)."""
        ni, nc = (2 * self.degree - 1) ** self.dim, (2 * self.degree + 1) ** self.dim
        out = np.empty((ni, nc), dtype=np.float64)
        check(self._lib.cf_host_interior_update(self._h, level, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def host_patches(self, level, with_inverse=True):
        """(interior vertices, [(vertex, lattice nodes, inverse or None)] of cut patches)."""
        ni = ctypes.c_int64()
        nc = ctypes.c_int64()
        check(self._lib.cf_host_patch_counts(self._h, level, ctypes.byref(ni), ctypes.byref(nc)))
        inter = []
        v = ctypes.c_int64()
        for j in range(ni.value):
            check(self._lib.cf_host_interior_patch(self._h, level, j, ctypes.byref(v)))
            inter.append(v.value)
        cmax = (2 * self.degree + 1) ** self.dim
        nodes = np.empty(cmax, dtype=np.int64)
        m = ctypes.c_int()
        cut = []
        for j in range(nc.value):
            inv = np.empty(cmax * cmax, dtype=np.float64) if with_inverse else None
            check(self._lib.cf_host_cut_patch(
                self._h, level, j, ctypes.byref(v), ctypes.byref(m),
                nodes.ctypes.data_as(ctypes.c_void_p),
                inv.ctypes.data_as(ctypes.c_void_p) if with_inverse else None))
            k = m.value
            cut.append((v.value, nodes[:k].copy(),
                        inv[:k * k].reshape(k, k).copy() if with_inverse else None))
        return inter, cut


class Batch:
    """Many problems solved together (cf_batch_*): one launch per V-cycle
    depth, colour and step for all problems of the same (dim, degree)."""

    def __init__(self, problems):
        self._lib = _lib.load()
        self.problems = list(problems)
        arr = (ctypes.c_void_p * len(self.problems))(*[p._h.value for p in self.problems])
        h = ctypes.c_void_p()
        check(self._lib.cf_batch_create(arr, len(self.problems), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self):
        return self._lib.cf_batch_launch_count(self._h)

    def solve(self, bs, xs, rtol=1e-8, maxit=500, precision=CF_FP64, stream=None, allow_noconv=False):
        k = len(self.problems)
        pb = (ctypes.c_void_p * k)(*[b.data_ptr() for b in bs])
        px = (ctypes.c_void_p * k)(*[x.data_ptr() for x in xs])
        infos = (_lib.cf_info * k)()
        st = self._lib.cf_batch_solve(self._h, precision, pb, px, rtol, maxit, infos, _stream(stream))
        if not (allow_noconv and st == _lib.CF_ENOCONV):
            check(st)
        return [{"iterations": i.iterations, "rel_residual": i.rel_residual,
                 "true_rel_residual": i.true_rel_residual, "solve_ms": i.solve_ms} for i in infos]


class Server:
    """Continuous-batching solve server (cf_server_*)."""

    def __init__(self, hbm_budget_bytes, max_active=64, precision=CF_FP64, keep_solutions=False):
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        check(self._lib.cf_server_create(int(hbm_budget_bytes), max_active, precision, int(keep_solutions),
                                         ctypes.byref(h)))
        self._h = h
        self.keep = keep_solutions
        self.ndofs = []
        self._levelsets = []

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cf_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, dim, n_cells, n_levels, degree, levelset, arrival_s, rtol=1e-8, maxit=500,
               lo=-1.0, hi=1.0):
        mesh = _lib.cf_mesh(dim, n_cells, lo, hi, n_levels)
        ls = _lib.make_levelset(levelset)
        self._levelsets.append(ls)  # callbacks run during run()
        prm = _lib.cf_params()
        rid = ctypes.c_int64()
        check(self._lib.cf_server_submit(self._h, ctypes.byref(mesh), ctypes.byref(ls), degree,
                                         ctypes.byref(prm), rtol, maxit, float(arrival_s), ctypes.byref(rid)))
        return rid.value

    def run(self, stream=None):
        check(self._lib.cf_server_run(self._h, _stream(stream)))

    def result(self, rid):
        info = _lib.cf_info()
        times = np.zeros(3)
        nd = ctypes.c_int64()
        check(self._lib.cf_server_result(self._h, rid, ctypes.byref(info), times.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.byref(nd), None))
        out = {"iterations": info.iterations, "rel_residual": info.rel_residual,
               "true_rel_residual": info.true_rel_residual, "arrival": times[0], "admitted": times[1],
               "done": times[2], "latency_s": times[2] - times[0], "ndof": nd.value}
        if self.keep:
            x = np.empty(nd.value)
            check(self._lib.cf_server_result(self._h, rid, None, None, None, x.ctypes.data_as(ctypes.c_void_p)))
            out["x"] = x
        return out

    def stats(self):
        out = np.zeros(4)
        check(self._lib.cf_server_stats(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return {"peak_device_bytes": out[0], "peak_active": int(out[1]), "ticks": int(out[2]), "run_s": out[3]}
