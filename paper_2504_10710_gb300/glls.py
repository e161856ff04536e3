"""Python binding of the C ABI in ``include/glls.h`` (ctypes; argument
marshalling only).  Every step of the solver runs in ``libglls.so``; if the
library is missing this module raises instead of falling back to anything.

Device vectors are passed as torch CUDA tensors (their data pointers) and
streams as ``torch.cuda.Stream`` objects or raw handles.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libglls.so")

NOT_READY, OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_BREAKDOWN = 1, 0, -1, -2, -3, -4, -5
ERR_TIMEOUT, ERR_BUDGET = -6, -7
PREC_FP64, PREC_MIXED = 0, 1
SMOOTHER_GLL, SMOOTHER_FEM, SMOOTHER_GLL_BAND1 = 0, 1, 2
RESTRICT_TRANSPOSE, RESTRICT_INTERP = 0, 1
KRYLOV_FCG, KRYLOV_PCG, KRYLOV_GMRES = 0, 1, 2
COARSE_AUTO, COARSE_DENSE, COARSE_BLOCK_CR = 0, 1, 2
SUM_ATOMIC, SUM_COLORED = 0, 1


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nelem", C.c_int * 3), ("order", C.c_int),
                ("coords", C.POINTER(C.c_double)), ("smoother", C.c_int), ("restriction", C.c_int),
                ("device", C.c_int), ("coarse_solver", C.c_int), ("coarse_cr_levels", C.c_int),
                ("summation", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("gamma", C.c_int), ("m", C.c_int),
                ("alpha", C.c_double), ("precision", C.c_int), ("krylov", C.c_int), ("use_graph", C.c_int),
                ("check_every", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double), ("status", C.c_int), ("kernels", C.c_longlong),
                ("queue_ms", C.c_double), ("setup_kind", C.c_int), ("group", C.c_int)]


class Info(C.Structure):
    _fields_ = [("dim", C.c_int), ("levels", C.c_int), ("order", C.c_int * 8), ("nodes", (C.c_int * 3) * 8),
                ("ndof", C.c_longlong * 8), ("coarse_unknowns", C.c_longlong), ("device_bytes", C.c_size_t),
                ("coarse_cr_levels", C.c_int), ("coarse_dense_unknowns", C.c_longlong),
                ("instance_bytes", C.c_size_t), ("nrhs", C.c_int), ("setup_phase_ms", C.c_double * 6)]


class ServerInfo(C.Structure):
    _fields_ = [("submitted", C.c_ulonglong), ("completed", C.c_ulonglong), ("failed", C.c_ulonglong),
                ("queued", C.c_ulonglong), ("running", C.c_ulonglong), ("resident_bytes", C.c_size_t),
                ("budget_bytes", C.c_size_t), ("cached_problems", C.c_int), ("cached_instances", C.c_int),
                ("clones", C.c_ulonglong), ("grouped", C.c_ulonglong)]


class GllsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"glls status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(the solver has no fallback path)")
        L = C.CDLL(LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        sig = {
            "glls_gll": [i, C.POINTER(d), C.POINTER(d)],
            "glls_problem_create": [C.POINTER(MeshDesc), C.POINTER(vp)],
            "glls_problem_create_nrhs": [C.POINTER(MeshDesc), i, C.POINTER(vp)],
            "glls_problem_info": [vp, C.POINTER(Info)],
            "glls_problem_clone": [vp, C.POINTER(vp)],
            "glls_solve_batch_worklist": [C.POINTER(vp), i, C.POINTER(SolveOpts), C.POINTER(vp), i, vp,
                                          C.POINTER(Stats)],
            "glls_problem_clone_nrhs": [vp, C.c_int, C.POINTER(vp)],
            "glls_set_dirichlet": [vp, vp, i, vp],
            "glls_set_rhs": [vp, vp, i, vp],
            "glls_solve": [vp, C.POINTER(SolveOpts), vp, i, vp, C.POINTER(Stats)],
            "glls_lift_f64": [vp, vp, vp, vp, vp],
            "glls_restrict_noalloc_f32": [vp, i, vp, vp, vp, vp],
            "glls_solve_batch": [C.POINTER(vp), i, C.POINTER(SolveOpts), C.POINTER(vp), i, vp, C.POINTER(Stats)],
            "glls_estimate_bytes": [C.POINTER(MeshDesc), C.POINTER(C.c_size_t)],
            "glls_autotune": [vp, C.POINTER(C.c_int), C.POINTER(C.c_float)],
            "glls_server_create": [i, C.c_size_t, i, C.POINTER(vp)],
            "glls_submit": [vp, C.POINTER(MeshDesc), vp, vp, C.POINTER(SolveOpts), vp, C.POINTER(C.c_ulonglong)],
            "glls_poll": [vp, C.c_ulonglong, i, C.POINTER(Stats)],
            "glls_server_info_get": [vp, C.POINTER(ServerInfo)],
            "glls_cancel": [vp, C.c_ulonglong],
            "glls_server_register": [vp, C.POINTER(MeshDesc), C.POINTER(C.c_ulonglong)],
            "glls_server_set_max_group": [vp, C.c_int],
            "glls_submit_mesh": [vp, C.c_ulonglong, vp, vp, C.POINTER(SolveOpts), vp, C.POINTER(C.c_ulonglong)],
            "glls_apply_partials_f64": [vp, i, vp, vp, vp, i, C.POINTER(i), vp],
            "glls_apply_partials_ff": [vp, i, vp, vp, vp, i, C.POINTER(i), vp],
        }
        for suf, real in (("f64", d), ("f32", C.c_float)):
            sig[f"glls_apply_{suf}"] = [vp, i, vp, vp, vp]
            sig[f"glls_apply_multi_{suf}"] = [vp, i, vp, vp, i, vp]
            sig[f"glls_line_solve_{suf}"] = [vp, i, i, vp, vp, vp]
            sig[f"glls_smooth_{suf}"] = [vp, i, i, real, vp, vp, vp]
            sig[f"glls_line_update_{suf}"] = [vp, i, i, real, vp, vp, vp, vp]
            sig[f"glls_restrict_{suf}"] = [vp, i, vp, vp, vp, vp]
            sig[f"glls_prolong_add_{suf}"] = [vp, i, vp, vp, vp]
            sig[f"glls_coarse_solve_{suf}"] = [vp, vp, vp, vp]
            sig[f"glls_precondition_{suf}"] = [vp, C.POINTER(SolveOpts), vp, vp, vp]
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.glls_debug_fail_alloc_after.argtypes = [C.c_longlong]
        L.glls_debug_fail_alloc_after.restype = None
        L.glls_problem_destroy.argtypes = [vp]
        L.glls_problem_destroy.restype = None
        L.glls_server_destroy.argtypes = [vp]
        L.glls_server_destroy.restype = None
        L.glls_last_error.argtypes = []
        L.glls_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise GllsError(status, lib().glls_last_error().decode())
    return status


def _ptr(t):
    """Data pointer of a torch tensor (or None)."""
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def gll(p: int):
    xi = (C.c_double * (p + 1))()
    rho = (C.c_double * (p + 1))()
    _check(lib().glls_gll(p, xi, rho))
    return np.array(xi[:]), np.array(rho[:])


def opts(tol=1e-10, max_iter=200, gamma=1, m=1, alpha=0.5, precision=PREC_MIXED, krylov=KRYLOV_FCG,
         use_graph=2, check_every=1) -> SolveOpts:
    return SolveOpts(tol, max_iter, gamma, m, alpha, precision, krylov, use_graph, check_every)


class Problem:
    """Owns a ``glls_problem``: mesh levels resident on the device."""

    def __init__(self, dim, nelem, order, coords, smoother=SMOOTHER_GLL, restriction=RESTRICT_TRANSPOSE,
                 device=0, coarse_solver=COARSE_AUTO, coarse_cr_levels=0, nrhs=1, summation=SUM_ATOMIC):
        desc, coords = mesh_desc(dim, nelem, order, coords, smoother, restriction, device, coarse_solver,
                                 coarse_cr_levels, summation)
        self._coords = coords
        h = C.c_void_p()
        _check(lib().glls_problem_create_nrhs(C.byref(desc), nrhs, C.byref(h)))
        self.h = h
        self.nrhs = nrhs
        self.dim = dim
        self.info = self._info()
        self.N = int(self.info.ndof[self.info.levels - 1])

    def clone(self, nrhs=None):
        """A problem on the same mesh sharing its read-only device data (with
        nrhs right-hand sides; default: as this one)."""
        h = C.c_void_p()
        nrhs = self.nrhs if nrhs is None else nrhs
        _check(lib().glls_problem_clone_nrhs(self.h, nrhs, C.byref(h)))
        c = Problem.__new__(Problem)
        c.h, c.dim, c._coords, c.nrhs = h, self.dim, self._coords, nrhs
        c.info = c._info()
        c.N = self.N
        return c

    def _info(self):
        inf = Info()
        _check(lib().glls_problem_info(self.h, C.byref(inf)))
        return inf

    @property
    def levels(self):
        return self.info.levels

    def level_shape(self, level):
        n = self.info.nodes[level]
        return tuple(n[a] for a in reversed(range(self.dim)))

    def close(self):
        if getattr(self, "h", None):
            lib().glls_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- data ------------------------------------------------------------
    def set_rhs(self, f, stream=None):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
            _check(lib().glls_set_rhs(self.h, f.ctypes.data_as(C.c_void_p), 0, _stream(stream)))
        else:
            _check(lib().glls_set_rhs(self.h, _ptr(f), 1, _stream(stream)))

    def set_dirichlet(self, g, stream=None):
        if isinstance(g, np.ndarray):
            g = np.ascontiguousarray(g, dtype=np.float64)
            _check(lib().glls_set_dirichlet(self.h, g.ctypes.data_as(C.c_void_p), 0, _stream(stream)))
        else:
            _check(lib().glls_set_dirichlet(self.h, _ptr(g), 1, _stream(stream)))

    def solve(self, out, o: SolveOpts, stream=None, raise_on_error=True):
        """Solve into ``out`` (numpy float64 host array or torch CUDA float64
        tensor of nrhs x N values).  Returns the Stats structure (a list of
        nrhs of them when nrhs > 1)."""
        st = (Stats * self.nrhs)()
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == self.N * self.nrhs
            status = lib().glls_solve(self.h, C.byref(o), out.ctypes.data_as(C.c_void_p), 0, _stream(stream), st)
        else:
            assert out.numel() == self.N * self.nrhs
            status = lib().glls_solve(self.h, C.byref(o), _ptr(out), 1, _stream(stream), st)
        if raise_on_error:
            _check(status)
        return st[0] if self.nrhs == 1 else list(st)

    def autotune(self):
        """Pick the lines per CTA of the line solve per level/precision/direction
        by timing (line blocks: 0 = the launch heuristic, or 1..16; band-1:
        2..16); returns {(level, 'f32'|'f64', axis): (choice, us_per_launch)}."""
        n = self.levels * 2 * 3
        ch = (C.c_int * n)()
        us = (C.c_float * n)()
        _check(lib().glls_autotune(self.h, ch, us))
        out = {}
        for l in range(1, self.levels):
            for pi, pn in enumerate(("f32", "f64")):
                for a in range(self.dim):
                    k = (l * 2 + pi) * 3 + a
                    out[(l, pn, a)] = (ch[k], us[k])
        return out

    # ---- level operations (device tensors) -------------------------------
    @staticmethod
    def _suffix(t):
        import torch
        return "f64" if t.dtype == torch.float64 else "f32"

    def apply(self, level, x, y, stream=None):
        _check(getattr(lib(), f"glls_apply_{self._suffix(x)}")(self.h, level, _ptr(x), _ptr(y), _stream(stream)))

    def apply_multi(self, level, x, y, nrhs, stream=None):
        """y = A_l x for nrhs stacked vectors in one launch."""
        _check(getattr(lib(), f"glls_apply_multi_{self._suffix(x)}")(self.h, level, _ptr(x), _ptr(y), nrhs,
                                                                      _stream(stream)))

    def apply_partials(self, level, x, y, partials, stream=None, ff=False):
        """FP64 y += A x with the fused per-CTA x.(A x) partials (y zero on
        entry); returns the number of partials written.  ff=True: the
        float-float form the mixed-precision outer iteration runs."""
        n = C.c_int()
        fn = lib().glls_apply_partials_ff if ff else lib().glls_apply_partials_f64
        _check(fn(self.h, level, _ptr(x), _ptr(y), _ptr(partials), partials.numel(), C.byref(n), _stream(stream)))
        return n.value

    def line_solve(self, level, axis, g, x, stream=None):
        _check(getattr(lib(), f"glls_line_solve_{self._suffix(g)}")(self.h, level, axis, _ptr(g), _ptr(x),
                                                                       _stream(stream)))

    def smooth(self, level, axis, alpha, r, x, stream=None):
        _check(getattr(lib(), f"glls_smooth_{self._suffix(r)}")(self.h, level, axis, alpha, _ptr(r), _ptr(x),
                                                                   _stream(stream)))

    def line_update(self, level, axis, alpha, r, y, x, stream=None):
        """x += alpha B_s^-1 (r - y) (the smoothing step's line update after
        y = A x); y's element-boundary entries are reset to 0."""
        _check(getattr(lib(), f"glls_line_update_{self._suffix(r)}")(self.h, level, axis, alpha, _ptr(r), _ptr(y),
                                                                        _ptr(x), _stream(stream)))

    def restrict(self, level, r, x, rc, stream=None):
        _check(getattr(lib(), f"glls_restrict_{self._suffix(r)}")(self.h, level, _ptr(r), _ptr(x), _ptr(rc),
                                                                     _stream(stream)))

    def prolong_add(self, level, e, x, stream=None):
        _check(getattr(lib(), f"glls_prolong_add_{self._suffix(e)}")(self.h, level, _ptr(e), _ptr(x),
                                                                        _stream(stream)))

    def coarse_solve(self, r, e, stream=None):
        _check(getattr(lib(), f"glls_coarse_solve_{self._suffix(r)}")(self.h, _ptr(r), _ptr(e), _stream(stream)))

    def precondition(self, o: SolveOpts, r, z, stream=None):
        _check(getattr(lib(), f"glls_precondition_{self._suffix(r)}")(self.h, C.byref(o), _ptr(r), _ptr(z),
                                                                         _stream(stream)))

    def lift(self, f, g, f0, stream=None):
        _check(lib().glls_lift_f64(self.h, _ptr(f), _ptr(g), _ptr(f0), _stream(stream)))


def solve_batch(problems, outs, o: SolveOpts, stream=None, raise_on_error=True, worklist=False):
    """Solve several problems in one graph launch; outs: numpy host arrays
    (or torch CUDA float64 tensors), one per problem.  worklist=True: the
    work-list kernels (glls_solve_batch_worklist), else one graph branch per
    problem.  Returns the stats."""
    n = len(problems)
    hs = (C.c_void_p * n)(*[p.h.value for p in problems])
    on_device = 0 if isinstance(outs[0], np.ndarray) else 1
    ptrs = (C.c_void_p * n)(*[(o_.ctypes.data if on_device == 0 else o_.data_ptr()) for o_ in outs])
    st = (Stats * n)()
    fn = lib().glls_solve_batch_worklist if worklist else lib().glls_solve_batch
    status = fn(hs, n, C.byref(o), ptrs, on_device, _stream(stream), st)
    if raise_on_error:
        _check(status)
    return list(st)


def solve_multi(problem, F, g, o: SolveOpts, clones=None):
    """Several right-hand sides on one mesh: F has shape (nrhs, N); g is the
    Dirichlet data (shared).  The RHS are solved together, as clones of
    `problem` sharing its mesh data, in one glls_solve_batch launch.
    Returns (U of shape (nrhs, N), stats, clones) - pass the clones back to
    reuse them (and the cached batch graph)."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    nrhs = F.shape[0]
    probs = [problem] + (clones if clones is not None else [problem.clone() for _ in range(nrhs - 1)])
    for p, f in zip(probs, F):
        p.set_rhs(f)
        p.set_dirichlet(g)
    U = np.zeros((nrhs, problem.N))
    stats = solve_batch(probs, list(U), o)
    return U, stats, probs[1:]


def mesh_desc(dim, nelem, order, coords, smoother=SMOOTHER_GLL, restriction=RESTRICT_TRANSPOSE, device=0,
              coarse_solver=COARSE_AUTO, coarse_cr_levels=0, summation=SUM_ATOMIC):
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    ne = (C.c_int * 3)(*(list(nelem) + [1] * (3 - len(nelem))))
    return MeshDesc(dim, ne, order, coords.ctypes.data_as(C.POINTER(C.c_double)), smoother, restriction,
                    device, coarse_solver, coarse_cr_levels, summation), coords


def estimate_bytes(dim, nelem, order, coords, coarse_solver=COARSE_AUTO, coarse_cr_levels=0):
    desc, _keep = mesh_desc(dim, nelem, order, coords, coarse_solver=coarse_solver, coarse_cr_levels=coarse_cr_levels)
    out = C.c_size_t()
    _check(lib().glls_estimate_bytes(C.byref(desc), C.byref(out)))
    return out.value


class Server:
    """Request loop with admission by HBM budget (native, see glls_submit)."""

    def __init__(self, budget_bytes, slots=4, device=0):
        h = C.c_void_p()
        _check(lib().glls_server_create(device, budget_bytes, slots, C.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, dim, nelem, order, coords, f, g, o: SolveOpts, out, smoother=SMOOTHER_GLL,
               restriction=RESTRICT_TRANSPOSE, summation=SUM_ATOMIC):
        desc, coords = mesh_desc(dim, nelem, order, coords, smoother, restriction, summation=summation)
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
        assert out.dtype == np.float64 and out.flags.c_contiguous
        t = C.c_ulonglong()
        _check(lib().glls_submit(self.h, C.byref(desc), f.ctypes.data_as(C.c_void_p),
                                 None if g is None else g.ctypes.data_as(C.c_void_p), C.byref(o),
                                 out.ctypes.data_as(C.c_void_p), C.byref(t)))
        self._keep[t.value] = out          # the output buffer must outlive the request
        return t.value

    def set_max_group(self, k):
        """Solve up to k queued requests of one mesh together (see glls_server_set_max_group)."""
        _check(lib().glls_server_set_max_group(self.h, k))

    def register(self, dim, nelem, order, coords, smoother=SMOOTHER_GLL, restriction=RESTRICT_TRANSPOSE,
                 summation=SUM_ATOMIC):
        """Registers a mesh; returns its id for submit_mesh."""
        desc, coords = mesh_desc(dim, nelem, order, coords, smoother, restriction, summation=summation)
        mid = C.c_ulonglong()
        _check(lib().glls_server_register(self.h, C.byref(desc), C.byref(mid)))
        return mid.value

    def submit_mesh(self, mesh_id, f, g, o: SolveOpts, out):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
        assert out.dtype == np.float64 and out.flags.c_contiguous
        t = C.c_ulonglong()
        _check(lib().glls_submit_mesh(self.h, mesh_id, f.ctypes.data_as(C.c_void_p),
                                      None if g is None else g.ctypes.data_as(C.c_void_p), C.byref(o),
                                      out.ctypes.data_as(C.c_void_p), C.byref(t)))
        self._keep[t.value] = (out, f, g)        # read by the request when it runs
        return t.value

    def poll(self, ticket, wait=False):
        """(status, stats) or (NOT_READY, None)."""
        st = Stats()
        status = lib().glls_poll(self.h, ticket, 1 if wait else 0, C.byref(st))
        if status == NOT_READY:
            return status, None
        self._keep.pop(ticket, None)
        return status, st

    def info(self):
        inf = ServerInfo()
        _check(lib().glls_server_info_get(self.h, C.byref(inf)))
        return inf

    def cancel(self, ticket):
        """OK (removed before it ran), NOT_READY (already running) or ERR_INVALID."""
        status = lib().glls_cancel(self.h, ticket)
        if status == OK:
            self._keep.pop(ticket, None)
        return status

    def close(self):
        if getattr(self, "h", None):
            lib().glls_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def problem_for(workload, smoother=SMOOTHER_GLL, restriction=RESTRICT_TRANSPOSE, device=0,
                coarse_solver=COARSE_AUTO, coarse_cr_levels=0, nrhs=1, summation=SUM_ATOMIC):
    """Problem of a workload description, with nodes placed at the library's
    own GLL points."""
    xi, _ = gll(workload.order)
    coords = workload.coords(xi)
    return Problem(workload.dim, workload.nelem, workload.order, coords, smoother, restriction, device,
                   coarse_solver, coarse_cr_levels, nrhs, summation), coords
