"""Thin ctypes binding of the C ABI in include/st_iga.h (libst_iga.so).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Device vectors are torch tensors (float64, contiguous, on the
CUDA device); their pointers are passed as-is.  The library is loaded
in-tree from this package directory; ``load()`` raises if it is missing.
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libst_iga.so")

ST_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "NOT_POSITIVE", -4: "ILL_CONDITIONED",
          -5: "NO_CONVERGENCE", -6: "TIMEOUT", -7: "CUDA", -8: "OVER_BUDGET",
          -9: "UNSUPPORTED", -10: "NOT_READY", -11: "CANCELLED", -12: "COMM"}
ST_ERR_INVALID_ARG = -1
ST_ERR_NO_CONVERGENCE = -5
ST_ERR_UNSUPPORTED = -9
GEOMETRY = {1: 1, 2: 2, 3: 3}
PRECISION = {"fp64": 0, "mixed_fp32": 1, "mixed_tf32": 2, "mixed_bf16": 3}
OUTER = {"fgmres": 0, "mg": 1, "ir": 2}
BASIS = {"nodal": 0, "spectral": 1}
VARIANT = {"rschur": 0, "eig": 1, "cschur": 2}
SPATIAL = {"fd": 0, "minres": 1}

# every symbol declared in include/st_iga.h
SYMBOLS = ["st_options_default", "st_setup", "st_setup_host", "st_destroy", "st_set_stream",
           "st_sizes", "st_apply", "st_residual", "st_residual_df", "st_load_coeffs", "st_load_gaussians", "st_smooth",
           "st_smooth_static", "st_set_wait_limit", "st_block_minres", "st_vcycle",
           "st_solve", "st_autotune", "st_profile", "st_profile_read", "st_time_factors", "st_time_spectrum", "st_space_factors",
           "st_time_prolongation", "st_level_shape", "st_space_prolongation", "st_last_error", "st_serve_opts_default", "st_serve_start",
           "st_serve_submit", "st_serve_resume", "st_serve_pause", "st_serve_cancel", "st_serve_poll", "st_serve_wait",
           "st_serve_stop", "st_setup_partitioned", "st_partition_plan", "st_comm_nccl_unique_id",
           "st_comm_nccl_create", "st_comm_nccl_destroy", "st_solve_history", "st_solve_host",
           "st_solve_group"]
PROF_CLASSES = ["stencil64", "stencil32", "gemm64", "gemm32", "shift", "update", "transfer",
                "vector", "dot", "tc", "spec", "stencil_df", "minres"]


class StOptions(ctypes.Structure):
    _fields_ = [("T", ctypes.c_double), ("theta", ctypes.c_double), ("omega", ctypes.c_double),
                ("ne_per_slab", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("precision", ctypes.c_int), ("outer", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("max_it", ctypes.c_int),
                ("nrhs", ctypes.c_int), ("hbm_budget", ctypes.c_size_t), ("basis", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("use_graphs", ctypes.c_int),
                ("variant", ctypes.c_int), ("autotune", ctypes.c_int),
                ("fused_vcycle", ctypes.c_int), ("spatial_solver", ctypes.c_int),
                ("minres_tol", ctypes.c_double), ("minres_maxit", ctypes.c_int),
                ("space_ratio", ctypes.c_double)]


class StSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("host_syncs", ctypes.c_int), ("vector_launches", ctypes.c_int)]


class StServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("workers", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("opt", StOptions), ("start_paused", ctypes.c_int),
                ("batch_dofs", ctypes.c_longlong), ("group_members", ctypes.c_int)]


class StRequest(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int), ("degree", ctypes.c_int),
                ("spans", ctypes.c_int * 3), ("slabs", ctypes.c_int),
                ("rhs", ctypes.POINTER(ctypes.c_double)), ("rhs_is_coeffs", ctypes.c_int),
                ("tol", ctypes.c_double)]


class StResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("refinements", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("queue_seconds", ctypes.c_double), ("solve_seconds", ctypes.c_double),
                ("latency_seconds", ctypes.c_double), ("batch_size", ctypes.c_int),
                ("n_dofs", ctypes.c_int64), ("error", ctypes.c_char * 128),
                ("group_requests", ctypes.c_int), ("host_syncs", ctypes.c_int),
                ("vector_launches", ctypes.c_int)]


ST_ERR_NOT_READY = -10

# st_comm callbacks (slab-partitioned handles)
SENDRECV_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                               ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p)
ALLGATHER_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_size_t, ctypes.c_void_p)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                ctypes.c_size_t)


class StComm(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int), ("size", ctypes.c_int), ("host_buffers", ctypes.c_int),
                ("ctx", ctypes.c_void_p), ("sendrecv", SENDRECV_FN),
                ("allgather", ALLGATHER_FN), ("allreduce_sum", ALLREDUCE_FN)]


class StError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


_lib = None


def load():
    """Load libst_iga.so (in-tree).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libst_iga.so is missing: run __graft_entry__.build() or "
                           "python paper_1802_09277_gb300/build.py first")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    ip = ctypes.POINTER(ctypes.c_int)
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "st_options_default": (V, [ctypes.POINTER(StOptions)]),
        "st_setup": (I, [ctypes.POINTER(P), I, I, ip, I, ctypes.POINTER(StOptions), P]),
        "st_setup_host": (I, [ctypes.POINTER(P), I, I, ip, I, ctypes.POINTER(StOptions)]),
        "st_destroy": (V, [P]),
        "st_set_stream": (I, [P, P]),
        "st_sizes": (I, [P, ctypes.POINTER(ctypes.c_int64), ip, ip, ip,
                         ctypes.POINTER(ctypes.c_size_t)]),
        "st_apply": (I, [P, P, P]),
        "st_residual": (I, [P, P, P, P]),
        "st_residual_df": (I, [P, P, P, P, I]),
        "st_load_coeffs": (I, [P, P, P]),
        "st_load_gaussians": (I, [P, I, dp, dp, dp, P]),
        "st_smooth": (I, [P, P, P, I]),
        "st_smooth_static": (I, [P, P, P, I, P]),
        "st_block_minres": (I, [P, D, D, D, P, P, I, D, I, ip, dp]),
        "st_vcycle": (I, [P, P, P]),
        "st_level_shape": (I, [P, I, ip, ip, ip]),
        "st_space_prolongation": (I, [P, I, I, ip, ip, dp]),
        "st_solve": (I, [P, P, D, P, I, ctypes.POINTER(StSolveInfo)]),
        "st_solve_host": (I, [P, I, P, D, P, I, ctypes.POINTER(StSolveInfo)]),
        "st_solve_group": (I, [I, ctypes.POINTER(P), ctypes.POINTER(P), D, ctypes.POINTER(P), I,
                               ctypes.POINTER(StSolveInfo)]),
        "st_autotune": (I, [P, ip, dp]),
        "st_profile": (I, [P, I]),
        "st_profile_read": (I, [P, I, ctypes.POINTER(ctypes.c_int64), dp, dp, dp]),
        "st_time_factors": (I, [P, I, ip, dp, dp, dp, dp, dp]),
        "st_time_spectrum": (I, [P, I, dp, dp, dp]),
        "st_space_factors": (I, [P, I, ip, dp, dp, dp, dp]),
        "st_time_prolongation": (I, [P, ip, dp]),
        "st_last_error": (ctypes.c_char_p, []),
        "st_serve_opts_default": (V, [ctypes.POINTER(StServerOpts)]),
        "st_serve_start": (I, [ctypes.POINTER(P), ctypes.POINTER(StServerOpts)]),
        "st_serve_submit": (I, [P, ctypes.POINTER(StRequest), ctypes.POINTER(ctypes.c_uint64)]),
        "st_set_wait_limit": (I, [P, D]),
        "st_serve_resume": (I, [P]),
        "st_serve_pause": (I, [P]),
        "st_serve_cancel": (I, [P, ctypes.c_uint64]),
        "st_serve_poll": (I, [P, ctypes.c_uint64, ctypes.POINTER(StResult), dp]),
        "st_serve_wait": (I, [P, ctypes.c_uint64, D, ctypes.POINTER(StResult), dp]),
        "st_serve_stop": (I, [P]),
        "st_solve_history": (I, [P, I, ip, dp, ip]),
        "st_setup_partitioned": (I, [ctypes.POINTER(P), I, I, ip, I, ctypes.POINTER(StOptions),
                                     ctypes.POINTER(StComm), P]),
        "st_partition_plan": (I, [I, I, I, ip, ip, ip]),
        "st_comm_nccl_unique_id": (I, [P]),
        "st_comm_nccl_create": (I, [ctypes.POINTER(StComm), I, I, P]),
        "st_comm_nccl_destroy": (V, [ctypes.POINTER(StComm)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != ST_OK:
        raise StError(rc, _lib.st_last_error().decode())


def options(**kw):
    """st_options with defaults, overridden by keyword (precision/outer may be
    given by name)."""
    lib = load()
    o = StOptions()
    lib.st_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k == "outer" and isinstance(v, str):
            v = OUTER[v]
        if k == "basis" and isinstance(v, str):
            v = BASIS[v]
        if k == "variant" and isinstance(v, str):
            v = VARIANT[v]
        if k == "spatial_solver" and isinstance(v, str):
            v = SPATIAL[v]
        setattr(o, k, v)
    return o


def _dptr(t, n, name):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
    if t.numel() != n:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), n))
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One handle of the library: geometry 1/2/3 (interval/square/cube),
    degree p, spans per axis, slabs; keyword options as in st_options.
    host_only=True builds only the FP64 factors (no GPU needed)."""

    def __init__(self, dim, degree, spans, slabs, host_only=False, stream=None, comm=None,
                 **opts):
        lib = load()
        self.dim = int(dim)
        self.opt = options(**opts)
        self._h = ctypes.c_void_p()
        self._comm = comm  # kept alive with the handle (its callbacks)
        sp = (ctypes.c_int * 3)(*([int(s) for s in spans] + [1] * (3 - len(spans))))
        if comm is not None:
            # slabs = the global slab count; this rank holds its own range
            if stream is None:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            rc = lib.st_setup_partitioned(ctypes.byref(self._h), self.dim, int(degree), sp,
                                          int(slabs), ctypes.byref(self.opt),
                                          ctypes.byref(comm.c), ctypes.c_void_p(stream))
        elif host_only:
            rc = lib.st_setup_host(ctypes.byref(self._h), self.dim, int(degree), sp, int(slabs),
                                   ctypes.byref(self.opt))
        else:
            if stream is None:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            rc = lib.st_setup(ctypes.byref(self._h), self.dim, int(degree), sp, int(slabs),
                              ctypes.byref(self.opt), ctypes.c_void_p(stream))
        _check(rc)
        n = ctypes.c_int64()
        nt = ctypes.c_int()
        nx = (ctypes.c_int * 3)()
        nl = ctypes.c_int()
        nb = ctypes.c_size_t()
        _check(lib.st_sizes(self._h, ctypes.byref(n), ctypes.byref(nt), nx, ctypes.byref(nl),
                            ctypes.byref(nb)))
        self.ndofs, self.nt, self.nx = n.value, nt.value, tuple(nx)
        self.nlevels, self.device_bytes = nl.value, nb.value

    def close(self):
        if self._h:
            _lib.st_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(_lib.st_set_stream(self._h, ctypes.c_void_p(stream)))

    def apply(self, x, y):
        _check(_lib.st_apply(self._h, _dptr(x, self.ndofs, "x"), _dptr(y, self.ndofs, "y")))

    def residual(self, u, f, r):
        _check(_lib.st_residual(self._h, _dptr(u, self.ndofs, "u"), _dptr(f, self.ndofs, "f"),
                                _dptr(r, self.ndofs, "r")))

    def residual_df(self, u, f, r, slabs_per_cta=0):
        """The refinement's double-float residual r = f - L u (FP64 data);
        slabs_per_cta 0 (library's choice), 1, 2, 4 or 8."""
        _check(_lib.st_residual_df(self._h, _dptr(u, self.ndofs, "u"), _dptr(f, self.ndofs, "f"),
                                   _dptr(r, self.ndofs, "r"), int(slabs_per_cta)))

    def load_coeffs(self, c, f):
        _check(_lib.st_load_coeffs(self._h, _dptr(c, self.ndofs, "c"), _dptr(f, self.ndofs, "f")))

    def load_gaussians(self, centers, widths, amps, f):
        import numpy as np
        c = np.ascontiguousarray(centers, dtype=np.float64)
        w = np.ascontiguousarray(widths, dtype=np.float64)
        a = np.ascontiguousarray(amps, dtype=np.float64)
        dpp = lambda z: z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(_lib.st_load_gaussians(self._h, len(w), dpp(c), dpp(w), dpp(a),
                                      _dptr(f, self.ndofs, "f")))

    def smooth(self, u, f, nsteps=1):
        _check(_lib.st_smooth(self._h, _dptr(u, self.ndofs, "u"), _dptr(f, self.ndofs, "f"),
                              int(nsteps)))

    def smooth_static(self, u, f, nsteps=1, stream=None):
        """FP64 smoothing steps with the library's static device work space
        (no device allocation; works on a host_only handle)."""
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        _check(_lib.st_smooth_static(self._h, _dptr(u, self.ndofs, "u"),
                                     _dptr(f, self.ndofs, "f"), int(nsteps),
                                     ctypes.c_void_p(stream)))

    def block_minres(self, alpha, beta1, beta2, f, u, tol=1e-10, maxit=0, check=True):
        """MinRes on nsys spatial 2x2 block systems (Theorem 3.3; a complex
        shift alpha + i beta is beta1 = -beta, beta2 = beta).  f, u: float64
        CUDA tensors of nsys * 2 * n_x elements ([sys][f, g][space]).
        Returns (iterations, relative P^{-1}-residuals, return code) per system."""
        import numpy as np
        m = int(np.prod(self.nx))
        nsys = f.numel() // (2 * m)
        if nsys * 2 * m != f.numel() or nsys < 1:
            raise ValueError("f must hold nsys * 2 * n_x elements")
        its = (ctypes.c_int * nsys)()
        rel = (ctypes.c_double * nsys)()
        rc = _lib.st_block_minres(self._h, float(alpha), float(beta1), float(beta2),
                                  _dptr(f, nsys * 2 * m, "f"), _dptr(u, nsys * 2 * m, "u"),
                                  int(nsys), float(tol), int(maxit), its, rel)
        if check:
            _check(rc)
        return np.array(its[:]), np.array(rel[:]), rc

    def vcycle(self, u, f):
        _check(_lib.st_vcycle(self._h, _dptr(u, self.ndofs, "u"), _dptr(f, self.ndofs, "f")))

    def solve(self, rhs, u, tol=1e-8, use_guess=False, check=True):
        info = StSolveInfo()
        rc = _lib.st_solve(self._h, _dptr(rhs, self.ndofs, "rhs"), float(tol),
                           _dptr(u, self.ndofs, "u"), int(bool(use_guess)), ctypes.byref(info))
        if check:
            _check(rc)
        return {"iterations": info.iterations, "refinements": info.refinements,
                "status": info.status,
                "rel_residual": info.rel_residual, "seconds": info.seconds,
                "host_syncs": info.host_syncs, "vector_launches": info.vector_launches, "rc": rc}

    def solve_host(self, rhs, u, tol=1e-8, use_guess=False, check=True):
        """st_solve_host: rhs and u are contiguous float64 CPU tensors of
        nbatch x ndofs values (pinned memory lets the copies overlap the
        solves); nbatch = rhs.numel() // ndofs."""
        import torch
        for t, name in ((rhs, "rhs"), (u, "u")):
            if not isinstance(t, torch.Tensor):
                raise TypeError("%s must be a torch tensor" % name)
            if t.dtype != torch.float64 or t.is_cuda or not t.is_contiguous():
                raise ValueError("%s must be a contiguous float64 CPU tensor" % name)
        if rhs.numel() == 0 or rhs.numel() % self.ndofs or u.numel() != rhs.numel():
            raise ValueError("rhs and u must hold the same whole number of batches of %d values"
                             % self.ndofs)
        info = StSolveInfo()
        rc = _lib.st_solve_host(self._h, rhs.numel() // self.ndofs,
                                ctypes.c_void_p(rhs.data_ptr()), float(tol),
                                ctypes.c_void_p(u.data_ptr()), int(bool(use_guess)),
                                ctypes.byref(info))
        if check:
            _check(rc)
        return {"iterations": info.iterations, "refinements": info.refinements,
                "status": info.status, "rel_residual": info.rel_residual,
                "seconds": info.seconds, "host_syncs": info.host_syncs,
                "vector_launches": info.vector_launches, "rc": rc}

    def set_wait_limit(self, seconds):
        """Bound of the tensor-core kernels' device-side waits (seconds)."""
        _check(_lib.st_set_wait_limit(self._h, float(seconds)))

    def history(self):
        """[(iterations, relative residual)] of the last solve."""
        n = ctypes.c_int()
        _check(_lib.st_solve_history(self._h, 0, None, None, ctypes.byref(n)))
        its = (ctypes.c_int * max(n.value, 1))()
        res = (ctypes.c_double * max(n.value, 1))()
        _check(_lib.st_solve_history(self._h, n.value, its, res, ctypes.byref(n)))
        return [(its[i], res[i]) for i in range(n.value)]

    def autotune(self):
        """Per axis: (choice, ms per pass); choice 0 = CUDA cores, k > 0 =
        tensor cores with k CTAs per SM."""
        ch = (ctypes.c_int * 3)()
        ms = (ctypes.c_double * 3)()
        _check(_lib.st_autotune(self._h, ch, ms))
        return [(ch[a], ms[a]) for a in range(self.dim)]

    def profile(self, enable):
        """Start (reset) or stop per-kernel-class event timing."""
        _check(_lib.st_profile(self._h, int(bool(enable))))

    def profile_read(self):
        """{class: {launches, ms, bytes, flops}} accumulated since profile(True)."""
        out = {}
        for c, name in enumerate(PROF_CLASSES):
            n = ctypes.c_int64()
            ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            _check(_lib.st_profile_read(self._h, c, ctypes.byref(n), ctypes.byref(ms),
                                        ctypes.byref(by), ctypes.byref(fl)))
            out[name] = {"launches": n.value, "ms": ms.value, "bytes": by.value,
                         "flops": fl.value}
        return out

    # host-side factor inspection -------------------------------------------
    def time_factors(self, level=0):
        import numpy as np
        nt = self.nt
        mats = [np.zeros((nt, nt)) for _ in range(5)]
        ptrs = [m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for m in mats]
        k = ctypes.c_int()
        _check(_lib.st_time_factors(self._h, int(level), ctypes.byref(k), *ptrs))
        return dict(zip(["Kt", "Mt", "X", "Z", "Y"], mats))

    def time_spectrum(self, level=0):
        """(eigenvalues (complex array), cond2 of the unit-column eigenvectors)."""
        import numpy as np
        re, im = np.zeros(self.nt), np.zeros(self.nt)
        c = ctypes.c_double()
        dpp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(_lib.st_time_spectrum(self._h, int(level), dpp(re), dpp(im), ctypes.byref(c)))
        return re + 1j * im, c.value

    def space_factors(self, axis=0):
        import numpy as np
        n = self.nx[axis]
        M1, K1, U = (np.zeros((n, n)) for _ in range(3))
        lam = np.zeros(n)
        cp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        k = ctypes.c_int()
        _check(_lib.st_space_factors(self._h, int(axis), ctypes.byref(k), cp(M1), cp(K1), cp(U),
                                     cp(lam)))
        return {"M1": M1, "K1": K1, "U": U, "lam": lam}

    def level_shapes(self):
        """[(slabs, spans (d entries), 'x' | 't' | '-') per level]: the step
        from the previous level ('-' on level 0)."""
        out = []
        for lvl in range(self.nlevels):
            n = ctypes.c_int()
            sp = (ctypes.c_int * 3)()
            x = ctypes.c_int()
            _check(_lib.st_level_shape(self._h, lvl, ctypes.byref(n), sp, ctypes.byref(x)))
            out.append((n.value, tuple(sp[:self.dim]), "-" if lvl == 0 else ("x" if x.value else "t")))
        return out

    def space_prolongation(self, level, axis):
        """The 1D knot-insertion matrix (n_f x n_c) of axis `axis` between
        level `level` and the space-coarsened level after it."""
        import numpy as np
        nf, nc = ctypes.c_int(), ctypes.c_int()
        _check(_lib.st_space_prolongation(self._h, int(level), int(axis), ctypes.byref(nf),
                                          ctypes.byref(nc), None))
        P = np.zeros((nf.value, nc.value))
        _check(_lib.st_space_prolongation(self._h, int(level), int(axis), None, None,
                                          P.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return P

    def time_prolongation(self):
        import numpy as np
        P = np.zeros((2 * self.nt, self.nt))
        k = ctypes.c_int()
        _check(_lib.st_time_prolongation(self._h, ctypes.byref(k),
                                         P.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return P


def solve_group(solvers, rhs, u, tol=1e-8, use_guess=False, check=True):
    """st_solve_group: solve the problems of several Solver handles together
    (one launch per Krylov vector operation over all their right-hand sides);
    rhs[k], u[k] are member k's device vectors.  Returns one info dict per
    member."""
    n = len(solvers)
    if n == 0 or len(rhs) != n or len(u) != n:
        raise ValueError("one rhs and one u per solver")
    P = ctypes.c_void_p
    hs = (P * n)(*[s._h for s in solvers])
    rp = (P * n)(*[_dptr(r, s.ndofs, "rhs") for s, r in zip(solvers, rhs)])
    up = (P * n)(*[_dptr(x, s.ndofs, "u") for s, x in zip(solvers, u)])
    infos = (StSolveInfo * n)()
    rc = _lib.st_solve_group(n, hs, rp, float(tol), up, int(bool(use_guess)), infos)
    if check:
        _check(rc)
    return [{"iterations": i.iterations, "refinements": i.refinements, "status": i.status,
             "rel_residual": i.rel_residual, "seconds": i.seconds, "host_syncs": i.host_syncs,
             "vector_launches": i.vector_launches, "rc": rc} for i in infos]


class Server:
    """Continuous-batching solve server (st_serve_*): submit host right-hand
    sides of any configuration, poll or wait for host solutions."""

    def __init__(self, workers=4, max_batch=8, hbm_budget=0, paused=False, batch_dofs=None,
                 group_members=None, **opts):
        lib = load()
        self.o = StServerOpts()
        lib.st_serve_opts_default(ctypes.byref(self.o))
        self.o.workers = int(workers)
        self.o.max_batch = int(max_batch)
        self.o.hbm_budget = int(hbm_budget)
        self.o.start_paused = 1 if paused else 0
        if batch_dofs is not None:
            self.o.batch_dofs = int(batch_dofs)
        if group_members is not None:
            self.o.group_members = int(group_members)
        opts.setdefault("autotune", 0)  # as st_serve_opts_default: no per-setup tuning
        self.o.opt = options(**opts)
        self._s = ctypes.c_void_p()
        _check(lib.st_serve_start(ctypes.byref(self._s), ctypes.byref(self.o)))
        self._n = {}

    def submit(self, dim, degree, spans, slabs, rhs, tol=1e-8, coeffs=False):
        import numpy as np
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        r = StRequest()
        r.geometry, r.degree, r.slabs = int(dim), int(degree), int(slabs)
        for a in range(3):
            r.spans[a] = int(spans[a]) if a < len(spans) else 1
        r.rhs = rhs.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.rhs_is_coeffs = 1 if coeffs else 0
        r.tol = float(tol)
        t = ctypes.c_uint64()
        _check(_lib.st_serve_submit(self._s, ctypes.byref(r), ctypes.byref(t)))
        self._n[t.value] = rhs.size
        return t.value

    def _take(self, fn, ticket, *extra):
        import numpy as np
        res = StResult()
        u = np.empty(self._n[ticket])
        rc = fn(self._s, ctypes.c_uint64(ticket), *extra, ctypes.byref(res),
                u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if rc == ST_ERR_NOT_READY:
            return None
        _check(rc)
        del self._n[ticket]
        out = {k: getattr(res, k) for k, _ in StResult._fields_}
        out["error"] = res.error.decode(errors="replace")
        return out, u

    def resume(self):
        """Let the workers of a server started (or set) paused take requests."""
        _check(_lib.st_serve_resume(self._s))

    def pause(self):
        """Workers take no further request until resume(); running batches
        finish."""
        _check(_lib.st_serve_pause(self._s))

    def cancel(self, ticket):
        """True if the request was withdrawn before a worker took it, False
        if it is already being solved."""
        rc = _lib.st_serve_cancel(self._s, ctypes.c_uint64(ticket))
        if rc == ST_ERR_NOT_READY:
            return False
        _check(rc)
        return True

    def poll(self, ticket):
        """(result dict, solution) or None while pending."""
        return self._take(_lib.st_serve_poll, ticket)

    def wait(self, ticket, timeout=-1.0):
        return self._take(_lib.st_serve_wait, ticket, ctypes.c_double(timeout))

    def stop(self):
        if self._s:
            _check(_lib.st_serve_stop(self._s))
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# slab partition over several processes
# ----------------------------------------------------------------------------

def partition_plan(slabs_global, size, rank):
    """(first slab, slab count, gathered level) of rank (st_partition_plan)."""
    b, n, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().st_partition_plan(int(slabs_global), int(size), int(rank), ctypes.byref(b),
                                    ctypes.byref(n), ctypes.byref(g)))
    return b.value, n.value, g.value


def _host_bytes(addr, nbytes):
    """A uint8 CPU tensor over host memory at addr (no copy)."""
    import torch
    return torch.frombuffer((ctypes.c_char * int(nbytes)).from_address(addr), dtype=torch.uint8)


class GlooComm:
    """st_comm over the default torch.distributed process group with HOST
    buffers (e.g. the gloo backend): the library stages its device data
    through pinned host memory and calls these callbacks with host pointers.
    Any exception inside a callback is reported to the library as a failure
    (the entry point then returns ST_ERR_COMM)."""

    def __init__(self):
        import torch
        import torch.distributed as dist
        self.rank, self.size = dist.get_rank(), dist.get_world_size()

        def sendrecv(ctx, send, dst, recv, src, nbytes, stream):
            try:
                req = dist.isend(_host_bytes(send, nbytes), dst) if dst >= 0 else None
                if src >= 0:
                    dist.recv(_host_bytes(recv, nbytes), src)
                if req is not None:
                    req.wait()
                return 0
            except Exception:
                return 1

        def allgather(ctx, send, recv, nbytes, stream):
            try:
                out = _host_bytes(recv, nbytes * self.size)
                parts = [torch.empty(nbytes, dtype=torch.uint8) for _ in range(self.size)]
                dist.all_gather(parts, _host_bytes(send, nbytes))
                for q, t in enumerate(parts):
                    out[q * nbytes:(q + 1) * nbytes].copy_(t)
                return 0
            except Exception:
                return 1

        def allreduce(ctx, vals, count):
            try:
                addr = ctypes.addressof(vals.contents)
                t = torch.frombuffer((ctypes.c_double * int(count)).from_address(addr),
                                     dtype=torch.float64)
                dist.all_reduce(t)
                return 0
            except Exception:
                return 1

        self._fns = (SENDRECV_FN(sendrecv), ALLGATHER_FN(allgather), ALLREDUCE_FN(allreduce))
        self.c = StComm(self.rank, self.size, 1, None, *self._fns)

    def close(self):
        pass


class NcclComm:
    """st_comm over an NCCL communicator that the library creates from a
    unique id (st_comm_nccl_create): device buffers, stream-ordered."""

    @staticmethod
    def unique_id():
        buf = (ctypes.c_char * 128)()
        _check(load().st_comm_nccl_unique_id(buf))
        return bytes(buf)

    def __init__(self, size, rank, unique_id):
        load()
        self.c = StComm()
        buf = (ctypes.c_char * 128).from_buffer_copy(bytes(unique_id))
        _check(_lib.st_comm_nccl_create(ctypes.byref(self.c), int(size), int(rank), buf))
        self.rank, self.size = int(rank), int(size)

    def close(self):
        if self.c.ctx:
            _lib.st_comm_nccl_destroy(ctypes.byref(self.c))
