"""Thin Python binding of libfdfd (include/fdfd.h): argument marshalling only.

Every step of the solve runs inside the library's CUDA kernels; this module
only passes device pointers of torch tensors and the current CUDA stream.
There is no fallback: if libfdfd.so is missing or fails to load, importing
this module raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfdfd.so")

FDFD_OK = 0
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_STATE", 3: "ERR_OOM", 4: "ERR_CUDA", 5: "ERR_PIVOT",
                6: "ERR_NOT_CONVERGED", 7: "ERR_TIMEOUT"}
MODE_MIXED, MODE_F64, MODE_PLAIN = 0, 1, 2
FORM_LU, FORM_SYMMETRIC = 0, 1

# Every symbol include/fdfd.h declares (the CPU test checks the library exports them).
EXPORTS = ["fdfd_default_options", "fdfd_create", "fdfd_analyze", "fdfd_factor", "fdfd_refactor_design",
           "fdfd_solve", "fdfd_objective", "fdfd_grad", "fdfd_apply", "fdfd_set_options", "fdfd_stats_get",
           "fdfd_plan_fronts", "fdfd_reset_counters", "fdfd_last_error", "fdfd_destroy",
           "fdfd_profile_enable", "fdfd_profile_get", "fdfd_solve_raw_noalloc", "fdfd_noalloc_scratch_bytes",
           "fdfd_selftest_wait", "fdfd_selftest_wait_async", "fdfd_selftest_mbar_wait", "fdfd_selftest_schur_tc", "fdfd_filter_project", "fdfd_filter_project_adjoint",
           "fdfd_slab_modes", "fdfd_objective_target", "fdfd_design_iteration", "fdfd_density_eps", "fdfd_front_copy",
           "fdfd_plan_sizes"]
HOST_EPS, HOST_OUT = 1, 2


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int)]


class Pml(C.Structure):
    _fields_ = [("npml_x", C.c_int), ("npml_y", C.c_int), ("ln_R", C.c_double), ("order", C.c_double)]


class Box(C.Structure):
    _fields_ = [("x0", C.c_int), ("y0", C.c_int), ("w", C.c_int), ("h", C.c_int)]


class Options(C.Structure):
    _fields_ = [("mode", C.c_int), ("ir_tol", C.c_double), ("ir_max_iter", C.c_int),
                ("gmres_restart", C.c_int), ("growth_bound", C.c_double), ("leaf_area", C.c_int),
                ("pivoting", C.c_int), ("tensor_form", C.c_int), ("tensor_min_m", C.c_int),
                ("tensor_min_tiles", C.c_int), ("factor_form", C.c_int), ("sweep_rhs_pairs", C.c_int),
                ("tensor_offdiag", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("sf", C.c_longlong), ("nf", C.c_longlong), ("bs", C.c_longlong), ("sweeps", C.c_longlong),
                ("ir_iters", C.c_longlong), ("ir_resid", C.c_double), ("fallbacks", C.c_longlong),
                ("growth", C.c_double), ("n_fronts", C.c_int), ("n_levels", C.c_int), ("max_front", C.c_int),
                ("factor_entries", C.c_longlong), ("store_bytes", C.c_longlong),
                ("flops_factor", C.c_double), ("flops_design", C.c_double), ("repivots", C.c_longlong),
                ("factor_form", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelProfile(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_longlong), ("ms", C.c_double),
                ("flops", C.c_double), ("bytes", C.c_double)]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libfdfd.so not built at {path}; run paper_2307_05388_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    lib.fdfd_default_options.argtypes = [C.POINTER(Options)]
    lib.fdfd_default_options.restype = None
    lib.fdfd_create.argtypes = [C.POINTER(vp), Grid, d, C.POINTER(C.c_double), i, Pml, Box, C.POINTER(Options), vp]
    lib.fdfd_analyze.argtypes = [vp]
    lib.fdfd_factor.argtypes = [vp, vp]
    lib.fdfd_refactor_design.argtypes = [vp, vp]
    lib.fdfd_solve.argtypes = [vp, vp, vp, i, i]
    lib.fdfd_objective.argtypes = [vp, vp, i, vp, vp, vp, vp, vp, vp]
    lib.fdfd_grad.argtypes = [vp, vp, vp, i, vp, vp, i]
    lib.fdfd_objective_target.argtypes = [vp, vp, i, vp, vp, vp, vp, vp, vp, vp]
    lib.fdfd_density_eps.argtypes = [vp, vp, d, d, vp]
    lib.fdfd_front_copy.argtypes = [vp, i, i, vp, vp]
    lib.fdfd_plan_sizes.argtypes = [vp, vp, vp, vp]
    lib.fdfd_design_iteration.argtypes = [vp, vp, vp, i, vp, vp, vp, vp, vp, vp, vp, vp, i]
    lib.fdfd_apply.argtypes = [vp, vp, vp, i, i]
    lib.fdfd_set_options.argtypes = [vp, C.POINTER(Options)]
    lib.fdfd_stats_get.argtypes = [vp, C.POINTER(Stats)]
    lib.fdfd_plan_fronts.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.fdfd_profile_enable.argtypes = [vp, i]
    lib.fdfd_profile_get.argtypes = [vp, C.POINTER(KernelProfile), i, C.POINTER(C.c_int)]
    lib.fdfd_reset_counters.argtypes = [vp]
    lib.fdfd_reset_counters.restype = None
    lib.fdfd_solve_raw_noalloc.argtypes = [vp, vp, vp, i, i]
    lib.fdfd_solve_raw_noalloc.restype = C.c_int
    lib.fdfd_noalloc_scratch_bytes.argtypes = []
    lib.fdfd_noalloc_scratch_bytes.restype = C.c_size_t
    lib.fdfd_filter_project.argtypes = [vp, vp, d, d, d, d, d, vp, vp]
    lib.fdfd_filter_project_adjoint.argtypes = [vp, vp, vp, d, vp]
    lib.fdfd_selftest_schur_tc.argtypes = [vp, vp, i, i, i, i]
    lib.fdfd_selftest_wait.argtypes = [vp]
    lib.fdfd_selftest_wait_async.argtypes = [vp]
    lib.fdfd_selftest_mbar_wait.argtypes = [vp]
    lib.fdfd_slab_modes.argtypes = [i, d, vp, i, vp, vp, vp]
    lib.fdfd_last_error.argtypes = [vp]
    lib.fdfd_last_error.restype = C.c_char_p
    lib.fdfd_destroy.argtypes = [vp]
    lib.fdfd_destroy.restype = None
    for name in ("fdfd_create", "fdfd_analyze", "fdfd_factor", "fdfd_refactor_design", "fdfd_solve",
                 "fdfd_objective", "fdfd_grad", "fdfd_apply", "fdfd_set_options", "fdfd_stats_get",
                 "fdfd_plan_fronts", "fdfd_profile_enable", "fdfd_profile_get", "fdfd_filter_project",
                 "fdfd_filter_project_adjoint", "fdfd_objective_target", "fdfd_design_iteration",
                 "fdfd_density_eps", "fdfd_front_copy", "fdfd_plan_sizes", "fdfd_selftest_mbar_wait", "fdfd_selftest_wait", "fdfd_selftest_wait_async", "fdfd_selftest_schur_tc", "fdfd_slab_modes"):
        getattr(lib, name).restype = C.c_int
    return lib


_lib = load_library()


class FdfdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def default_options(**kw) -> Options:
    o = Options()
    _lib.fdfd_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def slab_modes(eps_line, k0dx: float, n_modes: int):
    """Guided modes of an x-invariant cross-section (host call, no GPU): (mu, theta, phi).

    eps_line: [ny] relative permittivity along y; mu [n_modes] descending, theta [n_modes]
    (propagation constant times dx, NaN where the mode does not propagate along x), phi
    [n_modes, ny] unit-norm profiles.  A mode source on column i is b[i, :] = phi[m]; the
    matching monitor profile is g = phi[m]."""
    eps_line = np.ascontiguousarray(np.asarray(eps_line, dtype=np.float64).ravel())
    ny = eps_line.size
    mu = np.empty(n_modes)
    theta = np.empty(n_modes)
    phi = np.empty((n_modes, ny))
    st = _lib.fdfd_slab_modes(ny, float(k0dx), eps_line.ctypes.data, int(n_modes), mu.ctypes.data,
                              theta.ctypes.data, phi.ctypes.data)
    if st != FDFD_OK:
        raise FdfdError(st, "fdfd_slab_modes rejected its arguments")
    return mu, theta, phi


class Solver:
    """One cached FDFD solver for one grid, a set of wavelengths and one design box.

    k0: free-space wavenumbers 2 pi / lambda (per length unit of dx).  All field
    tensors are complex128 CUDA tensors of shape [n_omega, nrhs, nx*ny].
    """

    def __init__(self, nx: int, ny: int, dx: float, k0, npml, box=(0, 0, 0, 0), options: Options | None = None,
                 stream: torch.cuda.Stream | None = None, ln_R: float = math.log(1e-8), order: float = 3.0):
        self.nx, self.ny, self.dx = int(nx), int(ny), float(dx)
        self.k0 = np.ascontiguousarray(np.atleast_1d(np.asarray(k0, dtype=np.float64)))
        self.n_omega = len(self.k0)
        px, py = (npml, npml) if np.isscalar(npml) else npml
        self.box = tuple(int(v) for v in box)
        self.options = options or default_options()
        self._stream = stream
        sptr = None
        if torch.cuda.is_available():
            st = stream if stream is not None else torch.cuda.current_stream()
            sptr = C.c_void_p(st.cuda_stream)
        h = C.c_void_p()
        kp = self.k0.ctypes.data_as(C.POINTER(C.c_double))
        st = _lib.fdfd_create(C.byref(h), Grid(self.nx, self.ny), self.dx, kp, self.n_omega,
                              Pml(int(px), int(py), float(ln_R), float(order)), Box(*self.box),
                              C.byref(self.options), sptr)
        if st != FDFD_OK or not h.value:
            raise FdfdError(st, "fdfd_create rejected its arguments")
        self._h = h

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.fdfd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str, allow=()):
        if st != FDFD_OK and st not in allow:
            raise FdfdError(st, f"{what}: {_lib.fdfd_last_error(self._h).decode()}")
        return st

    @property
    def n(self) -> int:
        return self.nx * self.ny

    # -- C-ABI calls (same names) -------------------------------------------
    def analyze(self):
        self._check(_lib.fdfd_analyze(self._h), "fdfd_analyze")

    def factor(self, eps: torch.Tensor):
        eps = eps.reshape(-1)
        assert eps.dtype == torch.float64 and eps.numel() == self.n
        self._check(_lib.fdfd_factor(self._h, _ptr(eps)), "fdfd_factor")
        self._keep = eps

    def refactor_design(self, eps_design: torch.Tensor):
        eps_design = eps_design.reshape(-1)
        assert eps_design.dtype == torch.float64 and eps_design.numel() == self.box[2] * self.box[3]
        self._check(_lib.fdfd_refactor_design(self._h, _ptr(eps_design)), "fdfd_refactor_design")
        self._keep = eps_design

    def solve(self, b: torch.Tensor, transpose: bool = False, out: torch.Tensor | None = None,
              allow_not_converged: bool = False) -> torch.Tensor:
        assert b.dtype == torch.complex128 and b.is_cuda and b.numel() % (self.n_omega * self.n) == 0
        nrhs = b.numel() // (self.n_omega * self.n)
        x = out if out is not None else torch.empty_like(b)
        allow = (6,) if allow_not_converged else ()
        self._check(_lib.fdfd_solve(self._h, _ptr(b), _ptr(x), nrhs, int(bool(transpose))), "fdfd_solve", allow)
        return x

    def objective(self, x: torch.Tensor, cols: torch.Tensor, g: torch.Tensor, weight: torch.Tensor | None = None,
                  with_adjoint: bool = True, target: torch.Tensor | None = None):
        """F = sum w |o|^2 (target None) or F = sum w (|o|^2 - target)^2, the overlaps o and the adjoint
        source (fdfd_objective / fdfd_objective_target)."""
        nrhs = x.numel() // (self.n_omega * self.n)
        nsys = self.n_omega * nrhs
        assert cols.dtype == torch.int32 and cols.numel() == nsys
        assert g.dtype == torch.complex128 and g.numel() == nsys * self.ny
        assert target is None or (target.dtype == torch.float64 and target.numel() == nsys)
        o = torch.empty(nsys, dtype=torch.complex128, device=x.device)
        F = torch.empty((), dtype=torch.float64, device=x.device)
        badj = torch.empty_like(x) if with_adjoint else None
        self._check(_lib.fdfd_objective_target(self._h, _ptr(x), nrhs, _ptr(cols), _ptr(g), _ptr(weight),
                                               _ptr(target), _ptr(o), _ptr(F), _ptr(badj)),
                    "fdfd_objective_target")
        return F, o, badj

    def design_iteration(self, eps_design: torch.Tensor, b: torch.Tensor, cols: torch.Tensor, g: torch.Tensor,
                         weight: torch.Tensor | None = None, target: torch.Tensor | None = None,
                         F_out: torch.Tensor | None = None, grad_out: torch.Tensor | None = None,
                         x_out: torch.Tensor | None = None, xadj_out: torch.Tensor | None = None):
        """fdfd_design_iteration: refactor, forward solve, objective, adjoint solve, gradient in one
        call.  eps_design, F_out and grad_out may be CPU tensors (pinned for asynchronous copies):
        the library then copies them itself and returns once F and dF/deps are on the host."""
        nrhs = b.numel() // (self.n_omega * self.n)
        nd = self.box[2] * self.box[3]
        eps_design = eps_design.reshape(-1)
        assert eps_design.dtype == torch.float64 and eps_design.numel() == nd
        host_out = F_out is not None and not F_out.is_cuda
        dev = b.device
        if F_out is None:
            F_out = torch.empty((), dtype=torch.float64, device=dev)
        if grad_out is None:
            grad_out = torch.empty(nd, dtype=torch.float64, device="cpu" if host_out else dev,
                                   pin_memory=host_out)
        assert grad_out.is_cuda != host_out and F_out.numel() == 1 and grad_out.numel() == nd
        flags = (0 if eps_design.is_cuda else HOST_EPS) | (HOST_OUT if host_out else 0)
        self._check(_lib.fdfd_design_iteration(self._h, _ptr(eps_design), _ptr(b), nrhs, _ptr(cols), _ptr(g),
                                               _ptr(weight), _ptr(target), _ptr(F_out), _ptr(grad_out),
                                               _ptr(x_out), _ptr(xadj_out), flags), "fdfd_design_iteration")
        self._keep = eps_design
        return F_out, grad_out

    def grad(self, x_fwd: torch.Tensor, x_adj: torch.Tensor, weight: torch.Tensor | None = None,
             out: torch.Tensor | None = None, accumulate: bool = False) -> torch.Tensor:
        nrhs = x_fwd.numel() // (self.n_omega * self.n)
        g = out if out is not None else torch.empty(self.box[2] * self.box[3], dtype=torch.float64,
                                                     device=x_fwd.device)
        self._check(_lib.fdfd_grad(self._h, _ptr(x_fwd), _ptr(x_adj), nrhs, _ptr(weight), _ptr(g),
                                   int(bool(accumulate))), "fdfd_grad")
        return g

    def filter_project(self, rho: torch.Tensor, radius: float, beta: float, eta: float, eps_lo: float,
                       eps_hi: float) -> tuple[torch.Tensor, torch.Tensor]:
        """Design-box permittivity from the density (conic filter, tanh projection): (eps, work)."""
        n = self.box[2] * self.box[3]
        rho = rho.reshape(-1).contiguous()
        eps = torch.empty(n, dtype=torch.float64, device=rho.device)
        work = torch.empty(2 * n, dtype=torch.float64, device=rho.device)
        self._check(_lib.fdfd_filter_project(self._h, _ptr(rho), float(radius), float(beta), float(eta),
                                             float(eps_lo), float(eps_hi), _ptr(eps), _ptr(work)),
                    "fdfd_filter_project")
        return eps, work

    def density_eps(self, rho: torch.Tensor, eps_lo: float, eps_hi: float, out: torch.Tensor | None = None):
        """Design-box permittivity eps_lo + rho (eps_hi - eps_lo) (fdfd_density_eps)."""
        rho = rho.reshape(-1).contiguous()
        assert rho.dtype == torch.float64 and rho.numel() == self.box[2] * self.box[3]
        eps = out if out is not None else torch.empty_like(rho)
        self._check(_lib.fdfd_density_eps(self._h, _ptr(rho), float(eps_lo), float(eps_hi), _ptr(eps)),
                    "fdfd_density_eps")
        return eps

    def filter_project_adjoint(self, g_eps: torch.Tensor, work: torch.Tensor, radius: float) -> torch.Tensor:
        """dF/drho from dF/deps through the projection and the filter of filter_project."""
        g_eps = g_eps.reshape(-1).contiguous()
        g = torch.empty_like(g_eps)
        self._check(_lib.fdfd_filter_project_adjoint(self._h, _ptr(g_eps), _ptr(work), float(radius), _ptr(g)),
                    "fdfd_filter_project_adjoint")
        return g

    def apply(self, x: torch.Tensor, transpose: bool = False) -> torch.Tensor:
        nrhs = x.numel() // (self.n_omega * self.n)
        y = torch.empty_like(x)
        self._check(_lib.fdfd_apply(self._h, _ptr(x), _ptr(y), nrhs, int(bool(transpose))), "fdfd_apply")
        return y

    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.options, k, v)
        self._check(_lib.fdfd_set_options(self._h, C.byref(self.options)), "fdfd_set_options")

    def stats(self) -> dict:
        s = Stats()
        self._check(_lib.fdfd_stats_get(self._h, C.byref(s)), "fdfd_stats_get")
        return s.as_dict()

    def profile(self, on: bool = True):
        self._check(_lib.fdfd_profile_enable(self._h, int(bool(on))), "fdfd_profile_enable")

    def profile_get(self) -> dict:
        buf = (KernelProfile * 64)()
        n = C.c_int()
        self._check(_lib.fdfd_profile_get(self._h, buf, 64, C.byref(n)), "fdfd_profile_get")
        return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].ms, flops=buf[i].flops,
                                           bytes=buf[i].bytes) for i in range(min(n.value, 64))}

    def reset_counters(self):
        _lib.fdfd_reset_counters(self._h)

    def selftest_schur_tc(self, front, k: int, planes: int = 2):
        """Tensor-core update matrix of one front in place: front[k:, k:] -= front[k:, :k] @ front[:k, k:].

        front: (k + m) x ld complex64 CUDA tensor (row-major, ld >= k + m; only the
        first k + m columns are the front).  planes: operand form, 1 = TF32, 2 = TF32 hi + lo,
        3 = BF16 three-way split."""
        if front.dtype != torch.complex64 or not front.is_cuda or front.dim() != 2 or front.stride(1) != 1:
            raise ValueError("front must be a row-major complex64 CUDA matrix")
        n = front.shape[0]
        m = n - k
        self._check(_lib.fdfd_selftest_schur_tc(self._h, C.c_void_p(front.data_ptr()), int(k), int(m),
                                                int(front.stride(0)), int(planes)), "fdfd_selftest_schur_tc")

    def selftest_mbar_wait(self) -> int:
        """Runs the tensor-core pipeline's bounded mbarrier wait on a barrier nothing arrives at;
        returns the status (7 = gave up as designed)."""
        return int(_lib.fdfd_selftest_mbar_wait(self._h))

    def selftest_wait_async(self) -> int:
        """Queues the same wait without synchronising; the next call that checks the error word
        returns 7 (ERR_TIMEOUT).  Returns this call's status (0)."""
        return int(_lib.fdfd_selftest_wait_async(self._h))

    def selftest_wait(self) -> int:
        """Runs one bounded sweep wait on a counter nothing sets; returns the status (7 = gave up as designed)."""
        return int(_lib.fdfd_selftest_wait(self._h))

    def front_data(self, f: int, w: int = 0, f64: bool = False):
        """(front [n, ld], inverse block [k, ldk]) of front f at wavelength w as numpy complex arrays."""
        k, m, *_ = self.plan_fronts()
        n = np.zeros(len(k), np.int32); ld = np.zeros(len(k), np.int32); ldk = np.zeros(len(k), np.int32)
        self._check(_lib.fdfd_plan_sizes(self._h, n.ctypes.data, ld.ctypes.data, ldk.ctypes.data),
                    "fdfd_plan_sizes")
        dt = np.complex128 if f64 else np.complex64
        fr = np.zeros((int(n[f]), int(ld[f])), dt)
        iv = np.zeros((int(k[f]), max(1, int(ldk[f]))), dt)
        self._check(_lib.fdfd_front_copy(self._h, int(w), int(f), fr.ctypes.data, iv.ctypes.data), "fdfd_front_copy")
        return fr, iv

    def plan_fronts(self):
        """(k, m, parent, level, design, idx) of the symbolic plan as numpy arrays."""
        st = self.stats()
        nf = st["n_fronts"]
        k = np.zeros(nf, np.int32)
        m = np.zeros(nf, np.int32)
        par = np.zeros(nf, np.int32)
        lev = np.zeros(nf, np.int32)
        des = np.zeros(nf, np.int32)
        self._check(_lib.fdfd_plan_fronts(self._h, k.ctypes.data, m.ctypes.data, par.ctypes.data,
                                          lev.ctypes.data, des.ctypes.data, None), "fdfd_plan_fronts")
        idx = np.zeros(int((k + m).sum()), np.int32)
        self._check(_lib.fdfd_plan_fronts(self._h, None, None, None, None, None, idx.ctypes.data),
                    "fdfd_plan_fronts")
        return k, m, par, lev, des, idx
