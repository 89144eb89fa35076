"""GB300-native additive sweeping preconditioner for the PML Helmholtz equation.

Python face of libasp.so (include/asp.h).  The names follow the C ABI:
``asp_setup`` returns an :class:`AspHandle` whose methods ``factor``,
``apply_preconditioner``, ``matvec``, ``subproblem_solve`` and ``gmres_solve``
call ``asp_factor`` ... ``asp_gmres_solve`` with torch tensors' device
pointers and the current CUDA stream.  Vectors are complex128 CUDA tensors of
shape ``(n, n, nrhs)`` indexed ``[i2-1, i1-1, r]`` (x1 fastest per right-hand
side block, right-hand side fastest overall), which is the RHS-interleaved
layout of the C ABI.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (ASP_PREC_C64, ASP_PREC_C128, KIND_L, KIND_M, KIND_R, AspError,  # noqa: F401
                   asp_params, asp_solve_info)

__all__ = ["asp_setup", "asp_footprint_bytes", "layer_widths_from_velocity", "asp_residual_norms_noalloc",
           "asp_selftest_bounded_wait",
           "AspHandle", "make_params",
           "AspError",
           "ASP_PREC_C64", "ASP_PREC_C128", "KIND_M", "KIND_R", "KIND_L"]


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev_vec(t, n: int, name: str, dim: int = 2):
    """Checks a grid-function batch: contiguous complex128 CUDA tensor of shape
    (n,)*dim + (nrhs,), sweep axis first, x1 next to the right-hand sides."""
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128):
        raise TypeError(f"{name} must be a complex128 CUDA tensor")
    if t.dim() != dim + 1 or any(int(x) != n for x in t.shape[:dim]) or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape {(n,) * dim + ('nrhs',)}")
    return t


def make_params(n: int, omega: float, pml: int, b: int, pml_aux: int = 0, C: float = 20.0,
                precision: str = "c128", max_rhs: int = 1, restart: int = 40, dim: int = 2,
                slab_solver: str = "block") -> asp_params:
    """``slab_solver`` (3D only): "block" (block elimination over the x2 planes)
    or "nd" (nested dissection of the slab's column grid, Section 4)."""
    prec = {"c128": ASP_PREC_C128, "c64": ASP_PREC_C64, "c64sym": _lib.ASP_PREC_C64_SYM}[precision]
    solver = {"block": _lib.ASP_SLAB_BLOCK, "nd": _lib.ASP_SLAB_ND}[slab_solver]
    return asp_params(dim, n, float(omega), pml, pml_aux, b, float(C), prec, max_rhs, restart, solver)


def _widths_arg(widths):
    if widths is None:
        return None, 0, None
    w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
    return w.ctypes.data_as(ctypes.c_void_p), int(w.size), w


def asp_footprint_bytes(params: asp_params, widths=None) -> int:
    """Device bytes of a handle; ``widths``: physical layer widths (None: uniform b)."""
    ptr, m, _keep = _widths_arg(widths)
    return int(_lib.load().asp_footprint_bytes_layers(ctypes.byref(params), ptr, m))


def layer_widths_from_velocity(params: asp_params, c, b_min: int, b_max: int) -> list:
    """Layer widths chosen from the velocity (host computation in the library):
    at least b_min columns, grown up to b_max where the velocity jumps heavily
    along the sweep axis.  ``c``: the float64 velocity as a numpy array."""
    arr = np.ascontiguousarray(np.asarray(c, dtype=np.float64))
    if arr.size != params.n ** params.dim:
        raise ValueError("velocity has the wrong number of nodes")
    cap = params.n + 2
    out = np.zeros(cap, dtype=np.int32)
    m = _lib.load().asp_layer_widths_from_velocity(ctypes.byref(params), arr.ctypes.data_as(ctypes.c_void_p),
                                                   int(b_min), int(b_max), out.ctypes.data_as(ctypes.c_void_p),
                                                   cap)
    if m < 0:
        _lib.check(m, "asp_layer_widths_from_velocity")
    return [int(x) for x in out[:m]]


class AspHandle:
    """An asp_handle: the factored preconditioner of one (velocity, omega, grid)."""

    def __init__(self, ptr: int, params: asp_params):
        self._ptr = ctypes.c_void_p(ptr)
        self.params = params
        self.n = params.n
        self.dim = params.dim

    # -------------------------------------------------------------- info
    @property
    def num_layers(self) -> int:
        return int(_lib.load().asp_num_layers(self._ptr))

    def layer_range(self, p: int) -> tuple[int, int]:
        lo, hi = ctypes.c_int(), ctypes.c_int()
        _lib.check(_lib.load().asp_layer_range(self._ptr, p, ctypes.byref(lo), ctypes.byref(hi)),
                   "asp_layer_range")
        return lo.value, hi.value

    def subproblem_width(self, kind: int, p: int) -> int:
        w = int(_lib.load().asp_subproblem_width(self._ptr, kind, p))
        if w < 0:
            raise AspError(w, "asp_subproblem_width", "no such subproblem")
        return w

    def take_launch_count(self) -> int:
        return int(_lib.load().asp_take_launch_count(self._ptr))

    def set_phase_timing(self, enable: bool) -> None:
        _lib.check(_lib.load().asp_set_phase_timing(self._ptr, 1 if enable else 0), "asp_set_phase_timing")

    def phase_times(self) -> dict:
        """{phase: (milliseconds, launches)} since the last call (synchronizes)."""
        k = len(_lib.PHASES)
        ms = (ctypes.c_double * k)()
        cnt = (ctypes.c_longlong * k)()
        _lib.check(_lib.load().asp_phase_times(self._ptr, ms, cnt, k), "asp_phase_times")
        return {name: (ms[i], int(cnt[i])) for i, name in enumerate(_lib.PHASES)}

    # -------------------------------------------------------------- compute
    def autotune(self, nrhs: int, stream=None) -> dict:
        """Time the candidate launch shapes of the layer solves for ``nrhs``
        right-hand sides on this handle's factors and keep the fastest
        (asp_autotune).  Returns the choices and the candidates' times."""
        choice = np.zeros(4, dtype=np.int32)
        ms = np.zeros(6, dtype=np.float64)
        _lib.check(_lib.load().asp_autotune(self._ptr, int(nrhs), choice.ctypes.data_as(ctypes.c_void_p),
                                            ms.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(_stream_ptr(stream))),
                   "asp_autotune")
        return {"embed": {"cap": int(choice[0]), "variant": int(choice[1]), "candidate_ms": [float(x) for x in ms[:3]]},
                "fill": {"cap": int(choice[2]), "variant": int(choice[3]), "candidate_ms": [float(x) for x in ms[3:]]}}

    def set_solve_shape(self, nrhs: int, kind: str, cap: int, variant: int = 0) -> None:
        """Fix the launch shape of the M-solves (kind "embed") or the sweep fills
        ("fill") for applies with ``nrhs`` right-hand sides: one of the
        candidates asp_autotune times."""
        k = {"embed": 0, "fill": 1}[kind]
        _lib.check(_lib.load().asp_set_solve_shape(self._ptr, int(nrhs), k, int(cap), int(variant)),
                   "asp_set_solve_shape")

    def factor(self, stream=None) -> None:
        _lib.check(_lib.load().asp_factor(self._ptr, ctypes.c_void_p(_stream_ptr(stream))), "asp_factor")

    def apply_preconditioner(self, r, z=None, stream=None):
        torch = _torch()
        _dev_vec(r, self.n, "r", self.dim)
        if z is None:
            z = torch.empty_like(r)
        _dev_vec(z, self.n, "z", self.dim)
        _lib.check(_lib.load().asp_apply_preconditioner(
            self._ptr, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), r.shape[-1],
            ctypes.c_void_p(_stream_ptr(stream))), "asp_apply_preconditioner")
        return z

    def matvec(self, x, y=None, stream=None):
        torch = _torch()
        _dev_vec(x, self.n, "x", self.dim)
        if y is None:
            y = torch.empty_like(x)
        _dev_vec(y, self.n, "y", self.dim)
        _lib.check(_lib.load().asp_matvec(self._ptr, ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(y.data_ptr()), x.shape[-1],
                                          ctypes.c_void_p(_stream_ptr(stream))), "asp_matvec")
        return y

    def subproblem_solve(self, kind: int, p: int, g, v=None, stream=None):
        """v = H^-1 g for one subproblem; g, v complex128 of shape (w, n, nrhs)
        in 2D and (w, n, n, nrhs) in 3D (sweep axis first)."""
        torch = _torch()
        w = self.subproblem_width(kind, p)
        want = (w,) + (self.n,) * (self.dim - 1)
        if not (g.is_cuda and g.dtype == torch.complex128 and tuple(g.shape[:-1]) == want
                and g.dim() == self.dim + 1 and g.is_contiguous()):
            raise ValueError(f"g must be a contiguous complex128 CUDA tensor of shape {want + ('nrhs',)}")
        if v is None:
            v = torch.empty_like(g)
        _lib.check(_lib.load().asp_subproblem_solve(
            self._ptr, kind, p, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(v.data_ptr()), g.shape[-1],
            ctypes.c_void_p(_stream_ptr(stream))), "asp_subproblem_solve")
        return v

    def gmres_solve(self, f, u=None, tol: float = 1e-6, restart: int | None = None, maxit: int = 200,
                    stream=None, raise_on_nonconvergence: bool = True):
        """FGMRES; returns (u, info) with info a list of dicts per right-hand side."""
        torch = _torch()
        _dev_vec(f, self.n, "f", self.dim)
        if u is None:
            u = torch.empty_like(f)
        _dev_vec(u, self.n, "u", self.dim)
        nrhs = f.shape[-1]
        info = (asp_solve_info * nrhs)()
        rs = self.params.restart if restart is None else restart
        code = _lib.load().asp_gmres_solve(self._ptr, ctypes.c_void_p(f.data_ptr()),
                                           ctypes.c_void_p(u.data_ptr()), nrhs, float(tol), rs, maxit, info,
                                           ctypes.c_void_p(_stream_ptr(stream)))
        if code != _lib.ASP_OK and (raise_on_nonconvergence or code != _lib.ASP_ERR_NOT_CONVERGED):
            _lib.check(code, "asp_gmres_solve")
        out = [{"iterations": i.iterations, "converged": bool(i.converged), "rel_res_est": i.rel_res_est,
                "rel_res_true": i.rel_res_true} for i in info]
        return u, out

    def destroy(self) -> None:
        if self._ptr:
            _lib.load().asp_destroy(self._ptr)
            self._ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def asp_residual_norms_noalloc(params: asp_params, c, f, u, rel_res=None, stream=None):
    """||f_r - A u_r|| / ||f_r|| per right-hand side without any device allocation
    inside the library (for callers that cannot allocate: a process whose
    device memory belongs to another allocator, or a serving loop that must
    not allocate once it runs).  ``c`` is the float64
    CUDA velocity (n, n); ``f``, ``u`` complex128 CUDA tensors (n, n, nrhs);
    ``rel_res`` an optional float64 CUDA tensor of nrhs entries that receives
    the result (allocated here, by torch, if omitted)."""
    torch = _torch()
    n = params.n
    _dev_vec(f, n, "f")
    _dev_vec(u, n, "u")
    if not (c.is_cuda and c.dtype == torch.float64 and c.is_contiguous() and c.numel() == n * n):
        raise ValueError("c must be a contiguous float64 CUDA tensor with n*n entries")
    nrhs = f.shape[2]
    if rel_res is None:
        rel_res = torch.empty(nrhs, dtype=torch.float64, device=f.device)
    _lib.check(_lib.load().asp_residual_norms_noalloc(
        ctypes.byref(params), ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(f.data_ptr()),
        ctypes.c_void_p(u.data_ptr()), nrhs, ctypes.c_void_p(rel_res.data_ptr()),
        ctypes.c_void_p(_stream_ptr(stream))), "asp_residual_norms_noalloc")
    return rel_res


def asp_selftest_bounded_wait(polls: int = 4096, stream=None) -> int:
    """Run the device-side bounded-wait path on purpose (a barrier nothing
    arrives on) and return the library's status code: ASP_ERR_TIMEOUT is the
    expected result."""
    return int(_lib.load().asp_selftest_bounded_wait(int(polls), ctypes.c_void_p(_stream_ptr(stream))))


def asp_testhook_fail_device_alloc(after: int) -> None:
    """Test hook: make the setup's device allocation number ``after`` (0: the
    next one) fail as if the device were out of memory; the hook disarms itself
    once it has fired.  ``after`` < 0 disarms it."""
    _lib.check(_lib.load().asp_testhook_fail_device_alloc(int(after)), "asp_testhook_fail_device_alloc")


def asp_setup(c, params: asp_params, widths=None) -> AspHandle:
    """Set up a handle for velocity ``c`` (n x n float64, numpy or CUDA tensor);
    ``widths``: physical layer widths summing to n + 2 - 2*pml (None: uniform
    layers of params.b columns, the last taking the remainder)."""
    lib = _lib.load()
    out = ctypes.c_void_p()
    wptr, m, _keep = _widths_arg(widths)
    if isinstance(c, np.ndarray):
        arr = np.ascontiguousarray(c, dtype=np.float64)
        if arr.size != params.n ** params.dim:
            raise ValueError("velocity has the wrong number of nodes")
        code = lib.asp_setup_layers(ctypes.byref(params), wptr, m, arr.ctypes.data_as(ctypes.c_void_p), 0,
                                    ctypes.byref(out))
    else:
        torch = _torch()
        t = c.contiguous().to(torch.float64)
        code = lib.asp_setup_layers(ctypes.byref(params), wptr, m, ctypes.c_void_p(t.data_ptr()),
                                    1 if t.is_cuda else 0, ctypes.byref(out))
    _lib.check(code, "asp_setup")
    return AspHandle(out.value, params)
