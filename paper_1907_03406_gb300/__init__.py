"""GB300 Sparse Geometric Factorization (SGF) preconditioner.

Python surface over the C ABI of include/sgf.h.  Every step of the hot path
(assembly, elimination, compression, merge, apply, SpMV, PCG) runs in the
CUDA library; this module only marshals arguments.  torch provides device
memory and streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

STENCILS = {"5pt_2d": 0, "7pt_3d": 1, "7pt_fv_3d": 2, "q1_elastic_3d": 3}
SCHEMES = {"nest_all_all": 0, "nest_2_all": 1, "none": 2, "gen_all_all": 3, "nest_2_2": 4}
PRECISIONS = {"fp64": 0, "mixed": 1}

OK = 0
ERR_NO_CONVERGENCE = -5


class SGFError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        lib = L.load()
        msg = lib.sgf_status_string(code).decode()
        last = lib.sgf_last_error().decode()
        super().__init__(f"{what}: {msg} ({code}) {last}".strip())
        self.code = code


def _check(code: int, what: str):
    if code != OK:
        raise SGFError(code, what)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype="float64"):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if str(t.dtype) != f"torch.{dtype}":
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


class Plan:
    """Symbolic analysis of one grid (sgf_analyze)."""

    def __init__(self, n, dim: int, stencil: str, dirichlet: int, leaf: int, degree: int,
                 scheme: str = "nest_all_all", precision: str = "fp64", tau: float = 0.0,
                 compress_from_level: int = 1, basis: int = 0, dof: int = 1, nu: float = 0.0):
        self._lib = L.load()
        g = L.sgf_grid()
        g.dim = dim
        nn = list(n) + [1, 1, 1]
        g.n[0], g.n[1], g.n[2] = int(nn[0]), int(nn[1]), int(nn[2]) if dim == 3 else 1
        g.dof = dof
        g.dirichlet = int(dirichlet)
        o = L.sgf_opts()
        o.scheme = SCHEMES[scheme]
        o.leaf = int(leaf)
        o.degree = int(degree)
        o.basis = int(basis)
        o.precision = PRECISIONS[precision]
        o.tau = float(tau)
        o.compress_from_level = int(compress_from_level)
        o.nu = float(nu)
        h = C.c_void_p()
        _check(self._lib.sgf_analyze(C.byref(g), STENCILS[stencil], C.byref(o), C.byref(h)), "sgf_analyze")
        self.handle = h
        self.precision = precision
        nl = C.c_int()
        nu = C.c_int64()
        _check(self._lib.sgf_plan_info(h, C.byref(nl), C.byref(nu)), "sgf_plan_info")
        self.nlevels, self.n = nl.value, nu.value

    @classmethod
    def from_config(cls, cfg: dict, **kw):
        kw.setdefault("basis", 1 if cfg.get("basis") == "rbm" else 0)
        kw.setdefault("dof", cfg.get("dof", 1))
        kw.setdefault("scheme", cfg.get("scheme", "nest_all_all"))
        if "nu" in cfg:
            kw.setdefault("nu", cfg["nu"])
        return cls(cfg["n"], cfg["dim"], cfg["stencil"], cfg["dirichlet"], cfg["leaf"],
                   cfg["degree"], **kw)

    def export_level(self, level: int) -> dict:
        nn, npairs, npost = C.c_int(), C.c_int(), C.c_int()
        _check(self._lib.sgf_plan_export_level(self.handle, level, C.byref(nn), C.byref(npairs),
                                               C.byref(npost), None, None, None, None, None, None),
               "sgf_plan_export_level")
        nn, npairs, npost = nn.value, npairs.value, npost.value
        codes = np.zeros(3 * nn, dtype=np.int32)
        flags = np.zeros(nn, dtype=np.int32)
        cptr = np.zeros(nn + 1, dtype=np.int32)
        _check(self._lib.sgf_plan_export_level(self.handle, level, None, None, None,
                                               codes.ctypes.data_as(L._IP), flags.ctypes.data_as(L._IP),
                                               cptr.ctypes.data_as(L._IP), None, None, None), "export")
        cidx = np.zeros(max(int(cptr[-1]), 1), dtype=np.int32)
        pairs = np.zeros(max(2 * npairs, 1), dtype=np.int32)
        post = np.zeros(max(2 * npost, 1), dtype=np.int32)
        _check(self._lib.sgf_plan_export_level(self.handle, level, None, None, None, None, None, None,
                                               cidx.ctypes.data_as(L._IP), pairs.ctypes.data_as(L._IP),
                                               post.ctypes.data_as(L._IP)), "export")
        return dict(nnodes=nn, codes=codes.reshape(nn, 3), interior=(flags & 1).astype(bool),
                    eligible=((flags >> 1) & 1).astype(bool), cell_dim=(flags >> 4) & 15,
                    child_ptr=cptr, child_idx=cidx[: int(cptr[-1])],
                    pairs=pairs[: 2 * npairs].reshape(-1, 2), post=post[: 2 * npost].reshape(-1, 2))

    def footprint(self):
        a, b = C.c_size_t(), C.c_size_t()
        _check(self._lib.sgf_plan_footprint(self.handle, C.byref(a), C.byref(b)), "sgf_plan_footprint")
        return a.value, b.value

    @property
    def tuning(self) -> dict:
        """Launch shapes later factors of this plan use (sgf_plan_get_tuning)."""
        t = L.sgf_tuning()
        _check(self._lib.sgf_plan_get_tuning(self.handle, C.byref(t)), "sgf_plan_get_tuning")
        return {f: getattr(t, f) for f, _ in t._fields_}

    @tuning.setter
    def tuning(self, values: dict):
        t = L.sgf_tuning(**{**self.tuning, **values})
        _check(self._lib.sgf_plan_set_tuning(self.handle, C.byref(t)), "sgf_plan_set_tuning")

    def autotune(self, coeffs, napply: int = 10, stream=None):
        """Search of the launch shapes (sgf_autotune): factor shapes timed on
        factorizations, GEMV budgets on napply applies; keeps the fastest in
        the plan and returns (tuning dict, factor + apply ms)."""
        t, ms = L.sgf_tuning(), C.c_double()
        _check(self._lib.sgf_autotune(self.handle, _dev_ptr(coeffs), _stream_ptr(stream), int(napply),
                                      C.byref(t), C.byref(ms)), "sgf_autotune")
        return {f: getattr(t, f) for f, _ in t._fields_}, ms.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self._lib.sgf_plan_destroy(h)
            self.handle = None


class Factor:
    """Numeric factorization A_l of one coefficient field (sgf_factor)."""

    def __init__(self, plan: Plan, coeffs, stream=None):
        self._lib = plan._lib
        self.plan = plan
        h = C.c_void_p()
        rc = self._lib.sgf_factor(plan.handle, _dev_ptr(coeffs), _stream_ptr(stream), C.byref(h))
        _check(rc, "sgf_factor")
        self.handle = h
        self._coeffs = coeffs

    def _vec_call(self, fn, x, out, stream):
        import torch
        nrhs = x.numel() // self.plan.n
        if out is None:
            out = torch.empty_like(x)
        _check(fn(self.handle, _dev_ptr(x), _dev_ptr(out), nrhs, _stream_ptr(stream)), fn.__name__)
        return out

    @property
    def precision(self) -> str:
        """"mixed", or "fp64" (also when a mixed request fell back to FP64)."""
        return "mixed" if self._lib.sgf_factor_precision(self.handle) == 1 else "fp64"

    def apply(self, x, out=None, stream=None):
        """A_l^{-1} x."""
        return self._vec_call(self._lib.sgf_apply, x, out, stream)

    def apply_forward(self, x, out=None, stream=None):
        """A_l x."""
        return self._vec_call(self._lib.sgf_apply_forward, x, out, stream)

    def spmv(self, x, out=None, stream=None):
        """A x."""
        return self._vec_call(self._lib.sgf_spmv, x, out, stream)

    def pcg(self, b, rtol=1e-10, maxit=500, out=None, stream=None, check=True):
        import torch
        nrhs = b.numel() // self.plan.n
        if out is None:
            out = torch.empty_like(b)
        info = L.sgf_solve_info()
        rc = self._lib.sgf_pcg_solve(self.handle, _dev_ptr(b), _dev_ptr(out), nrhs, float(rtol),
                                     int(maxit), _stream_ptr(stream), C.byref(info))
        if check and rc not in (OK,):
            raise SGFError(rc, "sgf_pcg_solve")
        return out, dict(iterations=info.iterations, rel_residual=info.rel_residual,
                         seconds=info.seconds, status=rc)

    def sync(self) -> int:
        """sgf_sync: wait for the device and return the factor's asynchronous
        status (0, or a negative status such as -3 for a non-finite value an
        apply produced since the last call)."""
        return self._lib.sgf_sync(self.handle)

    def level_stats(self, level: int):
        nc = C.c_int()
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(self._lib.sgf_factor_level_stats(self.handle, level, C.byref(nc), C.byref(a),
                                                C.byref(b), C.byref(c)), "level_stats")
        return dict(ncompressed=nc.value, size_before=a.value, size_after=b.value, bytes=c.value)

    def ranks(self, level: int, nnodes: int):
        m = np.zeros(nnodes, dtype=np.int32)
        r = np.zeros(nnodes, dtype=np.int32)
        _check(self._lib.sgf_factor_ranks(self.handle, level, m.ctypes.data_as(L._IP),
                                          r.ctypes.data_as(L._IP)), "ranks")
        return m, r

    def close(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self._lib.sgf_factor_destroy(h)
            self.handle = None

    def __del__(self):
        self.close()


def solve_host(plan: Plan, coeffs: np.ndarray, b: np.ndarray, rtol=1e-10, maxit=500, stream=None):
    """End-to-end call with host buffers: H2D copies, factor, PCG, D2H copy."""
    lib = plan._lib
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty_like(b)
    nrhs = b.size // plan.n
    info = L.sgf_solve_info()
    rc = lib.sgf_solve_host(plan.handle, coeffs.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p),
                            x.ctypes.data_as(C.c_void_p), nrhs, float(rtol), int(maxit),
                            _stream_ptr(stream), C.byref(info))
    _check(rc, "sgf_solve_host")
    return x, dict(iterations=info.iterations, rel_residual=info.rel_residual, seconds=info.seconds)


def memory_stats() -> dict:
    """sgf_memory_stats: the library's device allocation events so far and the
    bytes in use from the current device's default stream-ordered pool."""
    a, u = C.c_int64(), C.c_int64()
    _check(L.load().sgf_memory_stats(C.byref(a), C.byref(u)), "sgf_memory_stats")
    return dict(alloc_events=a.value, pool_used_bytes=u.value)


def profile_reset(timing=False):
    """Clear the launch counters.  timing: False (none), True or "all" (every
    launch bracketed by CUDA events), "contractions" (only the factor's GEMM,
    front and QR launches and the apply graph replays)."""
    mode = {False: 0, True: 1, "all": 1, "contractions": 2}[timing]
    L.load().sgf_profile_reset(mode)


def release_cached_memory():
    """Hand the device memory cached by freed factors back to the device
    (synchronizes the current device)."""
    _check(L.load().sgf_release_cached_memory(), "release_cached_memory")


def profile_read() -> dict:
    """{kernel name: dict(launches, ms, flops, bytes)} since the last reset."""
    lib = L.load()
    out = {}
    for k in range(64):
        name = lib.sgf_profile_kind_name(k).decode()
        if name == "?":
            break
        n = C.c_int64()
        ms, fl, by = C.c_double(), C.c_double(), C.c_double()
        _check(lib.sgf_profile_read(k, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)), "profile_read")
        out[name] = dict(launches=n.value, ms=ms.value, flops=fl.value, bytes=by.value)
    return out


def solve_host_ptr(plan: Plan, coeffs_ptr: int, b_ptr: int, x_ptr: int, nrhs: int, rtol=1e-10,
                   maxit=500, stream=None):
    """sgf_solve_host on raw host pointers (e.g. pinned torch CPU tensors)."""
    info = L.sgf_solve_info()
    rc = plan._lib.sgf_solve_host(plan.handle, C.c_void_p(coeffs_ptr), C.c_void_p(b_ptr), C.c_void_p(x_ptr),
                                  int(nrhs), float(rtol), int(maxit), _stream_ptr(stream), C.byref(info))
    _check(rc, "sgf_solve_host")
    return dict(iterations=info.iterations, rel_residual=info.rel_residual, seconds=info.seconds)
