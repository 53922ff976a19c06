"""Python binding of the C ABI in ``include/stencil.h`` (argument marshalling only).

Every smoother step runs in the CUDA library ``_lib/libstencil.so``; this
module only turns torch tensors into device pointers, shapes into ``dims``
and the current torch stream into the ``stream`` argument.  There is no CPU
fallback: if the library cannot be loaded, importing the functions raises.

Grids are torch tensors of shape ``(nz+2, ny+2, nx+2)`` (C order, halo
included) on a CUDA device; float64 for the FP64 entry points, float32 for
the ``_f32`` ones.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

STENCIL_OK = 0
STENCIL_ERR_ARG = -1
STENCIL_ERR_OOM = -2
STENCIL_ERR_CUDA = -3
STENCIL_ERR_TIMEOUT = -4
STENCIL_ERR_NOT_CONVERGED = -5
STENCIL_ERR_UNSUPPORTED = -6
STENCIL_ERR_CANCELLED = -7

STENCIL_JACOBI = 0
STENCIL_GS = 1
STENCIL_GS_RB = 2  # multigrid smoother only
STENCIL_F64 = 0
STENCIL_F32 = 1

_ERRNAMES = {
    -1: "STENCIL_ERR_ARG", -2: "STENCIL_ERR_OOM", -3: "STENCIL_ERR_CUDA", -4: "STENCIL_ERR_TIMEOUT",
    -5: "STENCIL_ERR_NOT_CONVERGED", -6: "STENCIL_ERR_UNSUPPORTED", -7: "STENCIL_ERR_CANCELLED",
}


class StencilError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "?"), code, msg))
        self.code = code


class stencil_params(ctypes.Structure):
    _fields_ = [("nt", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("tile_z", ctypes.c_int),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("variant", ctypes.c_int), ("int_adds", ctypes.c_int)]


class stencil_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dtype", ctypes.c_int), ("dims", ctypes.c_int64 * 3), ("h", ctypes.c_double),
                ("nsweeps", ctypes.c_int), ("rtol", ctypes.c_double), ("u_in", ctypes.c_void_p),
                ("f_in", ctypes.c_void_p), ("u_out", ctypes.c_void_p)]


class stencil_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("sweeps_done", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("queue_s", ctypes.c_double), ("latency_s", ctypes.c_double)]


class stencil_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("launches", ctypes.c_uint64), ("p50_s", ctypes.c_double),
                ("p99_s", ctypes.c_double), ("mean_s", ctypes.c_double), ("lup_total", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("glups", ctypes.c_double), ("hbm_in_use", ctypes.c_size_t),
                ("hbm_peak", ctypes.c_size_t), ("queue_depth", ctypes.c_int), ("active", ctypes.c_int),
                ("smooth_lup", ctypes.c_double), ("smooth_s", ctypes.c_double), ("solve_cycles", ctypes.c_double),
                ("solve_s", ctypes.c_double), ("copy_bytes", ctypes.c_double), ("copy_s", ctypes.c_double)]


class stencil_probe_result(ctypes.Structure):
    _fields_ = [("fp64_ops_per_s", ctypes.c_double), ("fp32_ops_per_s", ctypes.c_double),
                ("alu_ops_per_s", ctypes.c_double), ("int_add_f64_per_s", ctypes.c_double),
                ("int_add_fast_fraction", ctypes.c_double), ("int_add_any_f64_per_s", ctypes.c_double),
                ("copy_bytes_per_s", ctypes.c_double),
                ("sm_count", ctypes.c_int), ("clock_khz", ctypes.c_int)]


STENCIL_PENDING = 1
STENCIL_REQ_JACOBI = 0
STENCIL_REQ_GS = 1
STENCIL_REQ_SOLVE = 2
STENCIL_REQ_SOLVE_MIXED = 3

_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_I64P = ctypes.POINTER(ctypes.c_int64)
_PP = ctypes.POINTER(stencil_params)

_SIGS = {
    "stencil_create": (_I, [ctypes.POINTER(_P), _I, ctypes.c_size_t]),
    "stencil_destroy": (None, [_P]),
    "stencil_last_error": (ctypes.c_char_p, [_P]),
    "stencil_workspace_bytes": (ctypes.c_size_t, [_P]),
    "stencil_kernel_launches": (ctypes.c_ulonglong, [_P]),
    "stencil_jacobi": (_I, [_P, _P, _P, _I64P, _D, _I, _P]),
    "stencil_jacobi_ex": (_I, [_P, _P, _P, _I64P, _D, _I, _PP, _P]),
    "stencil_jacobi_f32": (_I, [_P, _P, _P, _I64P, _D, _I, _PP, _P]),
    "stencil_gs_lex": (_I, [_P, _P, _P, _I64P, _D, _I, _P]),
    "stencil_gs_lex_ex": (_I, [_P, _P, _P, _I64P, _D, _I, _PP, _P]),
    "stencil_gs_lex_f32": (_I, [_P, _P, _P, _I64P, _D, _I, _PP, _P]),
    "stencil_gs_rb": (_I, [_P, _P, _P, _I64P, _D, _I, _PP, _P]),
    "stencil_gs_rb_f32": (_I, [_P, _P, _P, _I64P, _D, _I, _PP, _P]),
    "residual_norm": (_I, [_P, _P, _P, _I64P, _D, _P, ctypes.POINTER(_D), ctypes.POINTER(_D), _P]),
    "stencil_batched": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _I64P, ctypes.POINTER(_D),
                             ctypes.POINTER(_I), _I, _I, _PP, _P]),
    "stencil_set_wait_limit": (_I, [_P, ctypes.c_longlong, ctypes.c_longlong]),
    "stencil_autotune": (_I, [_P, _I, _I, _P, _P, _I64P, _D, _I, _PP, ctypes.POINTER(_D), _P]),
    "stencil_server_create": (_I, [ctypes.POINTER(_P), _I, ctypes.c_size_t, _I, _I]),
    "stencil_server_submit": (_I, [_P, ctypes.POINTER(stencil_request), ctypes.POINTER(ctypes.c_uint64)]),
    "stencil_server_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(stencil_result)]),
    "stencil_server_wait": (_I, [_P, ctypes.c_uint64, _D, ctypes.POINTER(stencil_result)]),
    "stencil_server_cancel": (_I, [_P, ctypes.c_uint64]),
    "stencil_server_stats_get": (_I, [_P, ctypes.POINTER(stencil_server_stats)]),
    "stencil_server_destroy": (None, [_P]),
    "stencil_selftest_int_add": (_I, [_P, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                                      ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "residual_norm_noalloc": (_I, [_P, _P, _I64P, _D, _P, ctypes.POINTER(_D), ctypes.POINTER(_D), _P]),
    "stencil_solve_mixed": (_I, [_P, _P, _P, _I64P, _D, _I, _D, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_I), _P]),
    "stencil_solve_f64": (_I, [_P, _P, _P, _I64P, _D, _I, _D, _I, _I, _PP, ctypes.POINTER(_D), ctypes.POINTER(_I),
                               _P]),
    "stencil_mg_solve": (_I, [_P, _P, _P, _I64P, _D, _I, _I, _I, _I, _I, _D, _I, ctypes.POINTER(_D),
                              ctypes.POINTER(_I), _P]),
    "stencil_autotune_batched": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _I64P, ctypes.POINTER(_D),
                                      ctypes.POINTER(_I), _I, _I, _PP, ctypes.POINTER(_D), _P]),
    "stencil_probe_throughput": (_I, [_P, ctypes.c_size_t, ctypes.POINTER(stencil_probe_result)]),
    "stencil_solve_mixed_mg": (_I, [_P, _P, _P, _I64P, _D, _I, _I, _I, _I, _I, _D, _I, _I, ctypes.POINTER(_D),
                                    ctypes.POINTER(_I), _P]),
}

_LIB = None


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load ``_lib/libstencil.so`` (building it first if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError("CUDA library %s is missing; run paper_1004_1741_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def exported_names() -> list[str]:
    return list(_SIGS)


# ---------------------------------------------------------------------------
def _dims(u: torch.Tensor):
    if u.dim() != 3:
        raise ValueError("grid must be 3D (nz+2, ny+2, nx+2)")
    nz, ny, nx = (int(s) - 2 for s in u.shape)
    return (ctypes.c_int64 * 3)(nx, ny, nz)


def _grid(u: torch.Tensor, dtype: torch.dtype, name: str = "u"):
    if not isinstance(u, torch.Tensor) or not u.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if u.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, u.dtype))
    if not u.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(u.data_ptr())


def _opt_grid(f, like: torch.Tensor, dtype: torch.dtype):
    if f is None:
        return None
    if f.shape != like.shape or f.device != like.device:
        raise ValueError("f must have u's shape and device")
    return _grid(f, dtype, "f")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _params(nt=0, tile=(0, 0, 0), a=0.0, b=0.0, variant=0, int_adds=-1):
    p = stencil_params()
    p.nt, p.tile_x, p.tile_y, p.tile_z, p.a, p.b = int(nt), int(tile[0]), int(tile[1]), int(tile[2]), float(a), float(b)
    p.variant = int(variant)
    p.int_adds = int(int_adds)
    return p


def _check(ctx, rc: int, allow=()):
    if rc != STENCIL_OK and rc not in allow:
        msg = load_library().stencil_last_error(ctx.handle if ctx is not None else None)
        raise StencilError(rc, (msg or b"").decode())
    return rc


class Context:
    """Owns a ``stencil_ctx`` (workspace, task tables) on one device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        lib = load_library()
        h = ctypes.c_void_p()
        rc = lib.stencil_create(ctypes.byref(h), int(device), int(hbm_budget_bytes))
        if rc != STENCIL_OK:
            raise StencilError(rc, (lib.stencil_last_error(None) or b"").decode())
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            load_library().stencil_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def workspace_bytes(self) -> int:
        return int(load_library().stencil_workspace_bytes(self.handle))

    @property
    def kernel_launches(self) -> int:
        return int(load_library().stencil_kernel_launches(self.handle))

    def last_error(self) -> str:
        return (load_library().stencil_last_error(self.handle) or b"").decode()


# ------------------------------------------------------------ entry points --
def stencil_jacobi(ctx: Context, u: torch.Tensor, f: torch.Tensor | None, h: float, nsweeps: int, *, nt: int = 0,
                   tile=(0, 0, 0), a: float = 0.0, b: float = 0.0, variant: int = 0, int_adds: int = -1,
                   stream=None) -> None:
    """Jacobi sweeps in place on u (FP64 or FP32 by u's dtype).  The keywords are the fields of
    ``stencil_params`` (include/stencil.h): nt sweeps per pass, tile, weights a and b (0: 1/6),
    kernel variant, and int_adds (-1: the library default, for FP64 the adaptive integer-pipe form)."""
    lib = load_library()
    p = _params(nt, tile, a, b, variant, int_adds)
    if u.dtype == torch.float64:
        rc = lib.stencil_jacobi_ex(ctx.handle, _grid(u, torch.float64), _opt_grid(f, u, torch.float64), _dims(u),
                                   float(h), int(nsweeps), ctypes.byref(p), _stream(stream))
    else:
        rc = lib.stencil_jacobi_f32(ctx.handle, _grid(u, torch.float32), _opt_grid(f, u, torch.float32), _dims(u),
                                    float(h), int(nsweeps), ctypes.byref(p), _stream(stream))
    _check(ctx, rc)


def stencil_gs_lex(ctx: Context, u: torch.Tensor, f: torch.Tensor | None, h: float, nsweeps: int, *, nt: int = 0,
                   tile=(0, 0, 0), variant: int = 0, int_adds: int = -1, stream=None) -> None:
    """Lexicographic Gauss-Seidel sweeps in place on u (FP64 or FP32 by u's dtype).  The keywords
    are the fields of ``stencil_params`` (include/stencil.h); int_adds -1 is the library default."""
    lib = load_library()
    p = _params(nt, tile, variant=variant, int_adds=int_adds)
    if u.dtype == torch.float64:
        rc = lib.stencil_gs_lex_ex(ctx.handle, _grid(u, torch.float64), _opt_grid(f, u, torch.float64), _dims(u),
                                   float(h), int(nsweeps), ctypes.byref(p), _stream(stream))
    else:
        rc = lib.stencil_gs_lex_f32(ctx.handle, _grid(u, torch.float32), _opt_grid(f, u, torch.float32), _dims(u),
                                    float(h), int(nsweeps), ctypes.byref(p), _stream(stream))
    _check(ctx, rc)


def stencil_gs_rb(ctx: Context, u: torch.Tensor, f: torch.Tensor | None, h: float, nsweeps: int,
                  stream=None) -> None:
    """Red-black Gauss-Seidel sweeps in place on u (FP64 or FP32 by u's dtype)."""
    lib = load_library()
    p = _params()
    if u.dtype == torch.float64:
        rc = lib.stencil_gs_rb(ctx.handle, _grid(u, torch.float64), _opt_grid(f, u, torch.float64), _dims(u), float(h),
                               int(nsweeps), ctypes.byref(p), _stream(stream))
    else:
        rc = lib.stencil_gs_rb_f32(ctx.handle, _grid(u, torch.float32), _opt_grid(f, u, torch.float32), _dims(u),
                                   float(h), int(nsweeps), ctypes.byref(p), _stream(stream))
    _check(ctx, rc)


def residual_norm(ctx: Context, u: torch.Tensor, f: torch.Tensor | None, h: float, r_out: torch.Tensor | None = None,
                  stream=None):
    """Returns (||r||_2, ||r||_2/||f||_2) for r = f - A u (FP64); fills r_out's interior if given."""
    lib = load_library()
    ab, rel = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = lib.residual_norm(ctx.handle, _grid(u, torch.float64), _opt_grid(f, u, torch.float64), _dims(u), float(h),
                           _opt_grid(r_out, u, torch.float64), ctypes.byref(ab), ctypes.byref(rel), _stream(stream))
    _check(ctx, rc)
    return ab.value, rel.value


def stencil_batched(ctx: Context, us, fs, hs, nsweeps, smoother: int, *, nt: int = 0, tile=(0, 0, 0),
                    variant: int = 0, int_adds: int = -1, stream=None) -> None:
    """Smooth many grids (a list of tensors, one dtype): one persistent launch, or one z-march launch per sweep
    for Jacobi at nt = 1."""
    lib = load_library()
    n = len(us)
    if n == 0:
        return
    dt = us[0].dtype
    dtype = STENCIL_F64 if dt == torch.float64 else STENCIL_F32
    up = (ctypes.c_void_p * n)(*[_grid(u, dt).value for u in us])
    fp = None
    if fs is not None:
        fp = (ctypes.c_void_p * n)(*[(_opt_grid(f, u, dt).value if f is not None else None) for f, u in zip(fs, us)])
    dims = (ctypes.c_int64 * (3 * n))()
    for i, u in enumerate(us):
        d = _dims(u)
        dims[3 * i], dims[3 * i + 1], dims[3 * i + 2] = d[0], d[1], d[2]
    hh = (ctypes.c_double * n)(*[float(x) for x in hs])
    ns = (ctypes.c_int * n)(*[int(x) for x in nsweeps])
    p = _params(nt, tile, variant=variant, int_adds=int_adds)
    rc = lib.stencil_batched(ctx.handle, n, up, fp, dims, hh, ns, int(smoother), dtype, ctypes.byref(p),
                             _stream(stream))
    _check(ctx, rc)


def stencil_selftest_int_add(ctx: Context, n: int, seed: int = 1, with_any: bool = False):
    """Returns (mismatches, pairs the symmetric integer-pipe addition handled) over n generated
    pairs, and also the pairs the any-sign addition handled when with_any."""
    mm, fast, fast_any = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(ctx, load_library().stencil_selftest_int_add(ctx.handle, int(n), int(seed), ctypes.byref(mm),
                                                        ctypes.byref(fast), ctypes.byref(fast_any)))
    return (mm.value, fast.value, fast_any.value) if with_any else (mm.value, fast.value)


def stencil_set_wait_limit(ctx: Context, timeout_ns: int, never_publish: int = -1) -> None:
    _check(ctx, load_library().stencil_set_wait_limit(ctx.handle, int(timeout_ns), int(never_publish)))


def stencil_autotune(ctx: Context, smoother: int, u: torch.Tensor, f: torch.Tensor | None, h: float, nsweeps: int,
                     stream=None):
    """Returns (params dict, GLUP/s) of the fastest candidate on a copy of u."""
    lib = load_library()
    out = stencil_params()
    g = ctypes.c_double(0.0)
    dtype = STENCIL_F64 if u.dtype == torch.float64 else STENCIL_F32
    rc = lib.stencil_autotune(ctx.handle, int(smoother), dtype, _grid(u, u.dtype), _opt_grid(f, u, u.dtype), _dims(u),
                              float(h), int(nsweeps), ctypes.byref(out), ctypes.byref(g), _stream(stream))
    _check(ctx, rc)
    return ({"nt": out.nt, "tile": (out.tile_x, out.tile_y, out.tile_z), "variant": out.variant,
             "int_adds": out.int_adds}, g.value)


def stencil_autotune_batched(ctx: Context, us, fs, hs, nsweeps, smoother: int, stream=None):
    """The fastest batched parameters for these grids (tensors of one dtype) and sweep counts; returns
    (params dict for stencil_batched, whole-batch GLUP/s).  The grids are not modified."""
    lib = load_library()
    n = len(us)
    dt = us[0].dtype
    dtype = STENCIL_F64 if dt == torch.float64 else STENCIL_F32
    up = (ctypes.c_void_p * n)(*[_grid(u, dt).value for u in us])
    fp = None
    if fs is not None:
        fp = (ctypes.c_void_p * n)(*[(_opt_grid(f, u, dt).value if f is not None else None) for f, u in zip(fs, us)])
    dims = (ctypes.c_int64 * (3 * n))()
    for i, u in enumerate(us):
        d = _dims(u)
        dims[3 * i], dims[3 * i + 1], dims[3 * i + 2] = d[0], d[1], d[2]
    hh = (ctypes.c_double * n)(*[float(x) for x in hs])
    ns = (ctypes.c_int * n)(*[int(x) for x in nsweeps])
    out = stencil_params()
    g = ctypes.c_double(0.0)
    rc = lib.stencil_autotune_batched(ctx.handle, n, up, fp, dims, hh, ns, int(smoother), dtype, ctypes.byref(out),
                                      ctypes.byref(g), _stream(stream))
    _check(ctx, rc)
    return ({"nt": out.nt, "tile": (out.tile_x, out.tile_y, out.tile_z), "variant": out.variant,
             "int_adds": out.int_adds}, g.value)


def stencil_probe_throughput(ctx: Context, copy_bytes: int = 0) -> dict:
    """Measured whole-GPU rates of the pipes the smoothers use (include/stencil.h stencil_probe_throughput)."""
    out = stencil_probe_result()
    _check(ctx, load_library().stencil_probe_throughput(ctx.handle, int(copy_bytes), ctypes.byref(out)))
    return {name: getattr(out, name) for name, _ in stencil_probe_result._fields_}


def residual_norm_noalloc(u: torch.Tensor, f: torch.Tensor | None, h: float, r_out: torch.Tensor | None = None,
                          stream=None):
    """residual_norm for callers that cannot allocate device memory: no context,
    a fixed scratch array inside the library.  Runs on u's device (made current
    for the call) and, by default, on that device's current stream.  Returns
    (||r||_2, ||r||_2/||f||_2)."""
    lib = load_library()
    ab, rel = ctypes.c_double(0.0), ctypes.c_double(0.0)
    pu = _grid(u, torch.float64)
    with torch.cuda.device(u.device):
        st = _stream(stream if stream is not None else torch.cuda.current_stream(u.device))
        rc = lib.residual_norm_noalloc(pu, _opt_grid(f, u, torch.float64), _dims(u), float(h),
                                       _opt_grid(r_out, u, torch.float64), ctypes.byref(ab), ctypes.byref(rel), st)
    _check(None, rc)
    return ab.value, rel.value


def stencil_solve_mixed(ctx: Context, u: torch.Tensor, f: torch.Tensor, h: float, smoother: int, rtol: float,
                        max_outer: int, inner_sweeps: int, stream=None):
    """Defect correction, FP32 inner sweeps; returns (rel, outer_iters, converged)."""
    lib = load_library()
    rel, its = ctypes.c_double(0.0), ctypes.c_int(0)
    rc = lib.stencil_solve_mixed(ctx.handle, _grid(u, torch.float64), _grid(f, torch.float64, "f"), _dims(u),
                                 float(h), int(smoother), float(rtol), int(max_outer), int(inner_sweeps),
                                 ctypes.byref(rel), ctypes.byref(its), _stream(stream))
    _check(ctx, rc, allow=(STENCIL_ERR_NOT_CONVERGED,))
    return rel.value, its.value, rc == STENCIL_OK


def stencil_solve_f64(ctx: Context, u: torch.Tensor, f: torch.Tensor | None, h: float, smoother: int, rtol: float,
                      max_sweeps: int, check_every: int, *, nt: int = 0, tile=(0, 0, 0), stream=None):
    """FP64 sweeps until the relative residual <= rtol; returns (rel, sweeps, converged)."""
    lib = load_library()
    rel, sw = ctypes.c_double(0.0), ctypes.c_int(0)
    p = _params(nt, tile)
    rc = lib.stencil_solve_f64(ctx.handle, _grid(u, torch.float64), _opt_grid(f, u, torch.float64), _dims(u),
                               float(h), int(smoother), float(rtol), int(max_sweeps), int(check_every),
                               ctypes.byref(p), ctypes.byref(rel), ctypes.byref(sw), _stream(stream))
    _check(ctx, rc, allow=(STENCIL_ERR_NOT_CONVERGED,))
    return rel.value, sw.value, rc == STENCIL_OK


def stencil_mg_solve(ctx: Context, u: torch.Tensor, f: torch.Tensor | None, h: float, smoother: int, *,
                     nu1: int = 2, nu2: int = 2, ncoarse: int = 20, max_levels: int = 32, rtol: float = 1e-10,
                     max_cycles: int = 50, stream=None):
    """Multigrid V-cycles (FP64) until the relative residual <= rtol; returns (rel, cycles, converged)."""
    lib = load_library()
    rel, cyc = ctypes.c_double(0.0), ctypes.c_int(0)
    rc = lib.stencil_mg_solve(ctx.handle, _grid(u, torch.float64), _opt_grid(f, u, torch.float64), _dims(u),
                              float(h), int(smoother), int(nu1), int(nu2), int(ncoarse), int(max_levels), float(rtol),
                              int(max_cycles), ctypes.byref(rel), ctypes.byref(cyc), _stream(stream))
    _check(ctx, rc, allow=(STENCIL_ERR_NOT_CONVERGED,))
    return rel.value, cyc.value, rc == STENCIL_OK


def stencil_solve_mixed_mg(ctx: Context, u: torch.Tensor, f: torch.Tensor | None, h: float, smoother: int, *,
                           nu1: int = 2, nu2: int = 2, ncoarse: int = 20, max_levels: int = 32, rtol: float = 1e-10,
                           max_outer: int = 50, inner_cycles: int = 1, stream=None):
    """Defect correction with FP32 multigrid V-cycles inside (FP64 residual and update) until the
    relative residual <= rtol; returns (rel, outer_iters, converged)."""
    lib = load_library()
    rel, its = ctypes.c_double(0.0), ctypes.c_int(0)
    rc = lib.stencil_solve_mixed_mg(ctx.handle, _grid(u, torch.float64), _opt_grid(f, u, torch.float64), _dims(u),
                                    float(h), int(smoother), int(nu1), int(nu2), int(ncoarse), int(max_levels),
                                    float(rtol), int(max_outer), int(inner_cycles), ctypes.byref(rel),
                                    ctypes.byref(its), _stream(stream))
    _check(ctx, rc, allow=(STENCIL_ERR_NOT_CONVERGED,))
    return rel.value, its.value, rc == STENCIL_OK


# ------------------------------------------------------------------ server --
def _result_dict(r: stencil_result) -> dict:
    return {"status": r.status, "sweeps_done": r.sweeps_done, "rel_residual": r.rel_residual, "queue_s": r.queue_s,
            "latency_s": r.latency_s}


class Server:
    """Continuous-batching server (stencil_server_*).  Grids are host numpy
    arrays of shape (nz+2, ny+2, nx+2), float64 or float32; they are referenced
    (not copied) until the request completes."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, sweeps_per_round: int = 10, max_active: int = 0):
        lib = load_library()
        h = ctypes.c_void_p()
        rc = lib.stencil_server_create(ctypes.byref(h), int(device), int(hbm_budget_bytes), int(sweeps_per_round),
                                       int(max_active))
        if rc != STENCIL_OK:
            raise StencilError(rc, (lib.stencil_last_error(None) or b"").decode())
        self.handle = h
        self._keep = {}

    def submit(self, kind: int, u_in, f_in=None, h: float = 1.0, nsweeps: int = 1, rtol: float = 0.0,
               u_out=None) -> int:
        import numpy as np

        for a in (u_in, f_in, u_out):
            if a is not None and (not isinstance(a, np.ndarray) or not a.flags.c_contiguous):
                raise ValueError("grids must be C-contiguous numpy arrays")
        r = stencil_request()
        r.kind = int(kind)
        r.dtype = STENCIL_F64 if u_in.dtype == np.float64 else STENCIL_F32
        nz, ny, nx = (int(x) - 2 for x in u_in.shape)
        r.dims[0], r.dims[1], r.dims[2] = nx, ny, nz
        r.h, r.nsweeps, r.rtol = float(h), int(nsweeps), float(rtol)
        r.u_in = u_in.ctypes.data
        r.f_in = None if f_in is None else f_in.ctypes.data
        r.u_out = None if u_out is None else u_out.ctypes.data
        t = ctypes.c_uint64(0)
        rc = load_library().stencil_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t))
        if rc != STENCIL_OK:
            raise StencilError(rc, "submit rejected")
        self._keep[t.value] = (u_in, f_in, u_out)
        return t.value

    def poll(self, ticket: int):
        res = stencil_result()
        rc = load_library().stencil_server_poll(self.handle, ticket, ctypes.byref(res))
        if rc == STENCIL_PENDING:
            return None
        if rc != STENCIL_OK:
            raise StencilError(rc, "poll")
        self._keep.pop(ticket, None)
        return _result_dict(res)

    def wait(self, ticket: int, timeout_s: float = 60.0):
        res = stencil_result()
        rc = load_library().stencil_server_wait(self.handle, ticket, float(timeout_s), ctypes.byref(res))
        if rc == STENCIL_PENDING:
            return None
        if rc != STENCIL_OK:
            raise StencilError(rc, "wait")
        self._keep.pop(ticket, None)
        return _result_dict(res)

    def cancel(self, ticket: int) -> bool:
        return load_library().stencil_server_cancel(self.handle, ticket) == STENCIL_OK

    def stats(self) -> dict:
        st = stencil_server_stats()
        _check(None, load_library().stencil_server_stats_get(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in stencil_server_stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load_library().stencil_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
