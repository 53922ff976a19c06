"""Oracle: plain serial CPU definitions of the 7-point smoothers (FP64 and FP32).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
touches it.

Every function follows the paper's serial loops (Sec. 3 listings) written out
in C (``stencil_oracle.c``), compiled without FMA contraction.  Arrays are
numpy arrays of shape ``(nz+2, ny+2, nx+2)`` (C order, ``u[k][j][i]``) that
include the one-cell Dirichlet halo; interior extents are ``nx, ny, nz``.

Functions and what pins them (see ``tests/test_oracle_pins.py``):

* ``jacobi`` (Sec. 3 first listing): pinned by the closed-form decay of a
  discrete sine mode, by the sparse matrix form ``D^-1 (L+U) u``, and by the
  harmonic-polynomial and constant fixed points.
* ``gs_lex`` (Sec. 3 second listing): pinned by the lower-triangular solve
  ``(D-L) u_new = U u_old + ...`` (a textbook routine), brute-force sorted
  enumeration on 4^3 grids, and the fixed points.
* ``gs_rb`` (red-black alternative named in Sec. 3): pinned by the two
  half-sweep closed forms (each colour is a Jacobi update of that colour).
* ``residual`` (not in the paper): pinned by the eigen-relation
  ``A phi = lambda phi`` and the sparse matrix form; its norm by ``math.fsum``.
* ``solve_mixed`` / ``solve_f64`` (not in the paper): pinned by the closed-form
  solution ``u* = sum a_m phi_m / lambda_m``.
* ``mg_restrict`` / ``mg_prolong_add`` / ``mg_solve`` (multigrid, named in Sec. 1
  and Sec. 3 as the setting of these smoothers; transfers are the textbook full
  weighting and trilinear interpolation): pinned by exact reproduction of linear
  functions by both transfers, by the restriction's weights summing to one, by
  the V-cycle's reduction factor on the error of the discrete Laplace problem,
  by convergence to the closed-form discrete solution, and by the one-level
  cycle reducing to plain smoothing sweeps.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

_I64 = ctypes.c_int64
_D = ctypes.c_double
_F = ctypes.c_float
_I = ctypes.c_int
_P = ctypes.c_void_p


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_jacobi_f64.argtypes = [_P, _P, _I64, _I64, _I64, _D, _D, _D, _I]
        lib.oracle_gs_lex_f64.argtypes = [_P, _P, _I64, _I64, _I64, _D, _D, _I]
        lib.oracle_gs_rb_f64.argtypes = [_P, _P, _I64, _I64, _I64, _D, _D, _I]
        lib.oracle_gs_rb_f32.argtypes = [_P, _P, _I64, _I64, _I64, _D, _F, _I]
        lib.oracle_residual_f64.argtypes = [_P, _P, _I64, _I64, _I64, _D, _P, _P, _P]
        lib.oracle_jacobi_f32.argtypes = [_P, _P, _I64, _I64, _I64, _D, _F, _F, _I]
        lib.oracle_gs_lex_f32.argtypes = [_P, _P, _I64, _I64, _I64, _D, _F, _I]
        lib.oracle_solve_mixed.argtypes = [_P, _P, _I64, _I64, _I64, _D, _I, _D, _I, _I, _P, _P]
        lib.oracle_solve_f64.argtypes = [_P, _P, _I64, _I64, _I64, _D, _I, _D, _I, _I, _P, _P]
        lib.oracle_mg_restrict_f64.argtypes = [_P, _I64, _I64, _I64, _P]
        lib.oracle_mg_prolong_add_f64.argtypes = [_P, _I64, _I64, _I64, _P]
        lib.oracle_mg_solve_f64.argtypes = [_P, _P, _I64, _I64, _I64, _D, _I, _I, _I, _I, _I, _D, _I, _P, _P]
        lib.oracle_residual_f32.argtypes = [_P, _P, _I64, _I64, _I64, _D, _P]
        lib.oracle_mg_restrict_f32.argtypes = [_P, _I64, _I64, _I64, _P]
        lib.oracle_mg_prolong_add_f32.argtypes = [_P, _I64, _I64, _I64, _P]
        lib.oracle_mg_cycles_f32.argtypes = [_P, _P, _I64, _I64, _I64, _D, _I, _I, _I, _I, _I, _I]
        lib.oracle_solve_mixed_mg.argtypes = [_P, _P, _I64, _I64, _I64, _D, _I, _I, _I, _I, _I, _D, _I, _I, _P, _P]
        for name in ("oracle_jacobi_f64", "oracle_gs_lex_f64", "oracle_gs_rb_f64", "oracle_gs_rb_f32", "oracle_residual_f64",
                     "oracle_jacobi_f32", "oracle_gs_lex_f32", "oracle_solve_mixed", "oracle_solve_f64",
                     "oracle_mg_restrict_f64", "oracle_mg_prolong_add_f64", "oracle_mg_solve_f64",
                     "oracle_residual_f32", "oracle_mg_restrict_f32", "oracle_mg_prolong_add_f32", "oracle_mg_cycles_f32",
                     "oracle_solve_mixed_mg"):
            getattr(lib, name).restype = _I
        _LIB = lib
    return _LIB


B64 = 1.0 / 6.0                    # the Jacobi/GS weight b, as a double
B32 = float(np.float32(1.0 / 6.0))  # the same weight rounded to float

SMOOTHER_JACOBI = 0
SMOOTHER_GS = 1


def _dims(u: np.ndarray):
    nz, ny, nx = (s - 2 for s in u.shape)
    return nx, ny, nz


def _check(u: np.ndarray, f, dtype):
    if u.dtype != dtype or not u.flags.c_contiguous or u.ndim != 3 or min(u.shape) < 2:
        raise ValueError("u must be a C-contiguous 3D %s array with a halo" % np.dtype(dtype).name)
    if f is not None and (f.dtype != dtype or f.shape != u.shape or not f.flags.c_contiguous):
        raise ValueError("f must match u")


def _ptr(a):
    return None if a is None else a.ctypes.data


def jacobi(u: np.ndarray, f: np.ndarray | None = None, h: float = 1.0, nsweeps: int = 1,
           a: float = 0.0, b: float | None = None) -> np.ndarray:
    """Return u after ``nsweeps`` Jacobi sweeps (Sec. 3 first listing); u is not modified.
    float64 or float32 by u's dtype."""
    out = np.array(u, copy=True, order="C")
    if out.dtype == np.float64:
        _check(out, f, np.float64)
        rc = _lib().oracle_jacobi_f64(_ptr(out), _ptr(f), *_dims(out), h, a, B64 if b is None else b, nsweeps)
    elif out.dtype == np.float32:
        _check(out, f, np.float32)
        rc = _lib().oracle_jacobi_f32(_ptr(out), _ptr(f), *_dims(out), h, a, B32 if b is None else b, nsweeps)
    else:
        raise ValueError("dtype")
    if rc != 0:
        raise RuntimeError("oracle_jacobi rc=%d" % rc)
    return out


def gs_lex(u: np.ndarray, f: np.ndarray | None = None, h: float = 1.0, nsweeps: int = 1,
           b: float | None = None) -> np.ndarray:
    """Return u after ``nsweeps`` lexicographic Gauss-Seidel sweeps (Sec. 3 second listing)."""
    out = np.array(u, copy=True, order="C")
    if out.dtype == np.float64:
        _check(out, f, np.float64)
        rc = _lib().oracle_gs_lex_f64(_ptr(out), _ptr(f), *_dims(out), h, B64 if b is None else b, nsweeps)
    elif out.dtype == np.float32:
        _check(out, f, np.float32)
        rc = _lib().oracle_gs_lex_f32(_ptr(out), _ptr(f), *_dims(out), h, B32 if b is None else b, nsweeps)
    else:
        raise ValueError("dtype")
    if rc != 0:
        raise RuntimeError("oracle_gs_lex rc=%d" % rc)
    return out


def gs_rb(u: np.ndarray, f: np.ndarray | None = None, h: float = 1.0, nsweeps: int = 1) -> np.ndarray:
    """Return u after ``nsweeps`` red-black Gauss-Seidel sweeps (red = (i+j+k) even first,
    0-based interior coordinates); float64 or float32 by u's dtype."""
    out = np.array(u, copy=True, order="C")
    if out.dtype == np.float32:
        _check(out, f, np.float32)
        rc = _lib().oracle_gs_rb_f32(_ptr(out), _ptr(f), *_dims(out), h, B32, nsweeps)
        if rc != 0:
            raise RuntimeError("oracle_gs_rb rc=%d" % rc)
        return out
    _check(out, f, np.float64)
    rc = _lib().oracle_gs_rb_f64(_ptr(out), _ptr(f), *_dims(out), h, B64, nsweeps)
    if rc != 0:
        raise RuntimeError("oracle_gs_rb rc=%d" % rc)
    return out


def residual(u: np.ndarray, f: np.ndarray | None, h: float):
    """Return (r, ||r||_2, ||f||_2) with r = f - A u on the interior (halo of r zero), FP64."""
    _check(u, f, np.float64)
    r = np.zeros_like(u)
    rn = ctypes.c_double(0.0)
    fn = ctypes.c_double(0.0)
    rc = _lib().oracle_residual_f64(_ptr(u), _ptr(f), *_dims(u), h, _ptr(r),
                                    ctypes.addressof(rn), ctypes.addressof(fn))
    if rc != 0:
        raise RuntimeError("oracle_residual rc=%d" % rc)
    return r, rn.value, fn.value


def solve_mixed(u: np.ndarray, f: np.ndarray | None, h: float, smoother: int, rtol: float,
                max_outer: int, inner_sweeps: int):
    """Defect correction with FP32 inner sweeps.  Returns (u, rel, outer_iters, converged)."""
    out = np.array(u, copy=True, order="C")
    _check(out, f, np.float64)
    rel = ctypes.c_double(0.0)
    its = ctypes.c_int(0)
    rc = _lib().oracle_solve_mixed(_ptr(out), _ptr(f), *_dims(out), h, smoother, rtol, max_outer,
                                   inner_sweeps, ctypes.addressof(rel), ctypes.addressof(its))
    if rc not in (0, -5):
        raise RuntimeError("oracle_solve_mixed rc=%d" % rc)
    return out, rel.value, its.value, rc == 0


def solve_f64(u: np.ndarray, f: np.ndarray | None, h: float, smoother: int, rtol: float,
              max_sweeps: int, check_every: int):
    """FP64-only solve by plain sweeps.  Returns (u, rel, sweeps, converged)."""
    out = np.array(u, copy=True, order="C")
    _check(out, f, np.float64)
    rel = ctypes.c_double(0.0)
    sw = ctypes.c_int(0)
    rc = _lib().oracle_solve_f64(_ptr(out), _ptr(f), *_dims(out), h, smoother, rtol, max_sweeps,
                                 check_every, ctypes.addressof(rel), ctypes.addressof(sw))
    if rc not in (0, -5):
        raise RuntimeError("oracle_solve_f64 rc=%d" % rc)
    return out, rel.value, sw.value, rc == 0


MG_JACOBI = 0  # weighted Jacobi, omega = 6/7 (a = b = 1/7)
MG_GS = 1      # lexicographic Gauss-Seidel
MG_GS_RB = 2   # red-black Gauss-Seidel


def residual32(u: np.ndarray, f: np.ndarray | None, h: float) -> np.ndarray:
    """FP32 residual r = f - (6u - sum) * (float)(1/h^2), every operation in binary32 (halo of r zero)."""
    _check(u, f, np.float32)
    r = np.zeros_like(u)
    rc = _lib().oracle_residual_f32(_ptr(u), _ptr(f), *_dims(u), h, _ptr(r))
    if rc != 0:
        raise RuntimeError("oracle_residual_f32 rc=%d" % rc)
    return r


def mg_restrict(r: np.ndarray) -> np.ndarray:
    """Full-weighting restriction of the interior of r (odd extents) to the coarse
    grid of extents (n-1)/2 (zero halo); float64 or float32 by r's dtype."""
    nx, ny, nz = _dims(r)
    fc = np.zeros(((nz - 1) // 2 + 2, (ny - 1) // 2 + 2, (nx - 1) // 2 + 2), dtype=r.dtype)
    if r.dtype == np.float32:
        _check(r, None, np.float32)
        rc = _lib().oracle_mg_restrict_f32(_ptr(r), nx, ny, nz, _ptr(fc))
    else:
        _check(r, None, np.float64)
        rc = _lib().oracle_mg_restrict_f64(_ptr(r), nx, ny, nz, _ptr(fc))
    if rc != 0:
        raise RuntimeError("oracle_mg_restrict rc=%d" % rc)
    return fc


def mg_prolong_add(u: np.ndarray, e: np.ndarray) -> np.ndarray:
    """u plus the trilinear prolongation of the coarse correction e (zero on the
    coarse boundary); u is not modified."""
    out = np.array(u, copy=True, order="C")
    dt = np.float32 if out.dtype == np.float32 else np.float64
    _check(out, None, dt)
    _check(e, None, dt)
    nx, ny, nz = _dims(out)
    if _dims(e) != ((nx - 1) // 2, (ny - 1) // 2, (nz - 1) // 2):
        raise ValueError("e must be the coarse grid of u")
    fn = _lib().oracle_mg_prolong_add_f32 if dt == np.float32 else _lib().oracle_mg_prolong_add_f64
    rc = fn(_ptr(out), nx, ny, nz, _ptr(e))
    if rc != 0:
        raise RuntimeError("oracle_mg_prolong_add rc=%d" % rc)
    return out


def mg_solve(u: np.ndarray, f: np.ndarray | None, h: float, smoother: int, nu1: int, nu2: int, ncoarse: int,
             max_levels: int, rtol: float, max_cycles: int):
    """Multigrid V-cycles until rel <= rtol or max_cycles.  Returns (u, rel, cycles, converged)."""
    out = np.array(u, copy=True, order="C")
    _check(out, f, np.float64)
    rel = ctypes.c_double(0.0)
    cyc = ctypes.c_int(0)
    rc = _lib().oracle_mg_solve_f64(_ptr(out), _ptr(f), *_dims(out), h, smoother, nu1, nu2, ncoarse, max_levels,
                                    rtol, max_cycles, ctypes.addressof(rel), ctypes.addressof(cyc))
    if rc not in (0, -5):
        raise RuntimeError("oracle_mg_solve_f64 rc=%d" % rc)
    return out, rel.value, cyc.value, rc == 0


def mg_cycles32(u: np.ndarray, f: np.ndarray, h: float, smoother: int, nu1: int, nu2: int, ncoarse: int,
                max_levels: int, ncycles: int) -> np.ndarray:
    """Exactly ``ncycles`` FP32 V-cycles on A u = f (float32 arrays); u is not modified."""
    out = np.array(u, copy=True, order="C")
    _check(out, f, np.float32)
    rc = _lib().oracle_mg_cycles_f32(_ptr(out), _ptr(f), *_dims(out), h, smoother, nu1, nu2, ncoarse, max_levels,
                                     ncycles)
    if rc != 0:
        raise RuntimeError("oracle_mg_cycles_f32 rc=%d" % rc)
    return out


def solve_mixed_mg(u: np.ndarray, f: np.ndarray | None, h: float, smoother: int, nu1: int, nu2: int, ncoarse: int,
                   max_levels: int, rtol: float, max_outer: int, inner_cycles: int):
    """Defect correction (FP64 residual and update) with ``inner_cycles`` FP32 V-cycles per outer
    iteration.  Returns (u, rel, outer_iters, converged)."""
    out = np.array(u, copy=True, order="C")
    _check(out, f, np.float64)
    rel = ctypes.c_double(0.0)
    its = ctypes.c_int(0)
    rc = _lib().oracle_solve_mixed_mg(_ptr(out), _ptr(f), *_dims(out), h, smoother, nu1, nu2, ncoarse, max_levels,
                                      rtol, max_outer, inner_cycles, ctypes.addressof(rel), ctypes.addressof(its))
    if rc not in (0, -5):
        raise RuntimeError("oracle_solve_mixed_mg rc=%d" % rc)
    return out, rel.value, its.value, rc == 0


# ------------------------------------------------------------------ all-core CPU baseline (OpenMP) --
_OMP = None


def _omp():
    global _OMP
    if _OMP is None:
        lib = ctypes.CDLL(_build.build_omp())
        lib.omp_jacobi_f64.argtypes = [_P, _P, _I64, _I64, _I64, _D, _D, _D, _I, _I]
        lib.omp_gs_lex_f64.argtypes = [_P, _P, _I64, _I64, _I64, _D, _D, _I, _I]
        lib.omp_jacobi_f64.restype = _I
        lib.omp_gs_lex_f64.restype = _I
        lib.omp_max_threads.restype = _I
        _OMP = lib
    return _OMP


def omp_threads() -> int:
    """Threads the OpenMP baseline uses by default (all host cores unless OMP_NUM_THREADS says otherwise)."""
    return int(_omp().omp_max_threads())


def jacobi_omp(u: np.ndarray, f: np.ndarray | None = None, h: float = 1.0, nsweeps: int = 1, a: float = 0.0,
               b: float | None = None, threads: int = 0) -> np.ndarray:
    """Jacobi sweeps on all host cores (planes split among threads); the oracle's bits.  FP64."""
    out = np.array(u, copy=True, order="C")
    _check(out, f, np.float64)
    rc = _omp().omp_jacobi_f64(_ptr(out), _ptr(f), *_dims(out), h, a, B64 if b is None else b, nsweeps, threads)
    if rc != 0:
        raise RuntimeError("omp_jacobi_f64 rc=%d" % rc)
    return out


def gs_lex_omp(u: np.ndarray, f: np.ndarray | None = None, h: float = 1.0, nsweeps: int = 1,
               b: float | None = None, threads: int = 0) -> np.ndarray:
    """Pipeline-parallel lexicographic Gauss-Seidel on all host cores (Sec. 3); the oracle's bits.  FP64."""
    out = np.array(u, copy=True, order="C")
    _check(out, f, np.float64)
    rc = _omp().omp_gs_lex_f64(_ptr(out), _ptr(f), *_dims(out), h, B64 if b is None else b, nsweeps, threads)
    if rc != 0:
        raise RuntimeError("omp_gs_lex_f64 rc=%d" % rc)
    return out
