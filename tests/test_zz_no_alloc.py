"""The allocation-free residual norm, checked against residual_norm.

residual_norm_noalloc serves callers that cannot allocate device memory when
they need a residual (they own the device memory through their own allocator,
or must not stall on cudaMalloc): it keeps
its reduction scratch in a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process and after the others."""
import ctypes

import numpy as np
import pytest

from paper_1004_1741_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1004_1741_gb300 import capi  # noqa: E402

DEV = torch.device("cuda:0")


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("dims,with_f", [((37, 19, 23), True), ((64, 64, 64), False), ((1, 1, 1), True),
                                         ((130, 33, 70), True)])
def test_noalloc_matches_residual_norm_twice(dims, with_f):
    torch.cuda.set_device(DEV)
    u0, f0 = W.random_grid(*dims, seed=17, with_f=with_f)
    h = W.grid_h(*dims)
    u, f = _dev(u0), _dev(f0)
    r_ref = torch.zeros_like(u)
    with capi.Context(0) as ctx:
        ab_ref, rel_ref = capi.residual_norm(ctx, u, f, h, r_out=r_ref)
    for _ in range(2):  # two calls in a row share the fixed scratch
        r = torch.full_like(u, -7.0)
        ab, rel = capi.residual_norm_noalloc(u, f, h, r_out=r)
        # the same kernels in the same order as residual_norm: the same bits
        assert ab == ab_ref and rel == rel_ref, (ab, ab_ref, rel, rel_ref)
        inner = (slice(1, -1),) * 3
        assert torch.equal(r[inner], r_ref[inner])
        ab2, rel2 = capi.residual_norm_noalloc(u, f, h)
        assert ab2 == ab_ref and rel2 == rel_ref


def test_noalloc_after_a_larger_grid():
    """A smaller grid after a larger one: stale partials of the earlier call are not read."""
    torch.cuda.set_device(DEV)
    big, fb = W.random_grid(200, 150, 120, seed=3, with_f=True)
    small, fs = W.random_grid(30, 20, 10, seed=4, with_f=True)
    with capi.Context(0) as ctx:
        ref_big = capi.residual_norm(ctx, _dev(big), _dev(fb), 0.01)
        ref_small = capi.residual_norm(ctx, _dev(small), _dev(fs), 0.02)
    got_big = capi.residual_norm_noalloc(_dev(big), _dev(fb), 0.01)
    got_small = capi.residual_norm_noalloc(_dev(small), _dev(fs), 0.02)
    assert got_big == ref_big and got_small == ref_small


def test_noalloc_rejects_grids_beyond_the_scratch():
    torch.cuda.set_device(DEV)
    lib = capi.load_library()
    u = torch.zeros((3, 3, 3), dtype=torch.float64, device=DEV)
    dims = (ctypes.c_int64 * 3)(1024, 1024, 1024)  # 32*128*32 partial sums > 32768
    ab, rel = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = lib.residual_norm_noalloc(ctypes.c_void_p(u.data_ptr()), None, dims, 1.0, None, ctypes.byref(ab),
                                   ctypes.byref(rel), None)
    assert rc == capi.STENCIL_ERR_ARG
    assert b"32768" in lib.stencil_last_error(None)


def test_noalloc_rejects_host_memory_before_launching():
    """A host pointer for u (or r_out) is refused on the host; no kernel runs on it."""
    torch.cuda.set_device(DEV)
    lib = capi.load_library()
    host = np.zeros((5, 5, 5))
    dims = (ctypes.c_int64 * 3)(3, 3, 3)
    ab, rel = ctypes.c_double(-1.0), ctypes.c_double(-1.0)
    rc = lib.residual_norm_noalloc(ctypes.c_void_p(host.ctypes.data), None, dims, 0.25, None, ctypes.byref(ab),
                                   ctypes.byref(rel), None)
    assert rc == capi.STENCIL_ERR_ARG
    assert b"u is not device memory" in lib.stencil_last_error(None)
    assert ab.value == -1.0
    u = torch.zeros((5, 5, 5), dtype=torch.float64, device=DEV)
    rc = lib.residual_norm_noalloc(ctypes.c_void_p(u.data_ptr()), None, dims, 0.25, ctypes.c_void_p(host.ctypes.data),
                                   ctypes.byref(ab), ctypes.byref(rel), None)
    assert rc == capi.STENCIL_ERR_ARG
    assert b"r_out is not device memory" in lib.stencil_last_error(None)
    # a valid call afterwards succeeds and clears the message
    assert capi.residual_norm_noalloc(u, None, 0.25) == (0.0, 0.0)
    assert lib.stencil_last_error(None) == b""
