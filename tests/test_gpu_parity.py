"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

FP64 and FP32 smoother results must be bit-exact (fixed expression order, no
contraction on either side).  Residual norms differ only in the reduction
order and must agree to 1e-12 relative."""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
from paper_1004_1741_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts skip at collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1004_1741_gb300 import capi  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def ctx():
    c = capi.Context(0)
    yield c
    c.close()


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _run(ctx, fn, u0, f0, h, nsweeps, **kw):
    u = _dev(u0)
    fn(ctx, u, _dev(f0), h, nsweeps, **kw)
    torch.cuda.synchronize()
    return u.cpu().numpy()


def _assert_exact(got, ref, what):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        i = tuple(bad[0])
        raise AssertionError("%s: %d sites differ, first %s got %r want %r" % (what, len(bad), i, got[i], ref[i]))


RAGGED = [(37, 19, 23), (1, 1, 1), (1, 1, 9), (9, 1, 1), (33, 9, 50), (64, 17, 5), (3, 70, 4)]


# ------------------------------------------------------------------ Jacobi --
def test_config1_laplace64_jacobi_full_field(ctx):
    """64^3 Laplace, halo U[0,1) seed 0, interior 0, 10 sweeps: full field bit-exact."""
    u0 = W.laplace_64()
    _assert_exact(_run(ctx, capi.stencil_jacobi, u0, None, 1.0, 10), oracle.jacobi(u0, None, 1.0, 10), "config1")


@pytest.mark.parametrize("dims", RAGGED)
@pytest.mark.parametrize("nsweeps", [1, 2, 5])
@pytest.mark.parametrize("poisson", [False, True])
def test_jacobi_f64_ragged(ctx, dims, nsweeps, poisson):
    u0, f0 = W.random_grid(*dims, seed=sum(dims) + nsweeps, with_f=poisson)
    h = W.grid_h(*dims)
    _assert_exact(_run(ctx, capi.stencil_jacobi, u0, f0, h, nsweeps), oracle.jacobi(u0, f0, h, nsweeps), "jacobi f64")


@pytest.mark.parametrize("dims", RAGGED)
@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_jacobi_zmarch_variants(ctx, dims, variant, dtype):
    """Plain and cp.async-pipelined z-march, odd and even sweep counts, chunks."""
    u0, f0 = W.random_grid(*dims, seed=7, dtype=dtype, with_f=True)
    for ns, tile in ((3, (0, 0, 0)), (4, (32, 16, 5)), (1, (32, 4, 2)), (2, (32, 8, 1))):
        _assert_exact(_run(ctx, capi.stencil_jacobi, u0, f0, 0.3, ns, tile=tile, variant=variant),
                      oracle.jacobi(u0, f0, 0.3, ns), "variant %d %s %s" % (variant, dims, tile))


@pytest.mark.parametrize("tile", [(32, 4, 7), (32, 16, 3), (0, 8, 1), (0, 0, 0)])
def test_jacobi_f64_tiles_and_zchunks(ctx, tile):
    u0, f0 = W.random_grid(45, 38, 29, seed=5, with_f=True)
    _assert_exact(_run(ctx, capi.stencil_jacobi, u0, f0, 0.1, 3, tile=tile), oracle.jacobi(u0, f0, 0.1, 3), str(tile))


def test_jacobi_weighted(ctx):
    u0, f0 = W.random_grid(30, 20, 10, seed=8, with_f=True)
    a, b = 1.0 - 0.8, 0.8 / 6.0
    _assert_exact(_run(ctx, capi.stencil_jacobi, u0, f0, 0.05, 4, a=a, b=b),
                  oracle.jacobi(u0, f0, 0.05, 4, a=a, b=b), "weighted")


@pytest.mark.parametrize("dims", [(37, 19, 23), (64, 64, 8), (1, 5, 3)])
def test_jacobi_f32_bit_exact(ctx, dims):
    u0, f0 = W.random_grid(*dims, seed=3, dtype=np.float32, with_f=True)
    _assert_exact(_run(ctx, capi.stencil_jacobi, u0, f0, 0.02, 3), oracle.jacobi(u0, f0, 0.02, 3), "jacobi f32")


@pytest.mark.parametrize("tile", [(32, 8, 8), (32, 16, 8), (32, 16, 16), (16, 16, 16), (64, 8, 8)])
@pytest.mark.parametrize("nt", [2, 3, 4, 8])
def test_jacobi_temporal_f64(ctx, tile, nt):
    """Temporal blocking (nt sweeps per pass on skewed tiles): bit-exact, odd and even counts."""
    u0, f0 = W.random_grid(45, 38, 29, seed=nt, with_f=True)
    for ns in (nt, 2 * nt + 1):
        _assert_exact(_run(ctx, capi.stencil_jacobi, u0, f0, 0.07, ns, nt=nt, tile=tile),
                      oracle.jacobi(u0, f0, 0.07, ns), "jacobi %s nt=%d ns=%d" % (tile, nt, ns))


@pytest.mark.parametrize("nt", [2, 4, 8, 16])
def test_jacobi_temporal_f32_and_weighted(ctx, nt):
    u0, f0 = W.random_grid(40, 33, 27, seed=9, dtype=np.float32, with_f=True)
    ns = 2 * nt + 3
    _assert_exact(_run(ctx, capi.stencil_jacobi, u0, f0, 0.03, ns, nt=nt), oracle.jacobi(u0, f0, 0.03, ns), "f32")
    u1, f1 = W.random_grid(21, 17, 13, seed=2, with_f=True)
    a, b = 0.2, 0.8 / 6.0
    _assert_exact(_run(ctx, capi.stencil_jacobi, u1, f1, 0.1, ns, nt=nt, a=a, b=b),
                  oracle.jacobi(u1, f1, 0.1, ns, a=a, b=b), "weighted temporal")


@pytest.mark.parametrize("nt", [1, 2, 3, 4])
@pytest.mark.parametrize("by", [16, 32])
@pytest.mark.parametrize("dims", [(45, 38, 29), (130, 70, 41), (1, 1, 9), (9, 1, 1), (64, 17, 5)])
def test_jacobi_onchip_temporal_f32(ctx, nt, by, dims):
    """variant 4: nt levels per pass in registers/shared memory, overlapped tiles (FP32)."""
    u0, f0 = W.random_grid(*dims, seed=nt + by, dtype=np.float32, with_f=True)
    for ns, zc in ((2 * nt + 1, 0), (nt, 7), (3 * nt, 40)):
        _assert_exact(_run(ctx, capi.stencil_jacobi, u0, f0, 0.05, ns, nt=nt, tile=(0, by, zc), variant=4),
                      oracle.jacobi(u0, f0, 0.05, ns), "onchip nt=%d by=%d %s ns=%d" % (nt, by, dims, ns))


@pytest.mark.parametrize("dims", RAGGED)
def test_jacobi_temporal_ragged(ctx, dims):
    u0, f0 = W.random_grid(*dims, seed=5, with_f=True)
    _assert_exact(_run(ctx, capi.stencil_jacobi, u0, f0, 0.3, 7, nt=4), oracle.jacobi(u0, f0, 0.3, 7), str(dims))


def test_jacobi_zero_sweeps_and_empty(ctx):
    u0, _ = W.random_grid(7, 6, 5, seed=1)
    _assert_exact(_run(ctx, capi.stencil_jacobi, u0, None, 1.0, 0), u0, "zero sweeps")
    e0 = np.random.default_rng(0).random((2, 5, 6))  # nz = 0
    _assert_exact(_run(ctx, capi.stencil_jacobi, e0, None, 1.0, 3), e0, "empty")


# ------------------------------------------------------------ Gauss-Seidel --
@pytest.mark.parametrize("dims", RAGGED)
@pytest.mark.parametrize("nsweeps", [1, 2, 5])
def test_gs_f64_ragged(ctx, dims, nsweeps):
    u0, f0 = W.random_grid(*dims, seed=11 + nsweeps, with_f=True)
    h = W.grid_h(*dims)
    _assert_exact(_run(ctx, capi.stencil_gs_lex, u0, f0, h, nsweeps), oracle.gs_lex(u0, f0, h, nsweeps), "gs f64")


@pytest.mark.parametrize("tile", [(16, 16, 16), (8, 8, 8), (32, 8, 8), (32, 16, 16)])
@pytest.mark.parametrize("nt", [1, 2, 3, 4])
@pytest.mark.parametrize("variant", [1, 2])
def test_gs_f64_tiles_temporal(ctx, tile, nt, variant):
    u0, f0 = W.random_grid(45, 38, 29, seed=nt, with_f=True)
    ns = 2 * nt + 1
    _assert_exact(_run(ctx, capi.stencil_gs_lex, u0, f0, 0.07, ns, nt=nt, tile=tile, variant=variant),
                  oracle.gs_lex(u0, f0, 0.07, ns), "gs %s nt=%d variant %d" % (tile, nt, variant))


@pytest.mark.parametrize("dims", RAGGED + [(45, 38, 29), (70, 9, 33), (20, 20, 2), (17, 18, 3)])
@pytest.mark.parametrize("tile", [(0, 0, 0), (16, 8, 0), (8, 16, 0), (16, 8, 7), (8, 8, 13), (8, 16, 40), (8, 8, 1),
                                  (16, 8, 2), (8, 8, 1000)])
@pytest.mark.parametrize("variant", [4, 5])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_gs_column_march(ctx, dims, tile, variant, dtype):
    """variants 4 / 5 (one launch per level / one persistent dataflow launch): one thread per
    column marching up the tile-local wavefront, chunked or whole columns (odd chunks, chunks of
    one plane), ragged tiles, odd and even sweep counts, with and without f."""
    u0, f0 = W.random_grid(*dims, seed=11, dtype=dtype, with_f=True)
    for ns, ff in ((1, f0), (4, None), (7, f0)):
        _assert_exact(_run(ctx, capi.stencil_gs_lex, u0, ff, 0.04, ns, tile=tile, variant=variant),
                      oracle.gs_lex(u0, ff, 0.04, ns), "gs column v%d %s %s ns=%d" % (variant, dims, tile, ns))


@pytest.mark.parametrize("int_adds", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("variant", [4, 5])
def test_gs_column_int_adds(ctx, int_adds, variant):
    """Every integer-pipe share of the column march gives the oracle's bits (Laplace field, where
    the integer path is taken, and a random field with f)."""
    u0 = W.laplace_cube(70, 1, 2)
    _assert_exact(_run(ctx, capi.stencil_gs_lex, u0, None, 1.0, 9, variant=variant, int_adds=int_adds),
                  oracle.gs_lex(u0, None, 1.0, 9), "gs column laplace int_adds=%d" % int_adds)
    u1, f1 = W.random_grid(41, 35, 30, seed=int_adds, with_f=True)
    _assert_exact(_run(ctx, capi.stencil_gs_lex, u1, f1, 0.2, 5, variant=variant, int_adds=int_adds,
                       tile=(16, 8, 9)),
                  oracle.gs_lex(u1, f1, 0.2, 5), "gs column random int_adds=%d" % int_adds)


@pytest.mark.parametrize("dims", RAGGED + [(45, 38, 29), (70, 9, 33), (20, 20, 2), (17, 18, 3), (2, 2, 2)])
@pytest.mark.parametrize("tile", [(0, 0, 0), (8, 8, 7), (16, 8, 0), (8, 8, 1), (16, 8, 2), (8, 8, 1000)])
@pytest.mark.parametrize("nt", [2, 3, 4])
@pytest.mark.parametrize("variant", [4, 5])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_gs_column_march_several_sweeps_per_task(ctx, dims, tile, nt, variant, dtype):
    """The column march with nt sweeps per task (sweep s on the tile shifted by -s, two steps behind
    sweep s - 1, one shared-memory ring): level launches and the persistent launch, ragged tiles,
    chunks shorter than nt (raised to nt), sweep counts below, at and above multiples of nt, with and
    without f."""
    u0, f0 = W.random_grid(*dims, seed=13, dtype=dtype, with_f=True)
    for ns, ff in ((1, f0), (nt, None), (2 * nt + 1, f0), (5, None)):
        _assert_exact(_run(ctx, capi.stencil_gs_lex, u0, ff, 0.04, ns, nt=nt, tile=tile, variant=variant),
                      oracle.gs_lex(u0, ff, 0.04, ns),
                      "gs column nt=%d v%d %s %s ns=%d" % (nt, variant, dims, tile, ns))


@pytest.mark.parametrize("int_adds", [0, 2, 6])
@pytest.mark.parametrize("nt", [2, 4])
@pytest.mark.parametrize("variant", [4, 5])
def test_gs_column_several_sweeps_int_adds(ctx, int_adds, nt, variant):
    """Every integer-pipe form the multi-sweep march offers (0, 2, adaptive) gives the oracle's bits:
    the positive Laplace field, a random field with f (h^2 f once per call), Poisson data of both
    signs from u = 0."""
    u0 = W.laplace_cube(70, 1, 2)
    _assert_exact(_run(ctx, capi.stencil_gs_lex, u0, None, 1.0, 9, nt=nt, variant=variant, int_adds=int_adds),
                  oracle.gs_lex(u0, None, 1.0, 9), "gs column nt=%d laplace int_adds=%d" % (nt, int_adds))
    u1, f1 = W.random_grid(41, 35, 30, seed=int_adds, with_f=True)
    _assert_exact(_run(ctx, capi.stencil_gs_lex, u1, f1, 0.2, 5, nt=nt, variant=variant, int_adds=int_adds,
                       tile=(16, 8, 9)),
                  oracle.gs_lex(u1, f1, 0.2, 5), "gs column nt=%d random int_adds=%d" % (nt, int_adds))
    u2 = np.zeros_like(u1)
    _assert_exact(_run(ctx, capi.stencil_gs_lex, u2, f1, 0.2, 6, nt=nt, variant=variant, int_adds=int_adds),
                  oracle.gs_lex(u2, f1, 0.2, 6), "gs column nt=%d both signs int_adds=%d" % (nt, int_adds))


def test_gs_column_rejects_nt(ctx):
    u = _dev(W.random_grid(9, 9, 9, seed=1)[0])
    with pytest.raises(capi.StencilError):
        capi.stencil_gs_lex(ctx, u, None, 1.0, 4, nt=5, variant=4)
    with pytest.raises(capi.StencilError):
        capi.stencil_gs_lex(ctx, u, None, 1.0, 4, tile=(32, 16, 0), variant=4)
    with pytest.raises(capi.StencilError):
        capi.stencil_gs_lex(ctx, u, None, 1.0, 4, tile=(32, 16, 0), variant=5)
    with pytest.raises(capi.StencilError):
        capi.stencil_gs_lex(ctx, u, None, 1.0, 4, nt=2, variant=5, tile=(8, 16, 0))
    with pytest.raises(capi.StencilError):
        capi.stencil_gs_lex(ctx, u, None, 1.0, 4, nt=2, variant=4, int_adds=3)
    with pytest.raises(capi.StencilError):
        capi.stencil_gs_lex(ctx, u, None, 1.0, 4, variant=6)


@pytest.mark.parametrize("nt", [1, 4, 8])
@pytest.mark.parametrize("variant", [1, 2])
def test_gs_f32_temporal(ctx, nt, variant):
    u0, f0 = W.random_grid(40, 33, 27, seed=9, dtype=np.float32, with_f=True)
    ns = 2 * nt + 3
    _assert_exact(_run(ctx, capi.stencil_gs_lex, u0, f0, 0.03, ns, nt=nt, variant=variant),
                  oracle.gs_lex(u0, f0, 0.03, ns), "gs f32")


@pytest.mark.parametrize("nt", [8, 16])
def test_gs_f64_deep_temporal_blocking(ctx, nt):
    """FP64 Gauss-Seidel with 8 and 16 sweeps per pass on 16^3 skewed tiles through L1 (variant 2, the
    default at nt > 4) and as one persistent launch (variant 3)."""
    u0, f0 = W.random_grid(45, 38, 40, seed=nt, with_f=True)
    ns = nt + 3
    ref = oracle.gs_lex(u0, f0, 0.05, ns)
    for variant in (0, 3):
        _assert_exact(_run(ctx, capi.stencil_gs_lex, u0, f0, 0.05, ns, nt=nt, tile=(16, 16, 16), variant=variant), ref,
                      "gs f64 nt=%d variant %d" % (nt, variant))


@pytest.mark.parametrize("nt", [2, 4])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_batched_gs_several_sweeps_per_task(ctx, nt, dtype):
    """Batched Gauss-Seidel with nt sweeps per column-march task: uneven grids (some with f, some not,
    sweep counts below and above nt, an empty grid) each equal to the oracle."""
    dims = [(33, 20, 17), (8, 8, 8), (50, 9, 31), (1, 1, 1), (17, 40, 5)]
    sweeps = [nt + 1, 1, 2 * nt, 0, 3]
    grids = [W.random_grid(*d, seed=i, dtype=dtype, with_f=(i % 2 == 0)) for i, d in enumerate(dims)]
    us = [_dev(u) for u, _ in grids]
    fs = [_dev(f) for _, f in grids]
    hs = [W.grid_h(*d) for d in dims]
    capi.stencil_batched(ctx, us, fs, hs, sweeps, capi.STENCIL_GS, nt=nt)
    torch.cuda.synchronize()
    for i, (u0, f0) in enumerate(grids):
        _assert_exact(us[i].cpu().numpy(), oracle.gs_lex(u0, f0, hs[i], sweeps[i]), "batched gs nt=%d grid %d" % (nt, i))


def test_gs_laplace_config1(ctx):
    u0 = W.laplace_64()
    _assert_exact(_run(ctx, capi.stencil_gs_lex, u0, None, 1.0, 10), oracle.gs_lex(u0, None, 1.0, 10), "gs config1")


# ------------------------------------------ FP64 additions on the integer pipes --
def test_int_add_selftest(ctx):
    """The integer-pipe binary64 additions equal the FP64 pipe on 2^26 generated pairs
    (random magnitudes, near-equal operands with ties and carries, raw bit patterns; random
    signs and both argument orders for the any-sign form)."""
    mism, fast, fast_any = capi.stencil_selftest_int_add(ctx, 1 << 26, seed=12345, with_any=True)
    assert mism == 0
    assert fast > (1 << 24)
    assert fast_any > (1 << 25)


@pytest.mark.parametrize("int_adds", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("smoother", ["jacobi", "gs"])
@pytest.mark.parametrize("dims", [(37, 19, 23), (64, 17, 5), (1, 1, 9)])
def test_int_adds_bit_exact(ctx, int_adds, smoother, dims):
    """Same bits whatever share of the additions runs on the integer pipes, for
    Laplace (all operands positive: the integer path) and Poisson (signs mixed:
    fallbacks to the FP64 pipe)."""
    fn, ofn = (capi.stencil_jacobi, oracle.jacobi) if smoother == "jacobi" else (capi.stencil_gs_lex, oracle.gs_lex)
    for poisson in (False, True):
        u0, f0 = W.random_grid(*dims, seed=int_adds, with_f=poisson)
        _assert_exact(_run(ctx, fn, u0, f0, 0.1, 5, int_adds=int_adds), ofn(u0, f0, 0.1, 5),
                      "%s int_adds=%d poisson=%s" % (smoother, int_adds, poisson))
    z0 = np.zeros((dims[2] + 2, dims[1] + 2, dims[0] + 2))  # zeros everywhere: +0 operands take the FP64 pipe
    z0[0] = 0.75
    _assert_exact(_run(ctx, fn, z0, None, 1.0, 4, int_adds=int_adds), ofn(z0, None, 1.0, 4), "zeros")


# ------------------------------------------------- persistent dataflow kernel --
@pytest.mark.parametrize("smoother", ["gs", "jacobi"])
@pytest.mark.parametrize("nt", [1, 2, 4])
@pytest.mark.parametrize("dims", [(45, 38, 29), (1, 1, 9), (64, 17, 5), (33, 9, 50)])
def test_dataflow_single_grid(ctx, smoother, nt, dims):
    """variant 3: one persistent launch over the dependency-ordered task queue."""
    u0, f0 = W.random_grid(*dims, seed=nt + 40, with_f=True)
    fn, ofn = (capi.stencil_gs_lex, oracle.gs_lex) if smoother == "gs" else (capi.stencil_jacobi, oracle.jacobi)
    tile = (16, 16, 16) if smoother == "gs" else (32, 8, 8)
    for ns in (1, 2 * nt + 1):
        _assert_exact(_run(ctx, fn, u0, f0, 0.07, ns, nt=nt, tile=tile, variant=3), ofn(u0, f0, 0.07, ns),
                      "dataflow %s nt=%d ns=%d %s" % (smoother, nt, ns, dims))


def test_dataflow_f32_and_repeat(ctx):
    u0, f0 = W.random_grid(70, 41, 33, seed=2, dtype=np.float32, with_f=True)
    ref = oracle.gs_lex(u0, f0, 0.01, 9)
    for _ in range(3):  # the cached plan and graph are replayed
        _assert_exact(_run(ctx, capi.stencil_gs_lex, u0, f0, 0.01, 9, nt=4, variant=3), ref, "f32 dataflow")


@pytest.mark.parametrize("smoother", [capi.STENCIL_JACOBI, capi.STENCIL_GS])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("nt", [1, 2])
def test_batched_uneven_grids(ctx, smoother, dtype, nt):
    dims = [(32, 48, 16), (17, 5, 40), (64, 64, 32), (1, 1, 1), (48, 16, 80), (9, 33, 7)]
    grids = [W.random_grid(*d, seed=i, dtype=dtype, with_f=(i % 2 == 0)) for i, d in enumerate(dims)]
    hs = [W.grid_h(*d) for d in dims]
    sweeps = [5, 4, 7, 3, 0, 6]
    us = [_dev(u) for u, _ in grids]
    fs = [_dev(f) for _, f in grids]
    capi.stencil_batched(ctx, us, fs, hs, sweeps, smoother, nt=nt)
    torch.cuda.synchronize()
    ofn = oracle.jacobi if smoother == capi.STENCIL_JACOBI else oracle.gs_lex
    for i, ((u0, f0), h, ns) in enumerate(zip(grids, hs, sweeps)):
        _assert_exact(us[i].cpu().numpy(), ofn(u0, f0, h, ns), "batched grid %d" % i)


@pytest.mark.parametrize("tile", [(0, 0, 0), (0, 8, 40), (32, 4, 7)])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("int_adds", [-1, 0, 5])
def test_batched_jacobi_zmarch_many_grids(ctx, dtype, int_adds, tile):
    """Jacobi at nt = 1: one launch per sweep over every grid's tile columns; grids of ragged x/y tiles, a
    column taller than one z-chunk (300 planes), grids that stop early and grids with and without f."""
    dims = [(33, 5, 7), (1, 1, 300), (40, 9, 3), (31, 4, 1), (65, 13, 2)] + [(8 + i, 3 + i % 5, 2 + i % 7)
                                                                          for i in range(40)]
    grids = [W.random_grid(*d, seed=100 + i, dtype=dtype, with_f=(i % 3 != 1)) for i, d in enumerate(dims)]
    hs = [W.grid_h(*d) for d in dims]
    sweeps = [(3 * i) % 8 for i in range(len(dims))]
    us = [_dev(u) for u, _ in grids]
    fs = [_dev(f) for _, f in grids]
    capi.stencil_batched(ctx, us, fs, hs, sweeps, capi.STENCIL_JACOBI, int_adds=int_adds, tile=tile)
    torch.cuda.synchronize()
    for i, ((u0, f0), h, ns) in enumerate(zip(grids, hs, sweeps)):
        _assert_exact(us[i].cpu().numpy(), oracle.jacobi(u0, f0, h, ns), "batched Jacobi grid %d" % i)


def test_batched_jacobi_task_variant_still_served(ctx):
    """variant 3 keeps Jacobi at nt = 1 on the persistent tile tasks; both routes give the oracle's bits."""
    u0, f0 = W.random_grid(37, 11, 13, seed=7, with_f=True)
    ref = oracle.jacobi(u0, f0, 0.05, 3)
    for variant in (0, 3):
        us, fs = [_dev(u0)], [_dev(f0)]
        capi.stencil_batched(ctx, us, fs, [0.05], [3], capi.STENCIL_JACOBI, nt=1, variant=variant)
        _assert_exact(us[0].cpu().numpy(), ref, "batched Jacobi variant %d" % variant)


@pytest.mark.parametrize("case", [("jacobi", -1, 0), ("jacobi", 0, 0), ("jacobi", 3, 0), ("gs", -1, 0),
                                  ("gs", 0, 0), ("gs", 2, 5), ("gs", -1, 5), ("gs", 3, 0)])
def test_prescaled_f_and_budget_fallback(case):
    """FP64 with f over several sweeps: hh*f is computed once into workspace and the sweeps add it as it is
    (one launch more); a budget with no room for it keeps the multiplication in the sweeps.  Both give the
    oracle's bits (Gauss-Seidel int_adds 3 has no prescaled form: no extra launch either way)."""
    smoother, int_adds, variant = case
    dims = (45, 19, 23)
    u0, f0 = W.random_grid(*dims, seed=21, with_f=True)
    u0 = u0 - 0.5  # mixed signs, as in a Poisson iterate
    fn, ofn = (capi.stencil_jacobi, oracle.jacobi) if smoother == "jacobi" else (capi.stencil_gs_lex, oracle.gs_lex)
    ref = ofn(u0, f0, 0.03, 5)
    launches = []
    # Jacobi needs a second grid of workspace, Gauss-Seidel only small task tables
    for budget in (0, int(u0.nbytes * (1.5 if smoother == "jacobi" else 0.9))):
        c = capi.Context(0, hbm_budget_bytes=budget)
        u, f = _dev(u0), _dev(f0)
        n0 = c.kernel_launches
        fn(c, u, f, 0.03, 5, int_adds=int_adds, variant=variant)
        torch.cuda.synchronize()
        launches.append(c.kernel_launches - n0)
        _assert_exact(u.cpu().numpy(), ref, "%s budget %d" % (case, budget))
        c.close()
    prescaled = not (smoother == "gs" and int_adds == 3)
    assert launches[0] - launches[1] == (1 if prescaled else 0), launches


def _two_sign_grid(dims, seed, with_f):
    """Upper half of the planes negative, lower half positive: warps of one launch take both branches of
    the adaptive arithmetic (and the planes between take mixed neighbourhoods)."""
    u0, f0 = W.random_grid(*dims, seed=seed, with_f=with_f)
    u0 = u0.copy()
    u0[u0.shape[0] // 2:] *= -1.0
    return u0, f0


@pytest.mark.parametrize("with_f", [False, True])
@pytest.mark.parametrize("case", [("jacobi", 0), ("jacobi", 6), ("gs", 4), ("gs", 5)])
def test_adaptive_arithmetic_both_signs(ctx, case, with_f):
    """int_adds = 6 (the FP64 default of the z-march and the column march): per warp and update the
    integer-pipe additions for non-negative neighbourhoods, else FP64-pipe additions and the integer-path
    multiplication; the oracle's bits either way."""
    smoother, variant = case
    dims = (70, 21, 30)
    u0, f0 = _two_sign_grid(dims, 31, with_f)
    fn, ofn = (capi.stencil_jacobi, oracle.jacobi) if smoother == "jacobi" else (capi.stencil_gs_lex, oracle.gs_lex)
    ref = ofn(u0, f0, 0.02, 5)
    for ia in (-1, 6):
        _assert_exact(_run(ctx, fn, u0, f0, 0.02, 5, variant=variant, int_adds=ia), ref,
                      "%s variant %d int_adds %d" % (smoother, variant, ia))
    # weighted Jacobi takes the adaptive z-march too
    if smoother == "jacobi" and variant == 0:
        ref_w = oracle.jacobi(u0, f0, 0.02, 3, a=0.25, b=0.125)
        _assert_exact(_run(ctx, fn, u0, f0, 0.02, 3, a=0.25, b=0.125), ref_w, "weighted adaptive")


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_adaptive_value_on_gs_tile_paths(ctx, variant):
    """int_adds = 6 on the Gauss-Seidel tile paths (nt = 2) runs their own default and gives the oracle's bits."""
    u0, f0 = _two_sign_grid((29, 17, 21), 41, True)
    ref = oracle.gs_lex(u0, f0, 0.05, 4)
    _assert_exact(_run(ctx, capi.stencil_gs_lex, u0, f0, 0.05, 4, nt=2, tile=(16, 16, 16), variant=variant,
                       int_adds=6), ref, "gs tiles variant %d" % variant)


def test_batched_adaptive_both_signs(ctx):
    dims = [(40, 12, 9), (33, 9, 16), (9, 33, 7)]
    grids = [_two_sign_grid(d, 70 + i, i != 1) for i, d in enumerate(dims)]
    hs = [W.grid_h(*d) for d in dims]
    sweeps = [4, 3, 6]
    for sm, ofn in ((capi.STENCIL_JACOBI, oracle.jacobi), (capi.STENCIL_GS, oracle.gs_lex)):
        us = [_dev(u) for u, _ in grids]
        fs = [_dev(f) for _, f in grids]
        capi.stencil_batched(ctx, us, fs, hs, sweeps, sm, int_adds=6)
        torch.cuda.synchronize()
        for i, ((u0, f0), h, ns) in enumerate(zip(grids, hs, sweeps)):
            _assert_exact(us[i].cpu().numpy(), ofn(u0, f0, h, ns), "batched adaptive %d grid %d" % (sm, i))


def test_batched_prescaled_f(ctx):
    """Batched FP64 Poisson grids (Jacobi z-march and Gauss-Seidel column tasks) with prescaled f, grids with
    and without f and one-sweep grids in the mix."""
    dims = [(40, 12, 9), (17, 5, 30), (9, 33, 7), (64, 8, 5)]
    grids = [W.random_grid(*d, seed=60 + i, with_f=(i != 2)) for i, d in enumerate(dims)]
    grids = [(u - 0.5, f) for u, f in grids]
    hs = [W.grid_h(*d) for d in dims]
    sweeps = [4, 1, 3, 6]
    for sm, ofn in ((capi.STENCIL_JACOBI, oracle.jacobi), (capi.STENCIL_GS, oracle.gs_lex)):
        us = [_dev(u) for u, _ in grids]
        fs = [_dev(f) for _, f in grids]
        capi.stencil_batched(ctx, us, fs, hs, sweeps, sm)
        torch.cuda.synchronize()
        for i, ((u0, f0), h, ns) in enumerate(zip(grids, hs, sweeps)):
            _assert_exact(us[i].cpu().numpy(), ofn(u0, f0, h, ns), "batched %d grid %d" % (sm, i))


@pytest.mark.parametrize("variant,nt", [(3, 1), (5, 1), (5, 2)])
def test_dataflow_wait_bound_reports_timeout(variant, nt):
    """A task whose completion is never published: the bounded waits expire, the
    call returns STENCIL_ERR_TIMEOUT, and the context keeps working (tile tasks,
    column-march tasks of one and of two sweeps)."""
    c = capi.Context(0)
    u0, _ = W.random_grid(40, 40, 40, seed=1)
    u = _dev(u0)
    capi.stencil_set_wait_limit(c, 50_000_000, never_publish=3)
    with pytest.raises(capi.StencilError) as e:
        capi.stencil_gs_lex(c, u, None, 1.0, 4, nt=nt, variant=variant)
    assert e.value.code == capi.STENCIL_ERR_TIMEOUT
    capi.stencil_set_wait_limit(c, 10_000_000_000, never_publish=-1)
    _assert_exact(_run(c, capi.stencil_gs_lex, u0, None, 1.0, 4, nt=nt, variant=variant),
                  oracle.gs_lex(u0, None, 1.0, 4), "after")
    c.close()


@pytest.mark.parametrize("smoother", [capi.STENCIL_JACOBI, capi.STENCIL_GS])
def test_autotune_picks_a_valid_config(ctx, smoother):
    u0, f0 = W.random_grid(64, 48, 40, seed=3, with_f=True)
    u = _dev(u0)
    params, glups = capi.stencil_autotune(ctx, smoother, u, _dev(f0), 0.02, 8)
    assert glups > 0
    assert params["int_adds"] in (-1, 2, 3), params  # never the all-FP64-pipe form a zeroed struct would give
    assert np.array_equal(u.cpu().numpy(), u0)  # the caller's grid is untouched
    fn, ofn = (capi.stencil_gs_lex, oracle.gs_lex) if smoother == capi.STENCIL_GS else (capi.stencil_jacobi, oracle.jacobi)
    _assert_exact(_run(ctx, fn, u0, f0, 0.02, 8, **params), ofn(u0, f0, 0.02, 8), "autotuned %s" % params)


# ---------------------------------------------------------- red-black GS --
@pytest.mark.parametrize("dims", RAGGED)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_gs_red_black(ctx, dims, dtype):
    u0, f0 = W.random_grid(*dims, seed=31, dtype=dtype, with_f=True)
    for ns in (1, 4):
        _assert_exact(_run(ctx, capi.stencil_gs_rb, u0, f0, 0.2, ns), oracle.gs_rb(u0, f0, 0.2, ns), "rb %s" % (dims,))


# ---------------------------------------------------------------- residual --
@pytest.mark.parametrize("dims", [(37, 19, 23), (1, 1, 1), (64, 64, 64)])
def test_residual_norm(ctx, dims):
    u0, f0 = W.random_grid(*dims, seed=4, with_f=True)
    h = W.grid_h(*dims)
    r = torch.zeros(u0.shape, dtype=torch.float64, device=DEV)
    ab, rel = capi.residual_norm(ctx, _dev(u0), _dev(f0), h, r_out=r)
    r_ref, ab_ref, fn_ref = oracle.residual(u0, f0, h)
    _assert_exact(r.cpu().numpy(), r_ref, "r")
    assert abs(ab - ab_ref) <= 1e-12 * ab_ref
    assert abs(rel - ab_ref / fn_ref) <= 1e-12 * (ab_ref / fn_ref)
    ab2, _ = capi.residual_norm(ctx, _dev(u0), _dev(f0), h)
    assert ab2 == ab  # fixed reduction order


# ------------------------------------------------------------------ solves --
@pytest.mark.parametrize("smoother", [capi.STENCIL_JACOBI, capi.STENCIL_GS])
def test_solve_mixed_fixed_iterations_bit_exact(ctx, smoother):
    """With rtol = 0 both sides run max_outer iterations: u must match bit for bit."""
    p = W.sine_modes_problem(24, seed=4)
    u = torch.zeros(p.f.shape, dtype=torch.float64, device=DEV)
    rel, its, ok = capi.stencil_solve_mixed(ctx, u, _dev(p.f), p.h, smoother, 0.0, 3, 7)
    uref, rel_ref, its_ref, _ = oracle.solve_mixed(np.zeros_like(p.f), p.f, p.h, smoother, 0.0, 3, 7)
    assert its == its_ref == 3 and not ok
    _assert_exact(u.cpu().numpy(), uref, "mixed u")
    assert abs(rel - rel_ref) <= 1e-12 * rel_ref


def test_solve_mixed_converges(ctx):
    p = W.sine_modes_problem(16, seed=4, noise_sigma=0.0)
    u = torch.zeros(p.f.shape, dtype=torch.float64, device=DEV)
    rel, its, ok = capi.stencil_solve_mixed(ctx, u, _dev(p.f), p.h, capi.STENCIL_GS, 1e-10, 400, 50)
    assert ok and rel <= 1e-10


def test_solve_f64_matches_oracle(ctx):
    p = W.sine_modes_problem(20, seed=4)
    u = torch.zeros(p.f.shape, dtype=torch.float64, device=DEV)
    rel, sw, ok = capi.stencil_solve_f64(ctx, u, _dev(p.f), p.h, capi.STENCIL_GS, 0.0, 30, 10)
    uref, rel_ref, sw_ref, _ = oracle.solve_f64(np.zeros_like(p.f), p.f, p.h, oracle.SMOOTHER_GS, 0.0, 30, 10)
    assert sw == sw_ref == 30
    _assert_exact(u.cpu().numpy(), uref, "solve_f64 u")


# ------------------------------------------------------------- arguments --
def test_argument_errors(ctx):
    u = torch.zeros((5, 5, 5), dtype=torch.float64, device=DEV)
    with pytest.raises(capi.StencilError) as e:
        capi.stencil_jacobi(ctx, u, None, 1.0, -1)
    assert e.value.code == capi.STENCIL_ERR_ARG
    with pytest.raises(capi.StencilError) as e:
        capi.stencil_gs_lex(ctx, u, None, 0.0, 1)
    assert e.value.code == capi.STENCIL_ERR_ARG
    with pytest.raises(capi.StencilError) as e:
        capi.stencil_gs_lex(ctx, u, None, 1.0, 1, tile=(7, 7, 7))
    assert e.value.code == capi.STENCIL_ERR_UNSUPPORTED
    with pytest.raises(capi.StencilError) as e:
        capi.stencil_jacobi(ctx, u, None, 1.0, 1, nt=17)
    assert e.value.code == capi.STENCIL_ERR_ARG
    with pytest.raises(capi.StencilError) as e:
        capi.stencil_gs_lex(ctx, u, None, 1.0, 1, nt=9, tile=(8, 8, 8))
    assert e.value.code == capi.STENCIL_ERR_UNSUPPORTED
    with pytest.raises(capi.StencilError) as e:
        capi.stencil_gs_lex(ctx, u, None, 1.0, 1, nt=16, tile=(16, 16, 16), variant=1)
    assert e.value.code == capi.STENCIL_ERR_UNSUPPORTED


def test_budget_oom():
    small = capi.Context(0, hbm_budget_bytes=1024)
    u = torch.zeros((66, 66, 66), dtype=torch.float64, device=DEV)
    with pytest.raises(capi.StencilError) as e:
        capi.stencil_jacobi(small, u, None, 1.0, 2)
    assert e.value.code == capi.STENCIL_ERR_OOM
    small.close()


# ------------------------------------------------- full size (400^3 FP64) --
@pytest.mark.parametrize("smoother", ["jacobi", "gs"])
def test_full_size_400_bench_config(ctx, smoother):
    """The benchmark grid (400^3 FP64, halo seed 1, interior seed 2) in the
    launch configuration bench.py times, 100 sweeps: full field bit-exact."""
    import bench

    cfg = bench.HEADLINE[smoother]
    u0 = W.laplace_cube(400)
    with cf.ThreadPoolExecutor(1) as ex:  # the oracle releases the GIL inside C
        fut = ex.submit(oracle.jacobi if smoother == "jacobi" else oracle.gs_lex, u0, None, 1.0, 100)
        fn = capi.stencil_jacobi if smoother == "jacobi" else capi.stencil_gs_lex
        got = _run(ctx, fn, u0, None, 1.0, 100, nt=cfg["nt"], tile=cfg["tile"], variant=cfg["variant"],
                   int_adds=cfg["int_adds"])
        ref = fut.result()
    _assert_exact(got, ref, "400^3 %s" % smoother)


@pytest.mark.parametrize("name,nt", [("gs", 2), ("gs", 4), ("gs_f32", 2), ("gs_f32", 4), ("gs", 16)])
def test_full_size_400_nt_sweep_config(ctx, name, nt):
    """The benchmark grid in the launch configuration of the benchmark's temporal-depth sweep (the
    multi-sweep column march at nt = 2, 4, the L1 tile tasks at nt = 16), 2 nt + 1 sweeps (the last pass
    shorter): full field bit-exact."""
    import bench

    cfg = bench._nt_cfg(name, nt)
    u0 = W.laplace_cube(400, dtype=np.float32 if name.endswith("f32") else np.float64)
    ns = 2 * nt + 1
    with cf.ThreadPoolExecutor(1) as ex:
        fut = ex.submit(oracle.gs_lex, u0, None, 1.0, ns)
        got = _run(ctx, capi.stencil_gs_lex, u0, None, 1.0, ns, nt=nt, **cfg)
        ref = fut.result()
    _assert_exact(got, ref, "400^3 %s nt=%d" % (name, nt))


# ------------------------------------------------------------ in-place Jacobi --
@pytest.mark.parametrize("dims", RAGGED + [(45, 38, 29), (33, 9, 70)])
@pytest.mark.parametrize("slab", [0, 1, 2, 7, 32, 1000])
def test_jacobi_inplace_slab_ring(ctx, dims, slab):
    """variant 6: no second grid; z-slabs of `slab` planes into a ring of three buffers,
    copied back two slabs behind: bit-exact for odd and even sweep counts, with f,
    weighted, FP32 (one, two and many slabs)."""
    u0, f0 = W.random_grid(*dims, seed=13, with_f=True)
    for ns, ff, a, b in ((1, f0, 0.0, 0.0), (4, None, 0.0, 0.0), (3, f0, 0.25, 0.125)):
        _assert_exact(_run(ctx, capi.stencil_jacobi, u0, ff, 0.07, ns, tile=(0, 0, slab), variant=6, a=a, b=b),
                      oracle.jacobi(u0, ff, 0.07, ns, a=a, b=(b or None)), "inplace %s slab=%d ns=%d" % (dims, slab, ns))
    u1, f1 = W.random_grid(*dims, seed=14, dtype=np.float32, with_f=True)
    _assert_exact(_run(ctx, capi.stencil_jacobi, u1, f1, 0.07, 5, tile=(0, 0, slab), variant=6),
                  oracle.jacobi(u1, f1, 0.07, 5), "inplace f32 %s slab=%d" % (dims, slab))


def test_jacobi_inplace_needs_no_second_grid():
    """The in-place form's workspace is three slabs, not a grid."""
    c = capi.Context(0)
    n = 128
    u0, _ = W.random_grid(n, n, n, seed=1)
    _run(c, capi.stencil_jacobi, u0, None, 1.0, 3, tile=(0, 0, 16), variant=6)
    grid_bytes = u0.nbytes
    assert c.workspace_bytes < grid_bytes / 2
    with pytest.raises(capi.StencilError):
        capi.stencil_jacobi(c, _dev(u0), None, 1.0, 2, nt=2, variant=6)
    c.close()


def test_throughput_probe(ctx):
    """The throughput probes report positive whole-GPU rates; the integer-pipe binary64 additions all take
    the exact fast path; FP32 issues faster than FP64; the copy kernel's bandwidth is a DRAM figure."""
    r = capi.stencil_probe_throughput(ctx, copy_bytes=1 << 30)
    assert r["int_add_fast_fraction"] == 1.0
    assert r["fp64_ops_per_s"] > 1e11 and r["fp32_ops_per_s"] > r["fp64_ops_per_s"]
    assert r["alu_ops_per_s"] > r["int_add_f64_per_s"] > r["int_add_any_f64_per_s"] > 0
    assert 5e11 < r["copy_bytes_per_s"] < 2e13
    assert r["sm_count"] > 0 and r["clock_khz"] > 0


@pytest.mark.parametrize("smoother,sweeps", [(capi.STENCIL_JACOBI, 50), (capi.STENCIL_GS, 20)])
def test_batched_full_config_sampled(ctx, smoother, sweeps):
    """The full 256-grid batch of uneven Poisson grids (extents multiples of 16 in [32, 192], seed 3) as the
    benchmark runs it: one batched call with the library defaults, then 16 of the grids (every 16th by size
    order, smallest to largest) compared with the oracle element by element."""
    cases = W.batched_poisson(256)
    us = [_dev(c.u) for c in cases]
    fs = [_dev(c.f) for c in cases]
    hs = [c.h for c in cases]
    capi.stencil_batched(ctx, us, fs, hs, [sweeps] * len(cases), smoother)
    torch.cuda.synchronize()
    order = sorted(range(len(cases)), key=lambda i: cases[i].nx * cases[i].ny * cases[i].nz)
    ofn = oracle.jacobi if smoother == capi.STENCIL_JACOBI else oracle.gs_lex
    for i in order[::16]:
        c = cases[i]
        _assert_exact(us[i].cpu().numpy(), ofn(c.u, c.f, c.h, sweeps), "batched grid %d %s" % (i, (c.nx, c.ny, c.nz)))


@pytest.mark.parametrize("smoother", [capi.STENCIL_JACOBI, capi.STENCIL_GS])
def test_autotune_batched_picks_a_valid_config(ctx, smoother):
    """The whole-batch autotuner leaves the grids as they were and returns parameters that the batched call
    runs to the oracle's bits."""
    dims = [(40, 24, 17), (17, 33, 9), (64, 16, 20)]
    grids = [W.random_grid(*d, seed=40 + i, with_f=True) for i, d in enumerate(dims)]
    us = [_dev(u) for u, _ in grids]
    fs = [_dev(f) for _, f in grids]
    hs = [W.grid_h(*d) for d in dims]
    sweeps = [6, 3, 5]
    params, glups = capi.stencil_autotune_batched(ctx, us, fs, hs, sweeps, smoother)
    assert glups > 0
    for u, (u0, _) in zip(us, grids):
        assert np.array_equal(u.cpu().numpy(), u0)
    capi.stencil_batched(ctx, us, fs, hs, sweeps, smoother, **params)
    torch.cuda.synchronize()
    ofn = oracle.jacobi if smoother == capi.STENCIL_JACOBI else oracle.gs_lex
    for i, (u0, f0) in enumerate(grids):
        _assert_exact(us[i].cpu().numpy(), ofn(u0, f0, hs[i], sweeps[i]), "autotuned batch %s grid %d" % (params, i))
