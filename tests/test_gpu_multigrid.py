"""GPU parity of the multigrid V-cycle solve (stencil_mg_solve) against the CPU
oracle: the same cycles give the same bits (smoothers, residual, full-weighting
restriction and trilinear prolongation all in one fixed order of IEEE
operations); the relative residual agrees to the reduction-order tolerance."""
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
SM = {"jacobi": (capi.STENCIL_JACOBI, oracle.MG_JACOBI), "gs": (capi.STENCIL_GS, oracle.MG_GS),
      "gs_rb": (capi.STENCIL_GS_RB, oracle.MG_GS_RB)}


@pytest.fixture(scope="module")
def ctx():
    c = capi.Context(0)
    yield c
    c.close()


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _assert_exact(got, ref, what):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        i = tuple(bad[0])
        raise AssertionError("%s: %d sites differ, first %s got %r want %r" % (what, len(bad), i, got[i], ref[i]))


def _case(ctx, u0, f0, h, smoother, nu1, nu2, ncoarse, levels, cycles):
    sg, so = SM[smoother]
    u = _dev(u0)
    rel, cyc, _ = capi.stencil_mg_solve(ctx, u, _dev(f0), h, sg, nu1=nu1, nu2=nu2, ncoarse=ncoarse,
                                        max_levels=levels, rtol=0.0, max_cycles=cycles)
    torch.cuda.synchronize()
    ref, rrel, rcyc, _ = oracle.mg_solve(u0, f0, h, so, nu1, nu2, ncoarse, levels, 0.0, cycles)
    assert cyc == rcyc == cycles
    assert abs(rel - rrel) <= 1e-12 * max(rrel, 1e-300)
    return u.cpu().numpy(), ref


@pytest.mark.parametrize("smoother", ["gs", "jacobi", "gs_rb"])
@pytest.mark.parametrize("dims", [(31, 31, 31), (15, 7, 31), (9, 9, 9), (63, 15, 7), (3, 3, 3), (1, 5, 7),
                                  (12, 9, 9), (45, 37, 23)])
def test_mg_vcycle_bit_exact(ctx, smoother, dims):
    """Cubic, non-cubic and ragged grids (several levels, levels of one cell,
    extents that cannot coarsen), Poisson and Laplace, two cycles."""
    nx, ny, nz = dims
    u0, f0 = W.random_grid(nx, ny, nz, seed=sum(dims), with_f=True)
    h = 1.0 / (max(dims) + 1)
    for f in (f0, None):
        got, ref = _case(ctx, u0, f, h, smoother, 2, 1, 7, 32, 2)
        _assert_exact(got, ref, "mg %s %s f=%s" % (smoother, dims, f is not None))


@pytest.mark.parametrize("levels,nu1,nu2,ncoarse", [(1, 2, 2, 3), (2, 1, 0, 5), (3, 0, 2, 1), (32, 3, 3, 0)])
def test_mg_cycle_shapes(ctx, levels, nu1, nu2, ncoarse):
    """Depth limits and sweep counts, including no pre-smoothing and no coarse sweeps."""
    u0, f0 = W.random_grid(31, 15, 31, seed=levels, with_f=True)
    for smoother in ("gs", "jacobi", "gs_rb"):
        got, ref = _case(ctx, u0, f0, 1.0 / 32, smoother, nu1, nu2, ncoarse, levels, 2)
        _assert_exact(got, ref, "mg shape %s %s" % (smoother, (levels, nu1, nu2, ncoarse)))


@pytest.mark.parametrize("n", [127, 255])
def test_mg_full_field_large(ctx, n):
    """127^3 and 255^3 (7 and 8 levels, grids above L2 at 255^3): three GS V(2,2)
    cycles, full field bit-exact."""
    u0, f0 = W.random_grid(n, n, n, seed=n, with_f=True)
    got, ref = _case(ctx, u0, f0, 1.0 / (n + 1), "gs", 2, 2, 20, 32, 3)
    _assert_exact(got, ref, "mg %d^3" % n)


@pytest.mark.parametrize("smoother", ["gs", "jacobi"])
def test_mg_solve_converges_to_closed_form(ctx, smoother):
    """Sine-mode right-hand side: the solve reaches rtol and the discrete solution
    u* = sum a phi / lambda."""
    n = 63
    h = 1.0 / (n + 1)
    modes, amps = [(1, 1, 1), (2, 3, 1), (7, 5, 9)], [1.0, -0.6, 0.3]
    f = np.zeros((n + 2,) * 3)
    ustar = np.zeros_like(f)
    ii = np.arange(1, n + 1)
    for (p, q, r), a in zip(modes, amps):
        phi = np.zeros_like(f)
        phi[1:-1, 1:-1, 1:-1] = (np.sin(np.pi * r * ii * h)[:, None, None] * np.sin(np.pi * q * ii * h)[None, :, None] *
                                 np.sin(np.pi * p * ii * h)[None, None, :])
        lam = (6 - 2 * np.cos(np.pi * p * h) - 2 * np.cos(np.pi * q * h) - 2 * np.cos(np.pi * r * h)) / (h * h)
        f += a * phi
        ustar += a * phi / lam
    u = _dev(np.zeros_like(f))
    rel, cycles, ok = capi.stencil_mg_solve(ctx, u, _dev(f), h, SM[smoother][0], rtol=1e-10, max_cycles=60)
    assert ok and rel <= 1e-10 and cycles <= 30
    got = u.cpu().numpy()
    assert np.abs(got - ustar).max() <= 1e-8 * np.abs(ustar).max()


def test_mg_rejects_bad_arguments(ctx):
    u = _dev(W.random_grid(7, 7, 7, seed=1)[0])
    with pytest.raises(capi.StencilError):
        capi.stencil_mg_solve(ctx, u, None, 0.0, capi.STENCIL_GS)
    with pytest.raises(capi.StencilError):
        capi.stencil_mg_solve(ctx, u, None, 0.1, 7)
    with pytest.raises(capi.StencilError):
        capi.stencil_mg_solve(ctx, u, None, 0.1, capi.STENCIL_GS, max_levels=0)
    with pytest.raises(capi.StencilError):
        capi.stencil_mg_solve(ctx, u, None, 0.1, capi.STENCIL_GS, nu1=-1)


# ------------------------------------------------ mixed-precision multigrid ----
def _mixed_case(ctx, u0, f0, h, smoother, nu1, nu2, ncoarse, levels, outer, inner):
    sg, so = SM[smoother]
    u = _dev(u0)
    rel, its, _ = capi.stencil_solve_mixed_mg(ctx, u, _dev(f0), h, sg, nu1=nu1, nu2=nu2, ncoarse=ncoarse,
                                              max_levels=levels, rtol=0.0, max_outer=outer, inner_cycles=inner)
    torch.cuda.synchronize()
    ref, rrel, rits, _ = oracle.solve_mixed_mg(u0, f0, h, so, nu1, nu2, ncoarse, levels, 0.0, outer, inner)
    assert its == rits == outer
    assert abs(rel - rrel) <= 1e-12 * max(rrel, 1e-300)
    return u.cpu().numpy(), ref


@pytest.mark.parametrize("smoother", ["gs", "jacobi", "gs_rb"])
@pytest.mark.parametrize("dims", [(31, 31, 31), (15, 7, 31), (63, 15, 7), (3, 3, 3), (1, 5, 7), (12, 9, 9),
                                  (45, 37, 23)])
def test_mixed_mg_bit_exact(ctx, smoother, dims):
    """FP64 residual rounded to FP32, FP32 V-cycles (FP32 smoothers, FP32 residual, FP32
    transfers), FP64 correction: two outer iterations of one and of two inner cycles, Poisson and
    Laplace, on grids with several levels, one-cell levels and extents that cannot coarsen."""
    nx, ny, nz = dims
    u0, f0 = W.random_grid(nx, ny, nz, seed=3 * sum(dims), with_f=True)
    h = 1.0 / (max(dims) + 1)
    for f, inner in ((f0, 1), (None, 2)):
        got, ref = _mixed_case(ctx, u0, f, h, smoother, 2, 2, 10, 32, 2, inner)
        _assert_exact(got, ref, "mixed mg %s %s f=%s" % (smoother, dims, f is not None))


@pytest.mark.parametrize("levels,nu1,nu2,ncoarse", [(1, 2, 2, 3), (3, 0, 2, 1), (32, 3, 1, 0)])
def test_mixed_mg_cycle_shapes(ctx, levels, nu1, nu2, ncoarse):
    u0, f0 = W.random_grid(31, 15, 31, seed=10 + levels, with_f=True)
    for smoother in ("gs", "jacobi", "gs_rb"):
        got, ref = _mixed_case(ctx, u0, f0, 1.0 / 32, smoother, nu1, nu2, ncoarse, levels, 2, 1)
        _assert_exact(got, ref, "mixed mg shape %s %s" % (smoother, (levels, nu1, nu2, ncoarse)))


@pytest.mark.parametrize("smoother", ["gs", "jacobi", "gs_rb"])
def test_mixed_mg_reaches_1e10_like_fp64_mg(ctx, smoother):
    """The sine-mode problem (8 modes + noise) at 63^3: the mixed solve reaches ||r||/||f|| <= 1e-10
    in as many outer iterations (+-1) as the FP64 multigrid needs cycles, and the two solutions agree
    to the accuracy the residual allows."""
    p = W.sine_modes_problem(63)
    u64 = _dev(np.zeros_like(p.f))
    rel64, cyc, ok64 = capi.stencil_mg_solve(ctx, u64, _dev(p.f), p.h, SM[smoother][0], rtol=1e-10, max_cycles=60)
    um = _dev(np.zeros_like(p.f))
    relm, outer, okm = capi.stencil_solve_mixed_mg(ctx, um, _dev(p.f), p.h, SM[smoother][0], rtol=1e-10,
                                                   max_outer=60)
    assert ok64 and okm and rel64 <= 1e-10 and relm <= 1e-10
    assert abs(outer - cyc) <= 1, (outer, cyc)
    a, b = u64.cpu().numpy(), um.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-8 * np.abs(a).max()


def test_mixed_mg_full_size_one_outer_iteration(ctx):
    """The 511^3 sine-mode problem (the largest cube below 512 whose levels nest; 9 levels) as the
    mixed solve runs it: one outer iteration of one FP32 Gauss-Seidel V(2,2) cycle, full field
    bit-exact against the oracle."""
    p = W.sine_modes_problem(511)
    got, ref = _mixed_case(ctx, np.zeros_like(p.f), p.f, p.h, "gs", 2, 2, 20, 32, 1, 1)
    _assert_exact(got, ref, "mixed mg 511^3")


def test_mixed_sweeps_full_size_two_outer_iterations(ctx):
    """The 512^3 sine-mode problem with plain FP32 sweeps inside (stencil_solve_mixed): two outer
    iterations of 4 Gauss-Seidel sweeps, full field bit-exact against the oracle."""
    p = W.sine_modes_problem(512)
    u = _dev(np.zeros_like(p.f))
    rel, its, _ = capi.stencil_solve_mixed(ctx, u, _dev(p.f), p.h, capi.STENCIL_GS, 0.0, 2, 4)
    torch.cuda.synchronize()
    ref, rrel, rits, _ = oracle.solve_mixed(np.zeros_like(p.f), p.f, p.h, oracle.SMOOTHER_GS, 0.0, 2, 4)
    assert its == rits == 2
    assert abs(rel - rrel) <= 1e-12 * rrel
    _assert_exact(u.cpu().numpy(), ref, "mixed sweeps 512^3")
