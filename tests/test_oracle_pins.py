"""Pins for the CPU oracle (no GPU): closed forms, textbook routines, brute force
and invariants, each chosen so a plausible mistake in the oracle (a dropped
term, a wrong sign or index, a transposed operand, old/new neighbours swapped,
another summation order) fails at least one of them."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from tests import _forms as F
from tests import _sched as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps
EPS32 = float(np.finfo(np.float32).eps)

# non-cubic so that a transposed stride or extent cannot pass
DIMS = [(7, 5, 6), (9, 4, 3), (5, 5, 5)]
MODES = [(1, 1, 1), (2, 1, 3), (3, 4, 2), (1, 3, 1)]


# ---------------------------------------------------------------- Jacobi ----
@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("mode", MODES)
def test_jacobi_sine_mode_decays_by_analytic_factor(dims, mode):
    """Sec. 3 Jacobi, f = 0, zero Dirichlet: a discrete sine mode is an
    eigenvector; one sweep multiplies it by mu = (cos a + cos b + cos c)/3."""
    nx, ny, nz = dims
    p, q, r = mode
    if p > nx or q > ny or r > nz:
        pytest.skip("mode beyond grid")
    u = F.sine_mode(nx, ny, nz, p, q, r)
    mu = F.jacobi_factor(nx, ny, nz, p, q, r)
    for sweeps in (1, 3):
        out = oracle.jacobi(u, None, 1.0, sweeps)
        np.testing.assert_allclose(out, (mu ** sweeps) * u, rtol=0, atol=12 * sweeps * EPS)


def test_jacobi_weighted_mode_factor():
    """Weighted form a*u + b*sum (Sec. 3 listing): factor a + 6 b mu."""
    nx, ny, nz = 7, 5, 6
    u = F.sine_mode(nx, ny, nz, 2, 1, 3)
    mu = F.jacobi_factor(nx, ny, nz, 2, 1, 3)
    a, b = 1.0 - 0.8, 0.8 / 6.0
    out = oracle.jacobi(u, None, 1.0, 1, a=a, b=b)
    np.testing.assert_allclose(out, (a + 6 * b * mu) * u, rtol=0, atol=16 * EPS)


@pytest.mark.parametrize("dims", DIMS)
def test_jacobi_matches_sparse_operator(dims):
    """u' = b (N u + boundary + h^2 f), N the sparse neighbour-sum matrix."""
    nx, ny, nz = dims
    rng = np.random.default_rng(11)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    h = 0.37
    out = oracle.jacobi(u, f, h, 1)
    ref = (F.neighbour_matrix(nx, ny, nz) @ F.interior(u) + F.boundary_sum(u) + h * h * F.interior(f)) / 6.0
    np.testing.assert_allclose(F.interior(out), ref, rtol=8 * EPS, atol=8 * EPS)
    # the halo is never written
    mask = np.ones(u.shape, bool)
    mask[1:-1, 1:-1, 1:-1] = False
    assert np.array_equal(out[mask], u[mask])


def test_jacobi_two_sweeps_is_operator_squared():
    """Out of place: sweep 2 reads only sweep-1 values (matrix form applied twice)."""
    nx, ny, nz = 6, 5, 4
    rng = np.random.default_rng(3)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    n = F.neighbour_matrix(nx, ny, nz)
    bnd = F.boundary_sum(u)
    x = F.interior(u)
    for _ in range(2):
        x = (n @ x + bnd) / 6.0
    np.testing.assert_allclose(F.interior(oracle.jacobi(u, None, 1.0, 2)), x, rtol=16 * EPS)


# ----------------------------------------------------------- Gauss-Seidel ----
@pytest.mark.parametrize("dims", DIMS)
def test_gs_is_lower_triangular_solve(dims):
    """Lexicographic GS (Sec. 3 second listing) is forward substitution:
    (6 I - L) u_new = U u_old + boundary + h^2 f, L / U the neighbours before /
    after a site in (k, j, i) order."""
    nx, ny, nz = dims
    rng = np.random.default_rng(5)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    h = 0.29
    L, U = F.lex_split(nx, ny, nz)
    m = (6.0 * sp.identity(nx * ny * nz) - L).tocsr()
    rhs = U @ F.interior(u) + F.boundary_sum(u) + h * h * F.interior(f)
    ref = spla.spsolve_triangular(m, rhs, lower=True)
    out = oracle.gs_lex(u, f, h, 1)
    np.testing.assert_allclose(F.interior(out), ref, rtol=64 * EPS, atol=64 * EPS)


@pytest.mark.parametrize("dims", [(4, 4, 4), (1, 1, 6), (6, 1, 1), (3, 5, 7), (1, 1, 1)])
def test_gs_equals_brute_force_sorted_enumeration(dims):
    nx, ny, nz = dims
    rng = np.random.default_rng(7)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    for ff in (None, f):
        out = oracle.gs_lex(u, ff, 0.5, 3)
        ref = S.gs_brute_force(u, ff, 0.5, 3)
        assert np.array_equal(out, ref)


def test_gs_red_black_half_sweeps():
    """Red-black GS: each colour is a simultaneous (Jacobi) update of that
    colour from the current values, red ((i+j+k) even) first."""
    nx, ny, nz = 5, 4, 3
    rng = np.random.default_rng(9)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    n = F.neighbour_matrix(nx, ny, nz)
    bnd = F.boundary_sum(u)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    red = ((i + j + k) % 2 == 0).ravel()
    x = F.interior(u)
    for colour in (red, ~red):
        y = (n @ x + bnd) / 6.0
        x = np.where(colour, y, x)
    np.testing.assert_allclose(F.interior(oracle.gs_rb(u, None, 1.0, 1)), x, rtol=16 * EPS)


def test_gs_red_black_f32_matches_f64_within_single_precision():
    nx, ny, nz = 6, 5, 4
    rng = np.random.default_rng(10)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    out32 = oracle.gs_rb(u.astype(np.float32), f.astype(np.float32), 0.2, 3)
    out64 = oracle.gs_rb(u, f, 0.2, 3)
    assert out32.dtype == np.float32
    np.testing.assert_allclose(out32.astype(np.float64), out64, rtol=0, atol=64 * EPS32)


@pytest.mark.parametrize("smoother", ["jacobi", "gs_lex"])
@pytest.mark.parametrize("with_f", [False, True])
def test_f32_error_against_f64_within_the_rounding_bound(smoother, with_f):
    """FP32 sweeps against FP64 sweeps from the same (FP32-representable) data: one sweep rounds the
    partial sums of the neighbour sum (at most 2..6 max|u|) to 2^-24 relative, 20 units of
    2^-24 max|u| times b = 1/6, plus the multiplication: 4.34 units; with f the bracket's last
    addition and h^2 f add (2 h^2 max|f| / 6 + ...) units.  Both smoothers are convex combinations
    of their neighbours (weights 1/6), so an error's max-norm never grows: after n sweeps
    |u32 - u64| <= n (4.34 max|u| + h^2 max|f|) 2^-24.  A wrong FP32 constant or operation
    breaks it by orders of magnitude."""
    nx, ny, nz = 30, 21, 17
    rng = np.random.default_rng(12)
    u = rng.random((nz + 2, ny + 2, nx + 2)).astype(np.float32)
    f = rng.standard_normal(u.shape).astype(np.float32) if with_f else None
    h = 1.0 / 31
    fn = oracle.jacobi if smoother == "jacobi" else oracle.gs_lex
    for n in (1, 10, 60):
        out32 = fn(u, f, h, n)
        out64 = fn(u.astype(np.float64), None if f is None else f.astype(np.float64), h, n)
        umax = max(np.abs(out64).max(), np.abs(u).max())
        hf = np.float32(h * h) * np.abs(f).max() if with_f else 0.0
        bound = n * (4.34 * umax + hf) * 2.0 ** -24
        err = np.abs(out32.astype(np.float64) - out64).max()
        assert err <= bound, (smoother, with_f, n, err, bound)
        assert err > 0 or n == 0  # FP32 really rounds differently


# ------------------------------------------------- schedules (exactness) ----
@pytest.mark.parametrize("nz", [1, 2, 5, 7, 12])
@pytest.mark.parametrize("slab", [1, 2, 3, 5, 32])
@pytest.mark.parametrize("copy_first", [False, True])
def test_jacobi_slab_ring_is_bit_exact(nz, slab, copy_first):
    """The GPU's in-place Jacobi (three slab buffers, copy-back two slabs behind, in either order
    against the computation of the same launch) gives the serial iterate."""
    rng = np.random.default_rng(nz * 7 + slab)
    u = rng.random((nz + 2, 6, 5))
    f = rng.standard_normal(u.shape)
    for ns in (1, 3):
        np.testing.assert_array_equal(S.jacobi_slab_ring(u, f, 0.3, ns, slab, copy_first), oracle.jacobi(u, f, 0.3, ns))


def test_jacobi_slab_ring_lag_one_breaks():
    """Copying back the slab just before the one being computed overwrites planes it still reads."""
    rng = np.random.default_rng(5)
    u = rng.random((12, 6, 5))
    got = S.jacobi_slab_ring(u, None, 1.0, 1, slab=2, copy_first=True, lag=1)
    assert not np.array_equal(got, oracle.jacobi(u, None, 1.0, 1))


@pytest.mark.parametrize("dims", [(4, 4, 4), (5, 3, 6), (1, 1, 5), (6, 2, 1)])
def test_gs_hyperplane_order_is_bit_exact(dims):
    """Sites with equal i+j+k+2t are independent: updating them level by level
    reproduces the serial sweeps exactly (the pipeline-parallel claim, Sec. 3)."""
    nx, ny, nz = dims
    u, f = (np.random.default_rng(1).random((nz + 2, ny + 2, nx + 2)),
            np.random.default_rng(2).standard_normal((nz + 2, ny + 2, nx + 2)))
    assert np.array_equal(S.gs_hyperplane(u, f, 0.3, 4), oracle.gs_lex(u, f, 0.3, 4))


@pytest.mark.parametrize("tile,nt", [((4, 4, 4), 1), ((3, 2, 4), 1), ((4, 4, 4), 2), ((4, 3, 5), 3),
                                     ((8, 4, 2), 2), ((2, 2, 2), 2), ((5, 5, 5), 4), ((3, 3, 3), 3),
                                     ((4, 4, 4), 4)])
@pytest.mark.parametrize("reverse", [False, True])
def test_gs_skewed_tiles_are_bit_exact(tile, nt, reverse):
    """The skewed-tile schedule (nt sweeps per task, tasks by level I+J+K+c*p)
    reproduces the serial sweeps exactly, whatever the order within a level."""
    nx, ny, nz = 9, 7, 8
    rng = np.random.default_rng(4)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    for nsweeps in (1, nt, 2 * nt + 1):
        ref = oracle.gs_lex(u, f, 0.2, nsweeps)
        out = S.gs_skewed_tiles(u, f, 0.2, nsweeps, tile, nt, reverse)
        assert np.array_equal(out, ref), (tile, nt, nsweeps)


@pytest.mark.parametrize("nt", [2, 4, 6])
def test_jacobi_paper_wavefront_is_bit_exact(nt):
    """Sec. 4 wavefront: nt updates per pass, distance two, odd updates in a
    4-plane ring per update, even updates in place: equals nt plain sweeps
    (no additional computations, no second grid)."""
    nx, ny, nz = 7, 6, 9
    rng = np.random.default_rng(8)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    for ff in (None, f):
        out = S.jacobi_wavefront_paper(u, ff, 0.25, 2 * nt, nt)
        assert np.array_equal(out, oracle.jacobi(u, ff, 0.25, 2 * nt))


# ------------------------------------------------------------ invariants ----
@pytest.mark.parametrize("name", list(F.harmonic_fields(3, 3, 3)))
def test_harmonic_polynomials_are_fixed_points(name):
    nx, ny, nz = 6, 5, 7
    u = F.harmonic_fields(nx, ny, nz)[name]
    scale = np.abs(u).max()
    for fn in (oracle.jacobi, oracle.gs_lex):
        out = fn(u, None, 1.0, 5)
        np.testing.assert_allclose(out, u, rtol=0, atol=40 * EPS * scale)
    r, rn, _ = oracle.residual(u, None, 1.0)
    assert rn <= 40 * EPS * scale * math.sqrt(nx * ny * nz)


@pytest.mark.parametrize("c", [1.0, 0.5, 0.25, 2.0, 3.0])
def test_constant_field_is_bit_exact_fixed_point(c):
    u = np.full((7, 6, 5), c)
    for fn in (oracle.jacobi, oracle.gs_lex):
        assert np.array_equal(fn(u, None, 1.0, 4), u)
    u32 = u.astype(np.float32)
    for fn in (oracle.jacobi, oracle.gs_lex):
        assert np.array_equal(fn(u32, None, 1.0, 4), u32)


def test_constant_not_representable_moves():
    """0.1: b * (6*0.1 summed) does not round back (shows the check is sharp)."""
    u = np.full((5, 5, 5), 0.1)
    assert not np.array_equal(oracle.jacobi(u, None, 1.0, 1), u)


def _golden_sum_order():
    rows = []
    with open(os.path.join(GOLDEN, "sum_order.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows.append((parts[0], [float.fromhex(x) for x in parts[1:7]], float.fromhex(parts[7])))
    return rows


@pytest.mark.parametrize("row", _golden_sum_order())
def test_summation_order_golden(row):
    dtype, (w, e, s, n, b, t), expected = row
    dt = np.float64 if dtype == "f64" else np.float32
    u = np.zeros((3, 3, 3), dtype=dt)
    u[1, 1, 0], u[1, 1, 2], u[1, 0, 1], u[1, 2, 1], u[0, 1, 1], u[2, 1, 1] = w, e, s, n, b, t
    for fn in (oracle.jacobi, oracle.gs_lex):
        out = fn(u, None, 1.0, 1)
        assert float(out[1, 1, 1]) == expected, (dtype, fn.__name__, float(out[1, 1, 1]).hex())


# ------------------------------------------------------------- residual ----
def test_residual_eigenrelation():
    """A phi = lambda phi for a sine mode: r = f - lambda phi."""
    nx, ny, nz = 8, 6, 7
    h = 1.0 / 9
    phi = F.sine_mode(nx, ny, nz, 2, 3, 1)
    lam = F.eigenvalue(nx, ny, nz, 2, 3, 1, h)
    f = np.random.default_rng(2).standard_normal(phi.shape)
    r, rn, fn = oracle.residual(phi, f, h)
    ref = F.interior(f) - lam * F.interior(phi)
    np.testing.assert_allclose(F.interior(r), ref, rtol=0, atol=64 * EPS * lam)
    assert r[0].max() == 0 and r[-1].max() == 0


def test_residual_sparse_form_and_norm():
    nx, ny, nz = 5, 7, 4
    rng = np.random.default_rng(12)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    h = 0.15
    r, rn, fn = oracle.residual(u, f, h)
    au = (6.0 * F.interior(u) - F.neighbour_matrix(nx, ny, nz) @ F.interior(u) - F.boundary_sum(u)) / (h * h)
    np.testing.assert_allclose(F.interior(r), F.interior(f) - au, rtol=1e-13, atol=1e-13 * np.abs(au).max())
    exact = math.sqrt(math.fsum(float(x) ** 2 for x in F.interior(r)))
    assert abs(rn - exact) <= 4 * EPS * exact
    exact_f = math.sqrt(math.fsum(float(x) ** 2 for x in F.interior(f)))
    assert abs(fn - exact_f) <= 4 * EPS * exact_f


# ---------------------------------------------------------------- solves ----
def _sine_rhs(n, modes, amps):
    h = 1.0 / (n + 1)
    f = np.zeros((n + 2,) * 3)
    ustar = np.zeros_like(f)
    for (p, q, r), a in zip(modes, amps):
        phi = F.sine_mode(n, n, n, p, q, r)
        f += a * phi
        ustar += a * phi / F.eigenvalue(n, n, n, p, q, r, h)
    return h, f, ustar


@pytest.mark.parametrize("smoother", [oracle.SMOOTHER_JACOBI, oracle.SMOOTHER_GS])
def test_solve_f64_reaches_closed_form(smoother):
    """-Lap_h u = f with f a sum of sine modes: u* = sum a phi / lambda.  Pins the
    sign of f and the h^2 scaling of the Poisson update."""
    n = 10
    h, f, ustar = _sine_rhs(n, [(1, 1, 1), (2, 1, 3), (1, 4, 2)], [1.0, -0.7, 0.4])
    u0 = np.zeros_like(f)
    u, rel, sweeps, ok = oracle.solve_f64(u0, f, h, smoother, 1e-12, 20000, 50)
    assert ok and rel <= 1e-12
    assert np.abs(u - ustar).max() <= 1e-10 * np.abs(ustar).max()


@pytest.mark.parametrize("smoother", [oracle.SMOOTHER_JACOBI, oracle.SMOOTHER_GS])
def test_solve_mixed_reaches_closed_form(smoother):
    """FP32 inner sweeps + FP64 defect correction reach FP64 accuracy."""
    n = 10
    h, f, ustar = _sine_rhs(n, [(1, 2, 1), (3, 1, 1)], [0.9, 0.3])
    u, rel, its, ok = oracle.solve_mixed(np.zeros_like(f), f, h, smoother, 1e-11, 200, 60)
    assert ok and rel <= 1e-11
    assert np.abs(u - ustar).max() <= 1e-9 * np.abs(ustar).max()
    # one outer iteration is not enough: FP32 alone stalls near 1e-7
    _, rel1, _, ok1 = oracle.solve_mixed(np.zeros_like(f), f, h, smoother, 1e-11, 1, 2000)
    assert not ok1 and rel1 > 1e-9


# ---------------------------------------------------------------- FP32 ----
def test_f32_mode_decay_and_precision():
    nx, ny, nz = 7, 5, 6
    u = F.sine_mode(nx, ny, nz, 2, 1, 3)
    mu = F.jacobi_factor(nx, ny, nz, 2, 1, 3)
    out = oracle.jacobi(u.astype(np.float32), None, 1.0, 2)
    assert out.dtype == np.float32
    np.testing.assert_allclose(out.astype(np.float64), mu * mu * u, rtol=0, atol=24 * EPS32)
    # genuinely single precision: differs from the FP64 result
    assert not np.array_equal(out.astype(np.float64), oracle.jacobi(u, None, 1.0, 2))


def test_f32_gs_is_lower_triangular_solve():
    nx, ny, nz = 6, 5, 4
    rng = np.random.default_rng(21)
    u = rng.random((nz + 2, ny + 2, nx + 2)).astype(np.float32)
    f = rng.standard_normal(u.shape).astype(np.float32)
    h = 0.3
    L, U = F.lex_split(nx, ny, nz)
    m = (6.0 * sp.identity(nx * ny * nz) - L).tocsr()
    u64, f64 = u.astype(np.float64), f.astype(np.float64)
    ref = spla.spsolve_triangular(m, U @ F.interior(u64) + F.boundary_sum(u64) + (h * h) * F.interior(f64), lower=True)
    out = oracle.gs_lex(u, f, h, 1)
    np.testing.assert_allclose(F.interior(out), ref, rtol=64 * EPS32, atol=64 * EPS32)


@pytest.mark.parametrize("tile,nt", [((4, 4, 4), 1), ((4, 4, 4), 2), ((4, 3, 5), 3), ((8, 4, 2), 2),
                                     ((2, 2, 2), 2), ((5, 5, 5), 4), ((3, 3, 3), 3), ((4, 4, 4), 4)])
@pytest.mark.parametrize("reverse", [False, True])
def test_jacobi_skewed_tiles_are_bit_exact(tile, nt, reverse):
    """Jacobi on the same skewed-tile schedule with two parity arrays equals the
    plain two-array sweeps (temporal blocking without extra computation, Sec. 4)."""
    nx, ny, nz = 9, 7, 8
    rng = np.random.default_rng(6)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    for nsweeps in (1, nt, 2 * nt + 1):
        ref = oracle.jacobi(u, f, 0.2, nsweeps)
        out = S.jacobi_skewed_tiles(u, f, 0.2, nsweeps, tile, nt, reverse)
        assert np.array_equal(out, ref), (tile, nt, nsweeps)


def test_skewed_tiles_depth_limit_is_sharp():
    """nt <= min(tile) is needed: with nt = min + 1 the result depends on the
    order of tasks within one level (tasks of a level then share sites)."""
    nx, ny, nz = 9, 7, 8
    rng = np.random.default_rng(6)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    ns = 9
    ref_g, ref_j = oracle.gs_lex(u, f, 0.2, ns), oracle.jacobi(u, f, 0.2, ns)
    assert not np.array_equal(S.gs_skewed_tiles(u, f, 0.2, ns, (3, 3, 3), 4, True), ref_g)
    assert not np.array_equal(S.jacobi_skewed_tiles(u, f, 0.2, ns, (3, 3, 3), 4, True), ref_j)


@pytest.mark.parametrize("tile,nt", [((4, 4, 4), 1), ((3, 2, 4), 1), ((4, 4, 4), 2), ((4, 3, 5), 3),
                                     ((3, 3, 3), 3), ((2, 2, 2), 2)])
def test_dataflow_orders_are_bit_exact(tile, nt):
    """The persistent dataflow kernel runs a task once its dependencies
    (tests/_sched.dataflow_deps) are done, in whatever order the hardware
    picks: random linearisations of that dependency graph must all give the
    serial result, for Gauss-Seidel in place and for Jacobi on two grids."""
    rng = np.random.default_rng(0)
    nx, ny, nz = 9, 7, 8
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    for ns in (1, 2 * nt + 1):
        refs = {"gs": oracle.gs_lex(u, f, 0.2, ns), "jacobi": oracle.jacobi(u, f, 0.2, ns)}
        for _ in range(4):
            order = S.random_dataflow_order(nx, ny, nz, tile, nt, ns, rng)
            for kind in ("gs", "jacobi"):
                assert np.array_equal(S.run_task_order(kind, u, f, 0.2, ns, tile, nt, order), refs[kind])


def test_dataflow_dependency_rule_is_sharp():
    """With only face dependencies on the previous pass (too few for skewed
    tiles), random orders break the result."""
    rng = np.random.default_rng(1)
    nx, ny, nz = 9, 7, 8
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    tile, nt, ns = (4, 4, 4), 2, 5
    ref = oracle.gs_lex(u, f, 0.2, ns)
    orig = S.dataflow_deps
    try:
        S.dataflow_deps = lambda I, J, K, p, nt_, dims: orig(I, J, K, p, 1, dims)
        broken = sum(not np.array_equal(S.run_task_order("gs", u, f, 0.2, ns, tile, nt,
                                                         S.random_dataflow_order(nx, ny, nz, tile, nt, ns, rng)), ref)
                     for _ in range(4))
    finally:
        S.dataflow_deps = orig
    assert broken > 0


# -------------------------------------------------------------- multigrid ----
def _padded(nx, ny, nz):
    return np.zeros((nz + 2, ny + 2, nx + 2))


def _fill_interior(a, fn):
    nz, ny, nx = (s - 2 for s in a.shape)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a[1:-1, 1:-1, 1:-1] = fn(i, j, k)
    return a


@pytest.mark.parametrize("dims", [(7, 5, 9), (5, 5, 5), (11, 3, 7)])
def test_mg_restriction_reproduces_linear_functions(dims):
    """Full weighting is exact for linear functions and its weights sum to one:
    the coarse value equals the fine value at the coarse site's fine position
    (2I+1, 2J+1, 2K+1), for a constant and for each axis separately."""
    nx, ny, nz = dims
    for fn in (lambda i, j, k: 0 * i + 3.0, lambda i, j, k: 2.0 * i - 1.0, lambda i, j, k: 3.0 * j + 0.5,
               lambda i, j, k: -4.0 * k + 2.0, lambda i, j, k: i + 2.0 * j - 3.0 * k):
        r = _fill_interior(_padded(nx, ny, nz), fn)
        fc = oracle.mg_restrict(r)
        want = _fill_interior(_padded((nx - 1) // 2, (ny - 1) // 2, (nz - 1) // 2),
                              lambda I, J, K: fn(2 * I + 1, 2 * J + 1, 2 * K + 1))
        np.testing.assert_array_equal(fc, want)


def test_mg_restriction_weights_by_position():
    """A unit value at each of the 27 fine sites around a coarse site: every
    coarse site C receives the product over the axes of w(fine - (2C+1)), with
    w(0) = 1/2, w(+-1) = 1/4 and 0 beyond (a transposed axis, a dropped term or
    a wrong weight changes one of the 27 images)."""
    nx, ny, nz = 7, 9, 5
    I, J, K = 1, 2, 1
    w1 = lambda d: np.where(d == 0, 0.5, np.where(np.abs(d) == 1, 0.25, 0.0))
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                fi, fj, fk = 2 * I + 1 + dx, 2 * J + 1 + dy, 2 * K + 1 + dz
                r = _padded(nx, ny, nz)
                r[fk + 1, fj + 1, fi + 1] = 1.0
                fc = oracle.mg_restrict(r)
                want = _fill_interior(_padded((nx - 1) // 2, (ny - 1) // 2, (nz - 1) // 2),
                                      lambda Ic, Jc, Kc: w1(fi - (2 * Ic + 1)) * w1(fj - (2 * Jc + 1)) *
                                      w1(fk - (2 * Kc + 1)))
                np.testing.assert_array_equal(fc, want)
                assert fc[K + 1, J + 1, I + 1] == 0.5 ** (3 + abs(dx) + abs(dy) + abs(dz))


@pytest.mark.parametrize("dims", [(9, 7, 11), (5, 5, 5)])
def test_mg_prolongation_reproduces_linear_functions(dims):
    """Trilinear interpolation is exact for linear functions away from the
    boundary (whose coarse values are the zero halo): a coarse linear function
    comes back as the same function on the fine sites between coarse sites."""
    nx, ny, nz = dims
    g = lambda i, j, k: 0.5 * i - 2.0 * j + 3.0 * k + 1.25
    e = _fill_interior(_padded((nx - 1) // 2, (ny - 1) // 2, (nz - 1) // 2),
                       lambda I, J, K: g(2 * I + 1, 2 * J + 1, 2 * K + 1))
    u = oracle.mg_prolong_add(_padded(nx, ny, nz), e)
    want = _fill_interior(_padded(nx, ny, nz), g)
    np.testing.assert_array_equal(u[2:-2, 2:-2, 2:-2], want[2:-2, 2:-2, 2:-2])
    # added, not assigned: a second application doubles it
    u2 = oracle.mg_prolong_add(u, e)
    np.testing.assert_array_equal(u2[2:-2, 2:-2, 2:-2], 2 * want[2:-2, 2:-2, 2:-2])


def test_mg_prolongation_of_a_spike_is_the_hat_function():
    """A unit coarse value at (I,J,K) spreads as the product of 1D hats
    (1 at 2I+1, 1/2 at 2I and 2I+2), zero elsewhere; near the boundary the
    missing coarse neighbour is the zero halo."""
    nx, ny, nz = 9, 7, 5
    for I, J, K in ((1, 1, 0), (0, 2, 1), (3, 0, 1)):
        e = _padded((nx - 1) // 2, (ny - 1) // 2, (nz - 1) // 2)
        e[K + 1, J + 1, I + 1] = 1.0
        u = oracle.mg_prolong_add(_padded(nx, ny, nz), e)
        hat = lambda x, c: np.maximum(0.0, 1.0 - np.abs(x - c) / 2.0)
        want = _fill_interior(_padded(nx, ny, nz),
                              lambda i, j, k: hat(i, 2 * I + 1) * hat(j, 2 * J + 1) * hat(k, 2 * K + 1))
        np.testing.assert_array_equal(u, want)


@pytest.mark.parametrize("smoother,bound", [(oracle.MG_GS, 0.2), (oracle.MG_JACOBI, 0.32), (oracle.MG_GS_RB, 0.2)])
def test_mg_vcycle_reduces_the_error_by_a_fixed_factor(smoother, bound):
    """Laplace problem with zero Dirichlet data (solution 0) from a random start:
    every V(2,2) cycle shrinks the error by a grid-independent factor (textbook
    multigrid; ~0.15 for Gauss-Seidel, ~0.27 for Jacobi with omega = 6/7).  A
    wrong sign of the correction, a wrong h scaling of a coarse level or a
    transfer that is not a weighted mean stalls or diverges."""
    rng = np.random.default_rng(7)
    for n in (15, 31):
        u = _padded(n, n, n)
        u[1:-1, 1:-1, 1:-1] = rng.random((n, n, n))
        prev = np.abs(u).max()
        for _ in range(4):
            u, _, _, _ = oracle.mg_solve(u, None, 1.0 / (n + 1), smoother, 2, 2, 10, 8, 0.0, 1)
            cur = np.abs(u).max()
            assert cur <= bound * prev
            prev = cur


@pytest.mark.parametrize("smoother", [oracle.MG_GS, oracle.MG_JACOBI, oracle.MG_GS_RB])
def test_mg_solve_reaches_closed_form(smoother):
    """f a sum of sine modes: the V-cycles converge to u* = sum a phi / lambda
    (the discrete solution, to rounding) within a handful of cycles."""
    n = 31
    h, f, ustar = _sine_rhs(n, [(1, 1, 1), (2, 1, 3), (5, 7, 2)], [1.0, -0.7, 0.4])
    u, rel, cycles, ok = oracle.mg_solve(np.zeros_like(f), f, h, smoother, 2, 2, 20, 8, 1e-11, 40)
    assert ok and rel <= 1e-11
    assert cycles <= (25 if smoother == oracle.MG_JACOBI else 15)
    assert np.abs(u - ustar).max() <= 1e-9 * np.abs(ustar).max()


def test_mg_one_level_is_plain_smoothing():
    """With one level (max_levels = 1, or an even extent that cannot coarsen) a
    cycle is ncoarse sweeps of the smoother: Gauss-Seidel, and Jacobi with
    a = b = 1/7."""
    rng = np.random.default_rng(3)
    for dims, levels in (((7, 5, 9), 1), ((8, 7, 7), 6)):
        nx, ny, nz = dims
        u0 = rng.random((nz + 2, ny + 2, nx + 2))
        f = _padded(nx, ny, nz)
        f[1:-1, 1:-1, 1:-1] = rng.standard_normal((nz, ny, nx))
        h = 0.1
        got, _, _, _ = oracle.mg_solve(u0, f, h, oracle.MG_GS, 3, 3, 5, levels, 0.0, 1)
        np.testing.assert_array_equal(got, oracle.gs_lex(u0, f, h, 5))
        got, _, _, _ = oracle.mg_solve(u0, f, h, oracle.MG_JACOBI, 3, 3, 5, levels, 0.0, 1)
        np.testing.assert_array_equal(got, oracle.jacobi(u0, f, h, 5, a=1.0 / 7.0, b=1.0 / 7.0))
        got, _, _, _ = oracle.mg_solve(u0, f, h, oracle.MG_GS_RB, 3, 3, 5, levels, 0.0, 1)
        np.testing.assert_array_equal(got, oracle.gs_rb(u0, f, h, 5))


# ------------------------------------------------- FP32 sparse forms ----
def test_gs_red_black_f32_half_sweeps():
    """FP32 red-black GS against its own definition (each colour a simultaneous update of
    that colour from the current values, red first), evaluated in float64 from the FP32
    oracle's own previous colour: every site within a few binary32 roundings.  A colour swap
    or a wrong neighbour in the FP32 copy moves sites by O(1)."""
    nx, ny, nz = 6, 5, 4
    rng = np.random.default_rng(21)
    u = rng.random((nz + 2, ny + 2, nx + 2)).astype(np.float32)
    f = rng.standard_normal(u.shape).astype(np.float32)
    h = 0.2
    n = F.neighbour_matrix(nx, ny, nz)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    red = ((i + j + k) % 2 == 0).ravel()
    bnd = F.boundary_sum(u.astype(np.float64))
    hh = float(np.float32(h * h))
    x = F.interior(u)
    out = oracle.gs_rb(u, f, h, 1)
    assert out.dtype == np.float32
    for colour in (red, ~red):
        y = (n @ x + bnd + hh * F.interior(f)) * float(oracle.B32)
        x = np.where(colour, y, x)
    scale = np.abs(x).max() + hh * np.abs(f).max()
    np.testing.assert_allclose(F.interior(out), x, rtol=0, atol=16 * EPS32 * scale)
    # black only after red: the red half alone differs from the full sweep on black sites
    y = (n @ F.interior(u) + bnd + hh * F.interior(f)) * float(oracle.B32)
    assert np.abs(np.where(~red, F.interior(out) - y, 0)).max() > 1e-3


@pytest.mark.parametrize("with_f", [False, True])
def test_jacobi_f32_weighted_sparse_form(with_f):
    """FP32 weighted Jacobi u' = a u + b (N u + bnd + hh f) with a = b = (float)(1/7): the sparse
    form in float64 from the same float32 data, within a few binary32 roundings per sweep, and
    the mode factor a + 6 b mu on a sine mode.  A dropped a*u term, a wrong weight or a wrong
    neighbour fails by far more."""
    nx, ny, nz = 7, 6, 5
    rng = np.random.default_rng(22)
    u = rng.random((nz + 2, ny + 2, nx + 2)).astype(np.float32)
    f = rng.standard_normal(u.shape).astype(np.float32) if with_f else None
    h = 0.125
    a = b = float(np.float32(1.0 / 7.0))
    hh = float(np.float32(h * h))
    n = F.neighbour_matrix(nx, ny, nz)
    bnd = F.boundary_sum(u.astype(np.float64))
    x = F.interior(u)
    for sweeps in range(1, 4):
        x = a * x + b * (n @ x + bnd + (hh * F.interior(f) if with_f else 0.0))
        out = oracle.jacobi(u, f, h, sweeps, a=a, b=b)
        assert out.dtype == np.float32
        scale = np.abs(x).max() + (hh * np.abs(f).max() if with_f else 0.0)
        np.testing.assert_allclose(F.interior(out), x, rtol=0, atol=8 * sweeps * EPS32 * scale)
    phi = F.sine_mode(nx, ny, nz, 2, 1, 3).astype(np.float32)
    mu = F.jacobi_factor(nx, ny, nz, 2, 1, 3)
    out = oracle.jacobi(phi, None, 1.0, 2, a=a, b=b)
    np.testing.assert_allclose(out.astype(np.float64), (a + 6 * b * mu) ** 2 * phi.astype(np.float64), rtol=0,
                               atol=32 * EPS32)


# -------------------------------------------- FP32 and mixed multigrid ----
def test_residual_f32_eigenrelation_and_sparse_form():
    """FP32 residual: r = f - lambda phi for a sine mode, and the sparse form (6u - N u - bnd)/h^2
    on random data, both within binary32 rounding of the FP32 operations; a harmonic polynomial
    with small integer values (exact in float32) has r exactly 0 with f = 0."""
    nx, ny, nz = 8, 6, 7
    h = 1.0 / 9
    phi = F.sine_mode(nx, ny, nz, 2, 3, 1)
    lam = F.eigenvalue(nx, ny, nz, 2, 3, 1, h)
    f = np.random.default_rng(2).standard_normal(phi.shape)
    r = oracle.residual32(phi.astype(np.float32), f.astype(np.float32), h)
    assert r.dtype == np.float32
    ref = F.interior(f.astype(np.float32)) - lam * F.interior(phi.astype(np.float32))
    np.testing.assert_allclose(F.interior(r), ref, rtol=0, atol=64 * EPS32 * (lam + np.abs(f).max()))
    assert r[0].max() == 0 and r[-1].max() == 0
    rng = np.random.default_rng(23)
    u = rng.random((nz + 2, ny + 2, nx + 2)).astype(np.float32)
    r = oracle.residual32(u, None, 0.15)
    au = (6.0 * F.interior(u) - F.neighbour_matrix(nx, ny, nz) @ F.interior(u) - F.boundary_sum(u.astype(np.float64)))
    au = au * float(np.float32(1.0 / (0.15 * 0.15)))
    np.testing.assert_allclose(F.interior(r), -au, rtol=0, atol=64 * EPS32 * np.abs(au).max() + 1e-30)
    for name, field in F.harmonic_fields(nx, ny, nz).items():
        if name in ("x+2y-3z", "x2-y2", "xy+yz+zx"):
            r = oracle.residual32(field.astype(np.float32), None, 0.5)
            assert not np.any(r), name


@pytest.mark.parametrize("dims", [(7, 5, 9), (11, 3, 7)])
def test_mg_f32_transfers_are_exact_on_linear_functions(dims):
    """FP32 full weighting and trilinear prolongation: a linear function with dyadic values (exact
    in float32, as every intermediate 1/4 and 1/2 multiple is) is reproduced exactly, the 27
    restriction weights are the products of (1/4, 1/2, 1/4), and a coarse spike prolongs to the
    product of hats -- the FP64 transfers' pins, now on the binary32 copies."""
    nx, ny, nz = dims
    for fn in (lambda i, j, k: 0 * i + 3.0, lambda i, j, k: i + 2.0 * j - 3.0 * k + 0.5):
        r = _fill_interior(_padded(nx, ny, nz), fn).astype(np.float32)
        fc = oracle.mg_restrict(r)
        assert fc.dtype == np.float32
        want = _fill_interior(_padded((nx - 1) // 2, (ny - 1) // 2, (nz - 1) // 2),
                              lambda I, J, K: fn(2 * I + 1, 2 * J + 1, 2 * K + 1))
        np.testing.assert_array_equal(fc, want.astype(np.float32))
    w1 = lambda d: np.where(d == 0, 0.5, np.where(np.abs(d) == 1, 0.25, 0.0))
    I, J, K = 1, min(1, (ny - 1) // 2 - 1), 1
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                fi, fj, fk = 2 * I + 1 + dx, 2 * J + 1 + dy, 2 * K + 1 + dz
                r = _padded(nx, ny, nz).astype(np.float32)
                r[fk + 1, fj + 1, fi + 1] = 1.0
                want = _fill_interior(_padded((nx - 1) // 2, (ny - 1) // 2, (nz - 1) // 2),
                                      lambda Ic, Jc, Kc: w1(fi - (2 * Ic + 1)) * w1(fj - (2 * Jc + 1)) *
                                      w1(fk - (2 * Kc + 1)))
                np.testing.assert_array_equal(oracle.mg_restrict(r), want.astype(np.float32))
    g = lambda i, j, k: 0.5 * i - 2.0 * j + 3.0 * k + 1.25
    e = _fill_interior(_padded((nx - 1) // 2, (ny - 1) // 2, (nz - 1) // 2),
                       lambda I, J, K: g(2 * I + 1, 2 * J + 1, 2 * K + 1)).astype(np.float32)
    u = oracle.mg_prolong_add(_padded(nx, ny, nz).astype(np.float32), e)
    assert u.dtype == np.float32
    want = _fill_interior(_padded(nx, ny, nz), g)
    np.testing.assert_array_equal(u[2:-2, 2:-2, 2:-2], want[2:-2, 2:-2, 2:-2].astype(np.float32))
    e = _padded((nx - 1) // 2, (ny - 1) // 2, (nz - 1) // 2).astype(np.float32)
    e[1, 1, 2] = 1.0  # coarse (I, J, K) = (1, 0, 0)
    u = oracle.mg_prolong_add(_padded(nx, ny, nz).astype(np.float32), e)
    hat = lambda x, c: np.maximum(0.0, 1.0 - np.abs(x - c) / 2.0)
    want = _fill_interior(_padded(nx, ny, nz), lambda i, j, k: hat(i, 3) * hat(j, 1) * hat(k, 1))
    np.testing.assert_array_equal(u, want.astype(np.float32))


@pytest.mark.parametrize("smoother,bound", [(oracle.MG_GS, 0.2), (oracle.MG_JACOBI, 0.32), (oracle.MG_GS_RB, 0.2)])
def test_mg_f32_vcycle_reduces_the_error_by_a_fixed_factor(smoother, bound):
    """The FP32 V(2,2) cycle on the zero-data Laplace problem shrinks a random error by the
    textbook grid-independent factor while the error is far above the binary32 floor."""
    rng = np.random.default_rng(8)
    for n in (15, 31):
        u = _padded(n, n, n).astype(np.float32)
        u[1:-1, 1:-1, 1:-1] = rng.random((n, n, n))
        f = np.zeros_like(u)
        prev = np.abs(u).max()
        for _ in range(4):
            u = oracle.mg_cycles32(u, f, 1.0 / (n + 1), smoother, 2, 2, 10, 8, 1)
            cur = float(np.abs(u).max())
            assert cur <= bound * prev
            prev = cur


def test_mg_f32_one_level_is_plain_fp32_smoothing():
    rng = np.random.default_rng(4)
    for dims, levels in (((7, 5, 9), 1), ((8, 7, 7), 6)):
        nx, ny, nz = dims
        u0 = rng.random((nz + 2, ny + 2, nx + 2)).astype(np.float32)
        f = _padded(nx, ny, nz).astype(np.float32)
        f[1:-1, 1:-1, 1:-1] = rng.standard_normal((nz, ny, nx))
        h = 0.1
        got = oracle.mg_cycles32(u0, f, h, oracle.MG_GS, 3, 3, 5, levels, 1)
        np.testing.assert_array_equal(got, oracle.gs_lex(u0, f, h, 5))
        got = oracle.mg_cycles32(u0, f, h, oracle.MG_JACOBI, 3, 3, 5, levels, 1)
        np.testing.assert_array_equal(got, oracle.jacobi(u0, f, h, 5, a=float(np.float32(1 / 7)),
                                                         b=float(np.float32(1 / 7))))
        got = oracle.mg_cycles32(u0, f, h, oracle.MG_GS_RB, 3, 3, 5, levels, 1)
        np.testing.assert_array_equal(got, oracle.gs_rb(u0, f, h, 5))


@pytest.mark.parametrize("smoother", [oracle.MG_GS, oracle.MG_JACOBI, oracle.MG_GS_RB])
def test_solve_mixed_mg_reaches_closed_form(smoother):
    """Defect correction with FP32 V-cycles inside: the FP64 residual reaches 1e-11 and u the
    closed-form discrete solution u* = sum a phi / lambda, in about as many outer iterations as
    the FP64 multigrid needs cycles; FP32 cycles alone (one outer iteration, many cycles) stall
    near the binary32 floor, so the FP64 correction is what reaches FP64 accuracy."""
    n = 31
    h, f, ustar = _sine_rhs(n, [(1, 1, 1), (2, 1, 3), (5, 7, 2)], [1.0, -0.7, 0.4])
    u, rel, outer, ok = oracle.solve_mixed_mg(np.zeros_like(f), f, h, smoother, 2, 2, 20, 8, 1e-11, 40, 1)
    assert ok and rel <= 1e-11
    assert np.abs(u - ustar).max() <= 1e-9 * np.abs(ustar).max()
    _, _, cycles, _ = oracle.mg_solve(np.zeros_like(f), f, h, smoother, 2, 2, 20, 8, 1e-11, 40)
    assert outer <= cycles + 3, (outer, cycles)
    _, rel1, _, ok1 = oracle.solve_mixed_mg(np.zeros_like(f), f, h, smoother, 2, 2, 20, 8, 1e-11, 1, 30)
    assert not ok1 and rel1 > 1e-9


def test_solve_mixed_mg_one_outer_step_is_its_definition():
    """One outer iteration equals the steps written out with the pinned pieces: r from the FP64
    residual, rounded to float32, FP32 cycles from zero, u + (double) e."""
    n = 15
    rng = np.random.default_rng(5)
    u0 = _padded(n, n, n)
    u0[1:-1, 1:-1, 1:-1] = rng.random((n, n, n))
    f = _padded(n, n, n)
    f[1:-1, 1:-1, 1:-1] = rng.standard_normal((n, n, n))
    h = 1.0 / (n + 1)
    got, _, its, _ = oracle.solve_mixed_mg(u0, f, h, oracle.MG_GS, 2, 2, 10, 8, 0.0, 1, 2)
    assert its == 1
    r, _, _ = oracle.residual(u0, f, h)
    e = oracle.mg_cycles32(np.zeros(u0.shape, np.float32), r.astype(np.float32), h, oracle.MG_GS, 2, 2, 10, 8, 2)
    want = u0.copy()
    want[1:-1, 1:-1, 1:-1] += e[1:-1, 1:-1, 1:-1].astype(np.float64)
    np.testing.assert_array_equal(got, want)
