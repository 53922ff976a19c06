"""Parallel schedules restated on the CPU (test helpers, numpy).

Each function reorders the same site updates as the plain serial loops and
must reproduce them bit for bit: that is the paper's claim for the pipelined /
wavefront Gauss-Seidel ("retains the same algorithm as a sequential
Gauss-Seidel", Sec. 3 and Sec. 5) and for temporal blocking ("no additional
computations", Sec. 4).  The site formula is the canonical one,
b*(((((W+E)+S)+N)+B)+T + h*h*f), evaluated with numpy elementwise IEEE
operations; arrays are padded (nz+2, ny+2, nx+2).
"""
from __future__ import annotations

import itertools

import numpy as np


def _update(src: np.ndarray, f, k, j, i, b, hh):
    """Vectorised site update at interior coordinates (arrays k, j, i, 0-based),
    reading neighbours from ``src``; returns the new values (not stored)."""
    K, J, I = k + 1, j + 1, i + 1
    s = src[K, J, I - 1] + src[K, J, I + 1]
    s = s + src[K, J - 1, I]
    s = s + src[K, J + 1, I]
    s = s + src[K - 1, J, I]
    s = s + src[K + 1, J, I]
    if f is not None:
        s = s + hh * f[K, J, I]
    return b * s


def _consts(u, h):
    if u.dtype == np.float32:
        return np.float32(1.0 / 6.0), np.float32(h * h)
    return np.float64(1.0 / 6.0), np.float64(h * h)


def gs_brute_force(u: np.ndarray, f=None, h: float = 1.0, nsweeps: int = 1) -> np.ndarray:
    """Pure-Python Gauss-Seidel: sites visited by explicitly sorting all (k, j, i)
    tuples; Python floats are IEEE binary64.  Tiny grids only."""
    nz, ny, nx = (s - 2 for s in u.shape)
    w = {idx: float(v) for idx, v in np.ndenumerate(u)}
    fv = None if f is None else {idx: float(v) for idx, v in np.ndenumerate(f)}
    b, hh = 1.0 / 6.0, h * h
    order = sorted(itertools.product(range(nz), range(ny), range(nx)))
    for _ in range(nsweeps):
        for (k, j, i) in order:
            K, J, I = k + 1, j + 1, i + 1
            s = w[(K, J, I - 1)] + w[(K, J, I + 1)]
            s = s + w[(K, J - 1, I)]
            s = s + w[(K, J + 1, I)]
            s = s + w[(K - 1, J, I)]
            s = s + w[(K + 1, J, I)]
            if fv is not None:
                s = s + hh * fv[(K, J, I)]
            w[(K, J, I)] = b * s
    out = np.empty_like(u)
    for idx in w:
        out[idx] = w[idx]
    return out


def gs_hyperplane(u: np.ndarray, f=None, h: float = 1.0, nsweeps: int = 1) -> np.ndarray:
    """Gauss-Seidel by levels L = i + j + k + 2t: every site of sweep t lies on
    level i+j+k+2t; all sites of one level are independent and are updated
    together (read all, then write all)."""
    u = u.copy()
    nz, ny, nx = (s - 2 for s in u.shape)
    b, hh = _consts(u, h)
    if nsweeps == 0 or nx * ny * nz == 0:
        return u
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = (ii + jj + kk).ravel()
    ks, js, is_ = kk.ravel(), jj.ravel(), ii.ravel()
    dmax = nx + ny + nz - 3
    for L in range(dmax + 2 * (nsweeps - 1) + 1):
        sel = []
        for t in range(nsweeps):
            dd = L - 2 * t
            if 0 <= dd <= dmax:
                sel.append(np.nonzero(d == dd)[0])
        if not sel:
            continue
        m = np.concatenate(sel)
        v = _update(u, f, ks[m], js[m], is_[m], b, hh)
        u[ks[m] + 1, js[m] + 1, is_[m] + 1] = v
    return u


def pass_stride(nt: int) -> int:
    return 2 if nt == 1 else 4


def skewed_tile_tasks(nx, ny, nz, tile, nt, nsweeps):
    """Tasks (I, J, K, p) of the skewed-tile schedule, sorted by level
    I + J + K + c*p.  Pass p covers sweeps [p*nt, min((p+1)*nt, nsweeps)); at the
    pass-local sweep s the tile covers x in [I*W - s, (I+1)*W - s) (same in y, z).

    c = 2 without skew (nt = 1): a task waits for its three backward face
    neighbours of the same pass and its three forward face neighbours of the
    previous pass.  With skew (nt > 1) the previous pass's tiles
    (I+a, J+b, K+c), a, b, c in {0, 1}, all end inside this task's box, the
    corner one three levels up, so passes are 4 levels apart."""
    W, H, D = tile
    ni = -(-(nx + nt - 1) // W)
    nj = -(-(ny + nt - 1) // H)
    nk = -(-(nz + nt - 1) // D)
    npass = -(-nsweeps // nt)
    tasks = [(I, J, K, p) for p in range(npass) for K in range(nk) for J in range(nj) for I in range(ni)]
    c = pass_stride(nt)
    tasks.sort(key=lambda t: (t[0] + t[1] + t[2] + c * t[3]))
    return tasks, (ni, nj, nk, npass)


def gs_skewed_tiles(u: np.ndarray, f=None, h: float = 1.0, nsweeps: int = 1, tile=(4, 4, 4),
                    nt: int = 1, reverse_within_level: bool = False) -> np.ndarray:
    """Gauss-Seidel by skewed tiles (levels I+J+K+c*p, see skewed_tile_tasks).

    A task owns, for each of its pass's sweeps s, the tile shifted by -s in x,
    y and z.  Tasks run in level order (ties in any order); inside a task the
    sites go by local level ii + jj + kk - s (ii, jj, kk the tile-local
    coordinates at sweep s), all sites of a local level together.  The global
    array is updated in place and doubles as the boundary store between tasks."""
    u = u.copy()
    nz, ny, nx = (s - 2 for s in u.shape)
    b, hh = _consts(u, h)
    if nsweeps == 0 or nx * ny * nz == 0:
        return u
    W, H, D = tile
    tasks, _ = skewed_tile_tasks(nx, ny, nz, tile, nt, nsweeps)
    if reverse_within_level:
        # same level order, reversed order among tasks of one level
        levels = {}
        for t in tasks:
            levels.setdefault(t[0] + t[1] + t[2] + pass_stride(nt) * t[3], []).append(t)
        tasks = [t for L in sorted(levels) for t in reversed(levels[L])]
    jj_, ii_ = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    jj_, ii_ = jj_.ravel(), ii_.ravel()
    for (I, J, K, p) in tasks:
        ns = min(nt, nsweeps - p * nt)
        X0, Y0, Z0 = I * W, J * H, K * D
        for lvl in range(-(ns - 1), W + H + D - 2):
            ks, js, is_ = [], [], []
            for s in range(ns):
                kk = lvl - ii_ - jj_ + s
                x = X0 - s + ii_
                y = Y0 - s + jj_
                z = Z0 - s + kk
                ok = (kk >= 0) & (kk < D) & (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz)
                ks.append(z[ok]); js.append(y[ok]); is_.append(x[ok])
            k = np.concatenate(ks); j = np.concatenate(js); i = np.concatenate(is_)
            if k.size == 0:
                continue
            v = _update(u, f, k, j, i, b, hh)
            u[k + 1, j + 1, i + 1] = v
    return u


def jacobi_wavefront_paper(u: np.ndarray, f=None, h: float = 1.0, nsweeps: int = 2, nt: int = 2) -> np.ndarray:
    """Jacobi by the Sec. 4 wavefront: one thread group of nt threads over the
    whole domain.  Thread s (1..nt) performs update s on z-plane p at step
    p + 2(s-1) (a distance of two between successive updates).  Odd updates
    write to a small temporary ring (4 planes per odd update, used round
    robin); even updates write back into ``src`` itself, so no second grid is
    needed.  nt must be even and divide nsweeps."""
    assert nt % 2 == 0 and nsweeps % nt == 0
    src = u.copy()
    nz, ny, nx = (s - 2 for s in u.shape)
    b, hh = _consts(u, h)
    R = 4
    ring = {s: np.zeros((R, ny + 2, nx + 2), dtype=u.dtype) for s in range(1, nt + 1, 2)}
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")

    def plane(level, z):
        """Padded plane z (padded index) of time level ``level`` as currently stored."""
        if z == 0 or z == nz + 1 or level % 2 == 0:
            return src[z]
        return ring[level][z % R]

    for _ in range(nsweeps // nt):
        # odd-level rings carry the Dirichlet halo of their planes
        for s in ring:
            for r in range(R):
                ring[s][r] = 0
        for n in range(nz + 2 * (nt - 1)):
            for s in range(1, nt + 1):
                p = n - 2 * (s - 1)          # interior plane index being updated
                if not (0 <= p < nz):
                    continue
                z = p + 1                     # padded index
                lo, mid, hi = plane(s - 1, z - 1), plane(s - 1, z), plane(s - 1, z + 1)
                J, I = jj + 1, ii + 1
                acc = mid[J, I - 1] + mid[J, I + 1]
                acc = acc + mid[J - 1, I]
                acc = acc + mid[J + 1, I]
                acc = acc + lo[J, I]
                acc = acc + hi[J, I]
                if f is not None:
                    acc = acc + hh * f[z, J, I]
                val = b * acc
                if s % 2 == 1:
                    dst = ring[s][z % R]
                    dst[...] = src[z]         # halo ring of the plane
                    dst[J, I] = val
                else:
                    src[z, J, I] = val
    return src


def jacobi_slab_ring(u: np.ndarray, f=None, h: float = 1.0, nsweeps: int = 1, slab: int = 2,
                     copy_first: bool = False, lag: int = 2) -> np.ndarray:
    """Jacobi in place through a ring of three z-slab buffers (the GPU's variant 6): slab s (planes
    [s*slab, (s+1)*slab)) is computed from ``src`` into buffer s % 3, and the same launch copies
    slab s - lag back from its buffer into ``src``; the last slabs still in the ring are copied back
    at the end of the sweep.  The copy-back and the computation of one launch may interleave in
    any way on the GPU; ``copy_first`` runs the copy before the computation (the other extreme), and
    both orders must give the serial result.  ``lag`` is 2 in the library."""
    src = u.copy()
    nz, ny, nx = (d - 2 for d in u.shape)
    b, hh = _consts(u, h)
    nslab = (nz + slab - 1) // slab
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    J, I = jj + 1, ii + 1
    buf = [np.zeros((slab, ny, nx), dtype=u.dtype) for _ in range(3)]

    def planes(s):
        return range(s * slab, min(nz, (s + 1) * slab))

    def compute(s):
        for q, p in enumerate(planes(s)):
            z = p + 1
            acc = src[z, J, I - 1] + src[z, J, I + 1]
            acc = acc + src[z, J - 1, I]
            acc = acc + src[z, J + 1, I]
            acc = acc + src[z - 1, J, I]
            acc = acc + src[z + 1, J, I]
            if f is not None:
                acc = acc + hh * f[z, J, I]
            buf[s % 3][q] = b * acc

    def copy_back(s):
        for q, p in enumerate(planes(s)):
            src[p + 1, J, I] = buf[s % 3][q]

    for _ in range(nsweeps):
        for s in range(nslab):
            if s >= lag and copy_first:
                copy_back(s - lag)
            compute(s)
            if s >= lag and not copy_first:
                copy_back(s - lag)
        for s in range(max(0, nslab - lag), nslab):
            copy_back(s)
    return src


def jacobi_skewed_tiles(u: np.ndarray, f=None, h: float = 1.0, nsweeps: int = 1, tile=(4, 4, 4),
                        nt: int = 1, reverse_within_level: bool = False) -> np.ndarray:
    """Jacobi by skewed tiles: the tasks and levels of skewed_tile_tasks, with two
    arrays holding alternate time levels (level v in array v % 2).  Inside a task
    the pass-local sweeps s = 0..ns-1 run one after the other, each over the
    whole shifted tile.  A tile's last column at level v+1 never overwrites the
    level-v value its forward neighbour still needs, because the skew moves
    that column out of the tile, so the two arrays alone carry every time level
    a neighbouring task reads (no boundary copies, no recomputation)."""
    nz, ny, nx = (s - 2 for s in u.shape)
    b, hh = _consts(u, h)
    arr = [u.copy(), u.copy()]  # both carry the halo; level 0 in arr[0]
    if nsweeps == 0 or nx * ny * nz == 0:
        return arr[0]
    W, H, D = tile
    tasks, _ = skewed_tile_tasks(nx, ny, nz, tile, nt, nsweeps)
    if reverse_within_level:
        levels = {}
        for t in tasks:
            levels.setdefault(t[0] + t[1] + t[2] + pass_stride(nt) * t[3], []).append(t)
        tasks = [t for L in sorted(levels) for t in reversed(levels[L])]
    kk_, jj_, ii_ = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    kk_, jj_, ii_ = kk_.ravel(), jj_.ravel(), ii_.ravel()
    for (I, J, K, p) in tasks:
        ns = min(nt, nsweeps - p * nt)
        X0, Y0, Z0 = I * W, J * H, K * D
        for s in range(ns):
            v = p * nt + s  # level read; level v+1 written
            x = X0 - s + ii_
            y = Y0 - s + jj_
            z = Z0 - s + kk_
            ok = (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz)
            k, j, i = z[ok], y[ok], x[ok]
            if k.size:
                arr[(v + 1) % 2][k + 1, j + 1, i + 1] = _update(arr[v % 2], f, k, j, i, b, hh)
    return arr[nsweeps % 2]


def dataflow_deps(I, J, K, p, nt, dims):
    """Tasks a task waits for in the dataflow form of the skewed-tile schedule:
    the three backward face neighbours of the same pass, and from the previous
    pass the task itself and its forward face neighbours (nt = 1), or the eight
    tiles (I+a, J+b, K+c), a, b, c in {0, 1} (nt > 1, whose shifted tiles end
    inside this task's box).  dims = (NI, NJ, NK)."""
    NI, NJ, NK = dims
    out = []
    for (a, b, c) in ((-1, 0, 0), (0, -1, 0), (0, 0, -1)):
        if I + a >= 0 and J + b >= 0 and K + c >= 0:
            out.append((I + a, J + b, K + c, p))
    if p > 0:
        if nt == 1:
            prev = ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))
        else:
            prev = [(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1)]
        for (a, b, c) in prev:
            if I + a < NI and J + b < NJ and K + c < NK:
                out.append((I + a, J + b, K + c, p - 1))
    return out


def random_dataflow_order(nx, ny, nz, tile, nt, nsweeps, rng):
    """A random linearisation of the dataflow dependency graph (Kahn's algorithm
    choosing uniformly among ready tasks)."""
    tasks, (NI, NJ, NK, npass) = skewed_tile_tasks(nx, ny, nz, tile, nt, nsweeps)
    deps = {t: dataflow_deps(*t, nt, (NI, NJ, NK)) for t in tasks}
    users = {t: [] for t in tasks}
    for t, ds in deps.items():
        for d in ds:
            users[d].append(t)
    missing = {t: len(ds) for t, ds in deps.items()}
    ready = [t for t in tasks if missing[t] == 0]
    order = []
    while ready:
        i = int(rng.integers(len(ready)))
        t = ready[i]
        ready[i] = ready[-1]
        ready.pop()
        order.append(t)
        for w in users[t]:
            missing[w] -= 1
            if missing[w] == 0:
                ready.append(w)
    assert len(order) == len(tasks)
    return order


def run_task_order(kind, u, f, h, nsweeps, tile, nt, order):
    """Run the tasks of the skewed-tile schedule in the given order (GS in place,
    Jacobi with two parity arrays)."""
    nz, ny, nx = (s - 2 for s in u.shape)
    b, hh = _consts(u, h)
    W, H, D = tile
    if kind == "gs":
        arr = [u.copy()]
    else:
        arr = [u.copy(), u.copy()]
    jj_, ii_ = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    jj_, ii_ = jj_.ravel(), ii_.ravel()
    kk3, jj3, ii3 = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    kk3, jj3, ii3 = kk3.ravel(), jj3.ravel(), ii3.ravel()
    for (I, J, K, p) in order:
        ns = min(nt, nsweeps - p * nt)
        X0, Y0, Z0 = I * W, J * H, K * D
        if kind == "gs":
            for lvl in range(-(ns - 1), W + H + D - 2):
                ks, js, is_ = [], [], []
                for s in range(ns):
                    kk = lvl - ii_ - jj_ + s
                    x, y, z = X0 - s + ii_, Y0 - s + jj_, Z0 - s + kk
                    ok = (kk >= 0) & (kk < D) & (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz)
                    ks.append(z[ok]); js.append(y[ok]); is_.append(x[ok])
                k = np.concatenate(ks); j = np.concatenate(js); i = np.concatenate(is_)
                if k.size:
                    arr[0][k + 1, j + 1, i + 1] = _update(arr[0], f, k, j, i, b, hh)
        else:
            for s in range(ns):
                v = p * nt + s
                x, y, z = X0 - s + ii3, Y0 - s + jj3, Z0 - s + kk3
                ok = (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz)
                k, j, i = z[ok], y[ok], x[ok]
                if k.size:
                    arr[(v + 1) % 2][k + 1, j + 1, i + 1] = _update(arr[v % 2], f, k, j, i, b, hh)
    return arr[0] if kind == "gs" else arr[nsweeps % 2]
