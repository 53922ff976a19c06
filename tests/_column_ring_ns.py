"""A value-level CPU model of the multi-sweep column march (gs_column.cu, NS sweeps per task).

Task (I, J, K, p) of the skewed-tile schedule (tiles.h, nt = NS) applies the ns sweeps of pass p
to tile (I, J, K); sweep s covers the tile's box shifted by -s in x, y and z.  Inside the task the
tile lives in a shared-memory ring of R plane slots; each slot holds rows -NS..TY and columns
-NS..TX of one plane (tile-local coordinates), cell (i, j, k) in slot (i + j + k) mod R.  Thread
(i, j), i < TX, j < TY, at step t updates, for every sweep s < ns, the site (i - s, j - s, k) with
k = t - i - j -- sweep s trails sweep s - 1 by two steps, the paper's "distance of two" between
successive time levels (Sec. 4) -- reading slots t - 2s - 1 (W, S, B: this sweep's values) and
t - 2s + 1 (E, N, T: the previous sweep's), writing slot t - 2s.

Row line (j, k) (columns -NS..TX) is copied into the ring at step j + k - 2 - PF and lands by the
end of step j + k - 2 (cp.async.wait_group PF before the step's barrier); the cells of row (j, k)
that this task updates are written back at step j + k + TX + NS - 1, after their last update.  A
right-hand side f travels in a second ring with the same slots (rows and columns -NS+1..TY-1 /
TX-1, the cells some sweep updates).

The model runs whole grids task by task (level order or any order that respects the dependency
flags of the persistent launch) with the real site arithmetic (numpy scalars: IEEE binary64 or
binary32), and reports the first hazard: a read of a ring cell whose copy may still be in flight
or that holds the wrong site, an update into a cell a copy may still overwrite, or a ring slot
refilled before its previous row was written back.  The final grid must equal the serial sweeps
bit for bit.
"""
from __future__ import annotations

import numpy as np


def ring_slots_ns(tx: int, ns: int, pf: int) -> int:
    """Ring depth of the multi-sweep column march: a row line lives from its copy (PF + 1 steps
    before its first reader) to its write-back (TX + NS + 1 steps after that reader)."""
    return tx + ns + pf + 2


def _tile_count(n: int, w: int, nt: int) -> int:
    return -(-(n + nt - 1) // w)


def tasks_in_level_order(nx, ny, nz, tx, ty, d, nt, nsweeps):
    NI, NJ, NK = _tile_count(nx, tx, nt), _tile_count(ny, ty, nt), _tile_count(nz, d, nt)
    npass = -(-nsweeps // nt)
    c = 2 if nt == 1 else 4
    tasks = [(I + J + K + c * p, p, K, J, I) for p in range(npass) for K in range(NK) for J in range(NJ)
             for I in range(NI)]
    tasks.sort()
    return [(I, J, K, p) for (_, p, K, J, I) in tasks], (NI, NJ, NK, npass)


def run_task(u, f, hh, b, I, J, K, p, tx, ty, d, NS, nsweeps, pf, R=None):
    """One task of the model on padded grid u (in place).  Returns None or a hazard description."""
    nz, ny, nx = (s - 2 for s in u.shape)
    R = ring_slots_ns(tx, NS, pf) if R is None else R
    nse = min(NS, nsweeps - p * NS)
    x0, y0, z0 = I * tx, J * ty, K * d
    ring = {}   # (slot, j, i) -> (site, value)
    pending = {}  # (slot, j, i) -> landing step
    fring = {}
    fpend = {}
    inflight = []  # (land step, key, content, which ring)
    live = {}  # slot-cell -> row (j, k) that owns it until written back
    ts = -2 * NS - 2 - pf
    te = tx + ty + d + NS - 3
    updated = set()

    def g(x, y, z):
        return (z + 1, y + 1, x + 1)

    def in_pad(x, y, z):
        return -1 <= x <= nx and -1 <= y <= ny and -1 <= z <= nz

    def interior(x, y, z):
        return 0 <= x < nx and 0 <= y < ny and 0 <= z < nz

    def updated_by_task(i, j, k):
        a = max(0, -i, -j, -k)
        bb = min(nse - 1, tx - 1 - i, ty - 1 - j, d - 1 - k)
        return a <= bb

    for t in range(ts, te + 1):
        # 1. copies of the row lines whose copy step is t
        for j in range(-NS, ty + 1):
            k = t + 2 + pf - j
            if not (-NS <= k <= d):
                continue
            for i in range(-NS, tx + 1):
                x, y, z = x0 + i, y0 + j, z0 + k
                if not in_pad(x, y, z):
                    continue
                key = ((i + j + k) % R, j, i)
                if key in live and live[key] != (j, k):
                    return "step %d: copy of row %s into a cell still owned by row %s" % (t, (j, k), live[key])
                live[key] = (j, k)
                inflight.append((t + pf, key, ((i, j, k), u[g(x, y, z)]), "u"))
                pending[key] = t + pf
                if f is not None and -NS + 1 <= i <= tx - 1 and -NS + 1 <= j <= ty - 1 and -NS + 1 <= k <= d - 1 \
                        and interior(x, y, z):
                    inflight.append((t + pf, key, ((i, j, k), f[g(x, y, z)]), "f"))
                    fpend[key] = t + pf
        # 2. updates: thread (i, j), sweep s -> site (i - s, j - s, t - i - j)
        writes = {}
        read_keys = set()
        for jt in range(ty):
            for it in range(tx):
                k = t - it - jt
                for s in range(nse):
                    a, bb = it - s, jt - s
                    if not (-s <= k <= d - 1 - s):
                        continue
                    x, y, z = x0 + a, y0 + bb, z0 + k
                    if not interior(x, y, z):
                        continue
                    vals = []
                    for (da, db, dk) in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
                        na, nb, nk = a + da, bb + db, k + dk
                        key = ((na + nb + nk) % R, nb, na)
                        if key in pending:
                            return "step %d: sweep %d at %s reads %s while its copy may be in flight" % (
                                t, s, (a, bb, k), (na, nb, nk))
                        read_keys.add(key)
                        got = ring.get(key)
                        if got is None or got[0] != (na, nb, nk):
                            return "step %d: sweep %d at %s finds %s for %s" % (t, s, (a, bb, k), got, (na, nb, nk))
                        vals.append(got[1])
                    acc = vals[0] + vals[1]
                    for v in vals[2:]:
                        acc = acc + v
                    if f is not None:
                        fk = ((a + bb + k) % R, bb, a)
                        if fk in fpend:
                            return "step %d: f of %s read while in flight" % (t, (a, bb, k))
                        fv = fring.get(fk)
                        if fv is None or fv[0] != (a, bb, k):
                            return "step %d: f ring holds %s for %s" % (t, fv, (a, bb, k))
                        acc = acc + hh * fv[1]
                    key = ((a + bb + k) % R, bb, a)
                    if key in pending:
                        return "step %d: update into a cell a copy may still overwrite" % t
                    writes[key] = ((a, bb, k), b * acc)
                    updated.add((a, bb, k, s))
        if read_keys & set(writes):
            return "step %d: a cell is read and written in the same step" % t
        ring.update(writes)
        # 3. write-backs of the rows whose write-back step is t
        for j in range(-NS + 1, ty):
            k = t - (tx + NS - 1) - j
            if not (-NS + 1 <= k <= d - 1):
                continue
            for i in range(-NS + 1, tx):
                x, y, z = x0 + i, y0 + j, z0 + k
                key = ((i + j + k) % R, j, i)
                if interior(x, y, z) and updated_by_task(i, j, k):
                    got = ring.get(key)
                    if key in pending or got is None or got[0] != (i, j, k):
                        return "step %d: write-back of %s finds %s" % (t, (i, j, k), got)
                    u[g(x, y, z)] = got[1]
        # every cell of the rows whose write-back step is t is free for the next copy from step t + 1
        for j in range(-NS, ty + 1):
            k = t - (tx + NS - 1) - j
            for i in range(-NS, tx + 1):
                key = ((i + j + k) % R, j, i)
                if live.get(key) == (j, k):
                    del live[key]
        # 4. end of step: copies issued PF steps ago have landed
        keep = []
        for land, key, content, which in inflight:
            if land <= t:
                if which == "u":
                    ring[key] = content
                    pending.pop(key, None)
                else:
                    fring[key] = content
                    fpend.pop(key, None)
            else:
                keep.append((land, key, content, which))
        inflight = keep
    # every site of every sweep of the task's boxes was updated
    for s in range(nse):
        for k in range(-s, d - s):
            for j in range(-s, ty - s):
                for i in range(-s, tx - s):
                    if interior(x0 + i, y0 + j, z0 + k) and (i, j, k, s) not in updated:
                        return "site %s of sweep %d not updated" % ((i, j, k), s)
    return None


def gs_column_ns(u, f, h, nsweeps, tx, ty, d, NS, pf, order=None, R=None):
    """Gauss-Seidel through the model: returns (grid, hazard or None)."""
    u = u.copy()
    dt = u.dtype.type
    b = dt(1.0 / 6.0)
    hh = dt(h * h)
    nz, ny, nx = (s - 2 for s in u.shape)
    if nsweeps == 0 or nx * ny * nz == 0:
        return u, None
    tasks, _ = tasks_in_level_order(nx, ny, nz, tx, ty, d, NS, nsweeps)
    if order is not None:
        tasks = order
    for (I, J, K, p) in tasks:
        err = run_task(u, f, hh, b, I, J, K, p, tx, ty, d, NS, nsweeps, pf, R)
        if err:
            return u, "task %s: %s" % ((I, J, K, p), err)
    return u, None


def random_dependency_order(nx, ny, nz, tx, ty, d, nt, nsweeps, seed):
    """A random order of the tasks that respects the persistent launch's dependency flags:
    the three backward faces of the same pass and the 2x2x2 tiles ahead of the previous pass."""
    tasks, (NI, NJ, NK, npass) = tasks_in_level_order(nx, ny, nz, tx, ty, d, nt, nsweeps)
    rng = np.random.default_rng(seed)
    done = set()
    left = list(tasks)
    out = []

    def ready(I, J, K, p):
        deps = []
        if I > 0:
            deps.append((I - 1, J, K, p))
        if J > 0:
            deps.append((I, J - 1, K, p))
        if K > 0:
            deps.append((I, J, K - 1, p))
        if p > 0:
            for c in range(2):
                for bb in range(2):
                    for a in range(2):
                        if I + a < NI and J + bb < NJ and K + c < NK:
                            deps.append((I + a, J + bb, K + c, p - 1))
        return all(x in done for x in deps)

    while left:
        cand = [x for x in left if ready(*x)]
        pick = cand[int(rng.integers(len(cand)))]
        out.append(pick)
        done.add(pick)
        left.remove(pick)
    return out
