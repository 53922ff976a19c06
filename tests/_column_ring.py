"""A step-by-step model of the column march's shared-memory ring (the schedule of
gs_column.cu's task body), checked on the CPU.

One task: tile columns i in [0, TX), rows j in [0, TY), local planes k in [0, nzl),
neighbour columns/rows/planes at -1 and TX / TY / nzl.  Cell (i, j, k) lives in ring slot
(k + i + j) mod R at row j + 1, column i + 1.  Thread (i, j) at step t:

  * copies its own row's cell of plane t - j + 2 + PF (into slot t + 2 + PF + i), the W / E
    neighbour column of that plane when it is the first / last lane, the S row of plane
    t + 3 + PF (row 0) or the N row of plane t - TY + 2 + PF (last row), each while its plane
    is in range;
  * updates plane t - i - j (reads slots t - 1 and t + 1, writes slot t);
  * writes back plane t - TX - j - 1 (from slot t - TX - 1 + i);
  * then every copy issued PF or more steps ago has landed (cp.async.wait_group PF) and
    the CTA synchronises.

A copy issued at step s may land at any moment until the end of step s + PF.  The model
tracks what every ring cell holds (which site, before or after this sweep's update) and
reports the first read that could see anything other than what the update or the
write-back needs: a cell whose copy may still be in flight, a stale or overwritten value, a
cell read and written in the same step, a site not updated or not written back exactly once.
Halo values below / west / south of the tile come from tasks of lower levels (already
swept), those above / east / north from higher levels (not yet swept).
"""
from __future__ import annotations


def ring_slots(tx: int, pf: int) -> int:
    """Ring depth of the kernel: a row line lives from its copy to its write-back."""
    return tx + pf + 4


def check_column_ring(tx: int, ty: int, nzl: int, pf: int, r: int | None = None) -> str | None:
    """None when the schedule is hazard-free for this tile, else a description of the first hazard."""
    R = ring_slots(tx, pf) if r is None else r
    cells: dict[tuple, tuple] = {}  # (slot, row, col) -> (site, version)
    inflight: list[tuple] = []  # (issue step, cell, content)

    def slot_of(i, j, k):
        return (k + i + j) % R

    def cell_of(i, j, k):
        return (slot_of(i, j, k), j + 1, i + 1)

    def halo_version(i, j, k):
        # lower levels (W, S, below) are swept before this task, higher levels (E, N, above) after
        if i < 0 or j < 0 or k < 0:
            return "new"
        return "old"

    def global_content(i, j, k):
        inside = 0 <= i < tx and 0 <= j < ty and 0 <= k < nzl
        return ((i, j, k), "old" if inside else halo_version(i, j, k))

    updated = {}
    written = {}
    ts = -3 - pf
    te = nzl + tx + ty - 1
    for t in range(ts, te + 1):
        reads = []  # (cell, expected content, what)
        writes = []  # (cell, content)
        # 1. copies issued this step
        for j in range(ty):
            for i in range(tx):
                ql = t - j + 2 + pf
                if -1 <= ql <= nzl:
                    inflight.append((t, cell_of(i, j, ql), global_content(i, j, ql)))
                    if i == 0:
                        inflight.append((t, cell_of(-1, j, ql), global_content(-1, j, ql)))
                    if i == tx - 1:
                        inflight.append((t, cell_of(tx, j, ql), global_content(tx, j, ql)))
                if j == 0:
                    q = t + 3 + pf
                    if 0 <= q < nzl:
                        inflight.append((t, cell_of(i, -1, q), global_content(i, -1, q)))
                if j == ty - 1:
                    q = t - ty + 2 + pf
                    if 0 <= q < nzl:
                        inflight.append((t, cell_of(i, ty, q), global_content(i, ty, q)))
        # 2. updates and write-backs of this step
        for j in range(ty):
            for i in range(tx):
                kk = t - i - j
                if 0 <= kk < nzl:
                    def nb(a, b, c):
                        inside = 0 <= a < tx and 0 <= b < ty and 0 <= c < nzl
                        return ((a, b, c), halo_version(a, b, c) if not inside else None)
                    for (a, b, c), lower in (((i - 1, j, kk), True), ((i, j - 1, kk), True), ((i, j, kk - 1), True),
                                             ((i + 1, j, kk), False), ((i, j + 1, kk), False), ((i, j, kk + 1), False)):
                        site, hv = nb(a, b, c)
                        want = hv if hv is not None else ("new" if lower else "old")
                        reads.append((cell_of(a, b, c), (site, want), "update of %s reads %s" % ((i, j, kk), site)))
                    writes.append((cell_of(i, j, kk), ((i, j, kk), "new")))
                    if (i, j, kk) in updated:
                        return "site %s updated twice" % ((i, j, kk),)
                    updated[(i, j, kk)] = t
                qw = t - tx - j - 1
                if 0 <= qw < nzl:
                    reads.append((cell_of(i, j, qw), ((i, j, qw), "new"), "write-back of %s" % ((i, j, qw),)))
                    if (i, j, qw) in written:
                        return "site %s written back twice" % ((i, j, qw),)
                    written[(i, j, qw)] = t
        pending = {c for (s, c, _) in inflight if s >= t - pf}
        written_cells = {c for c, _ in writes}
        for c, want, what in reads:
            if c in pending:
                return "step %d: %s while a copy into that cell may be in flight" % (t, what)
            if c in written_cells:
                return "step %d: %s from a cell written in the same step" % (t, what)
            got = cells.get(c)
            if got != want:
                return "step %d: %s finds %s, needs %s" % (t, what, got, want)
        for c, content in writes:
            if c in pending:
                return "step %d: update into a cell a copy may still overwrite" % t
            cells[c] = content
        # 3. end of step: copies issued pf steps ago (and earlier) have landed
        keep = []
        for s, c, content in inflight:
            if s <= t - pf:
                cells[c] = content
            else:
                keep.append((s, c, content))
        inflight = keep
    n = tx * ty * nzl
    if len(updated) != n:
        return "%d of %d sites updated" % (len(updated), n)
    if len(written) != n:
        return "%d of %d sites written back" % (len(written), n)
    return None
