"""GPU tests of the continuous-batching server: each result equals the oracle's
and is the same alone and in a mix; admission by budget, cancellation."""
import time

import numpy as np
import pytest

import oracle
from paper_1004_1741_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1004_1741_gb300 import capi  # noqa: E402


def _req(kind, dims, seed, dtype=np.float64, poisson=True, sweeps=7):
    u, f = W.random_grid(*dims, seed=seed, dtype=dtype, with_f=poisson)
    return {"kind": kind, "u": u, "f": f, "h": W.grid_h(*dims), "nsweeps": sweeps}


def _oracle(r):
    fn = oracle.jacobi if r["kind"] == capi.STENCIL_REQ_JACOBI else oracle.gs_lex
    return fn(r["u"], r["f"], r["h"], r["nsweeps"])


def test_results_same_alone_and_in_mix():
    reqs = [_req(capi.STENCIL_REQ_JACOBI, (40, 33, 21), 1), _req(capi.STENCIL_REQ_GS, (17, 50, 9), 2, sweeps=13),
            _req(capi.STENCIL_REQ_GS, (64, 64, 64), 3, dtype=np.float32, sweeps=25),
            _req(capi.STENCIL_REQ_JACOBI, (9, 9, 70), 4, dtype=np.float32, poisson=False, sweeps=31),
            _req(capi.STENCIL_REQ_GS, (100, 30, 40), 5, poisson=False, sweeps=4)]
    alone = []
    with capi.Server(0, sweeps_per_round=5) as srv:
        for r in reqs:  # one at a time
            out = np.empty_like(r["u"])
            t = srv.submit(r["kind"], r["u"], r["f"], r["h"], r["nsweeps"], u_out=out)
            res = srv.wait(t, 60)
            assert res is not None and res["status"] == capi.STENCIL_OK and res["sweeps_done"] == r["nsweeps"]
            alone.append(out)
        outs, tickets = [], []
        for r in reqs * 2:  # all at once, twice over, so rounds mix classes and sizes
            out = np.empty_like(r["u"])
            tickets.append(srv.submit(r["kind"], r["u"], r["f"], r["h"], r["nsweeps"], u_out=out))
            outs.append(out)
        for t in tickets:
            assert srv.wait(t, 60)["status"] == capi.STENCIL_OK
        st = srv.stats()
        assert st["completed"] == 3 * len(reqs) and st["p99_s"] >= st["p50_s"] > 0 and st["hbm_in_use"] == 0
    for i, r in enumerate(reqs):
        ref = _oracle(r)
        assert np.array_equal(alone[i], ref)
        assert np.array_equal(outs[i], ref) and np.array_equal(outs[i + len(reqs)], ref)


def test_solve_request_converges_and_caps():
    p = W.sine_modes_problem(16, seed=4, noise_sigma=0.0)
    u0 = np.zeros_like(p.f)
    with capi.Server(0, sweeps_per_round=20) as srv:
        out = np.empty_like(u0)
        res = srv.wait(srv.submit(capi.STENCIL_REQ_SOLVE, u0, p.f, p.h, 5000, rtol=1e-8, u_out=out), 120)
        assert res["status"] == capi.STENCIL_OK and res["rel_residual"] <= 1e-8
        assert res["sweeps_done"] % 20 == 0
        # the same solve capped early: not converged, residual reported, grid = that many GS sweeps
        out2 = np.empty_like(u0)
        res2 = srv.wait(srv.submit(capi.STENCIL_REQ_SOLVE, u0, p.f, p.h, 3, rtol=1e-8, u_out=out2), 60)
        assert res2["status"] == capi.STENCIL_ERR_NOT_CONVERGED and res2["rel_residual"] > 1e-8
        assert res2["sweeps_done"] == 3
        assert np.array_equal(out2, oracle.gs_lex(u0, p.f, p.h, 3))


def test_budget_admission_cancel_and_oom():
    big = _req(capi.STENCIL_REQ_GS, (160, 160, 160), 7, poisson=False, sweeps=20000)
    small = _req(capi.STENCIL_REQ_JACOBI, (20, 20, 20), 8)
    nbytes = big["u"].nbytes
    with capi.Server(0, hbm_budget_bytes=int(nbytes * 1.5), sweeps_per_round=10) as srv:
        t_big = srv.submit(big["kind"], big["u"], None, big["h"], big["nsweeps"])
        time.sleep(0.2)
        t_wait = srv.submit(big["kind"], big["u"], None, big["h"], 1)  # does not fit while the first runs
        assert srv.cancel(t_wait)
        res = srv.wait(t_wait, 10)
        assert res["status"] == capi.STENCIL_ERR_CANCELLED
        huge = W.random_grid(200, 200, 200, seed=9)[0]  # larger than the whole budget
        res_h = srv.wait(srv.submit(capi.STENCIL_REQ_GS, huge, None, 0.1, 1), 30)
        assert res_h["status"] == capi.STENCIL_ERR_OOM
        out = np.empty_like(small["u"])
        res_s = srv.wait(srv.submit(small["kind"], small["u"], small["f"], small["h"], small["nsweeps"], u_out=out), 60)
        assert res_s["status"] == capi.STENCIL_OK and np.array_equal(out, _oracle(small))
        assert srv.wait(t_big, 300)["status"] == capi.STENCIL_OK
        assert srv.stats()["hbm_peak"] <= int(nbytes * 1.5)


def test_slot_limit_keeps_results_exact():
    reqs = [_req(capi.STENCIL_REQ_GS if i % 2 else capi.STENCIL_REQ_JACOBI, (24 + 8 * i, 20, 16), 20 + i,
                 sweeps=9 + i) for i in range(6)]
    with capi.Server(0, sweeps_per_round=4, max_active=2) as srv:
        outs = [np.empty_like(r["u"]) for r in reqs]
        ts = [srv.submit(r["kind"], r["u"], r["f"], r["h"], r["nsweeps"], u_out=o) for r, o in zip(reqs, outs)]
        for t in ts:
            assert srv.wait(t, 60)["status"] == capi.STENCIL_OK
    for r, o in zip(reqs, outs):
        assert np.array_equal(o, _oracle(r))


def test_solve_request_runs_multigrid_cycles():
    """A solve request on odd extents runs multigrid V(2,2) cycles with the red-black smoother (up to
    sweeps_per_round / 4 per round, residual after each):
    the result equals the oracle's multigrid solve with the same stopping test, bit for bit, four sweeps
    counted per cycle; the same request capped before convergence reports its residual."""
    p = W.sine_modes_problem(31, seed=4)
    u0 = np.zeros_like(p.f)
    with capi.Server(0, sweeps_per_round=10) as srv:
        out = np.empty_like(u0)
        res = srv.wait(srv.submit(capi.STENCIL_REQ_SOLVE, u0, p.f, p.h, 400, rtol=1e-8, u_out=out), 120)
        assert res["status"] == capi.STENCIL_OK and res["rel_residual"] <= 1e-8
        cycles = res["sweeps_done"] // 4
        assert res["sweeps_done"] == 4 * cycles and 3 <= cycles <= 15
        ref, rel, rc, ok = oracle.mg_solve(u0, p.f, p.h, oracle.MG_GS_RB, 2, 2, 10, 32, 1e-8, cycles)
        assert ok and rc == cycles
        assert np.array_equal(out, ref)
        out2 = np.empty_like(u0)
        res2 = srv.wait(srv.submit(capi.STENCIL_REQ_SOLVE, u0, p.f, p.h, 9, rtol=1e-8, u_out=out2), 60)
        assert res2["status"] == capi.STENCIL_ERR_NOT_CONVERGED and res2["sweeps_done"] == 8
        ref2, _, _, _ = oracle.mg_solve(u0, p.f, p.h, oracle.MG_GS_RB, 2, 2, 10, 32, 1e-8, 2)
        assert np.array_equal(out2, ref2)


def test_mixed_solve_request_runs_fp32_cycles_in_defect_correction():
    """A mixed-precision solve request on odd extents runs FP32 multigrid V(2,2) cycles inside FP64 defect
    correction (up to sweeps_per_round / 4 outer iterations per round, the FP64 residual after each): the
    result equals the oracle's mixed solve with the same stopping test, bit for bit, four sweeps counted per
    outer iteration; capped before convergence it reports its residual; on even extents it falls back to the
    plain solve's lexicographic sweeps."""
    p = W.sine_modes_problem(31, seed=4)
    u0 = np.zeros_like(p.f)
    with capi.Server(0, sweeps_per_round=10) as srv:
        out = np.empty_like(u0)
        res = srv.wait(srv.submit(capi.STENCIL_REQ_SOLVE_MIXED, u0, p.f, p.h, 400, rtol=1e-8, u_out=out), 120)
        assert res["status"] == capi.STENCIL_OK and res["rel_residual"] <= 1e-8
        its = res["sweeps_done"] // 4
        assert res["sweeps_done"] == 4 * its and 3 <= its <= 15
        ref, rel, n, ok = oracle.solve_mixed_mg(u0, p.f, p.h, oracle.MG_GS_RB, 2, 2, 10, 32, 1e-8, its, 1)
        assert ok and n == its
        assert np.array_equal(out, ref)
        out2 = np.empty_like(u0)
        res2 = srv.wait(srv.submit(capi.STENCIL_REQ_SOLVE_MIXED, u0, p.f, p.h, 9, rtol=1e-8, u_out=out2), 60)
        assert res2["status"] == capi.STENCIL_ERR_NOT_CONVERGED and res2["sweeps_done"] == 8
        ref2, _, _, _ = oracle.solve_mixed_mg(u0, p.f, p.h, oracle.MG_GS_RB, 2, 2, 10, 32, 1e-8, 2, 1)
        assert np.array_equal(out2, ref2)
        # even extents: the same lexicographic sweeps as the plain solve request
        q = W.random_grid(12, 10, 8, seed=9, with_f=True)
        out3, out4 = np.empty_like(q[0]), np.empty_like(q[0])
        r3 = srv.wait(srv.submit(capi.STENCIL_REQ_SOLVE_MIXED, q[0], q[1], 0.1, 25, rtol=1e-12, u_out=out3), 60)
        r4 = srv.wait(srv.submit(capi.STENCIL_REQ_SOLVE, q[0], q[1], 0.1, 25, rtol=1e-12, u_out=out4), 60)
        assert r3["status"] == r4["status"] and r3["sweeps_done"] == r4["sweeps_done"]
        assert np.array_equal(out3, out4)


def test_many_requests_overlap_copies_and_rounds():
    """Forty requests of mixed kinds submitted at once through a four-slot server: copies and rounds
    interleave (admission keeps at most four on the device), every result equals the oracle, and the pool
    returns all memory."""
    reqs = []
    for i in range(40):
        kind = (capi.STENCIL_REQ_JACOBI, capi.STENCIL_REQ_GS)[i % 2]
        reqs.append(_req(kind, (20 + i % 7, 18, 11 + i % 5), 100 + i, dtype=(np.float64, np.float32)[i % 3 == 0],
                         sweeps=3 + i % 6))
    with capi.Server(0, sweeps_per_round=4, max_active=4) as srv:
        outs = [np.empty_like(r["u"]) for r in reqs]
        ts = [srv.submit(r["kind"], r["u"], r["f"], r["h"], r["nsweeps"], u_out=o) for r, o in zip(reqs, outs)]
        for t in ts:
            assert srv.wait(t, 120)["status"] == capi.STENCIL_OK
        st = srv.stats()
        assert st["hbm_in_use"] == 0 and st["completed"] == 40 and st["active"] == 0
    for r, o in zip(reqs, outs):
        assert np.array_equal(o, _oracle(r))
