"""The multi-sweep column march (gs_column.cu, NS sweeps per task, the temporal blocking of Sec. 4
inside a tile), checked on the CPU through a value-level model of its ring schedule
(tests/_column_ring_ns.py): whole grids, task by task, in level order and in random orders that
respect the persistent launch's dependency flags, equal the serial Gauss-Seidel sweeps of the
oracle bit for bit with no hazard; the ring depth tx + NS + PF + 2 is the smallest that works."""
import numpy as np
import pytest

import oracle
from paper_1004_1741_gb300 import workloads as W
from tests._column_ring_ns import gs_column_ns, random_dependency_order, ring_slots_ns


@pytest.mark.parametrize("dims", [(13, 11, 9), (17, 5, 7), (1, 1, 1), (3, 20, 5)])
@pytest.mark.parametrize("tile", [(8, 8, 8), (4, 4, 4), (3, 5, 4)])
@pytest.mark.parametrize("ns", [1, 2, 3, 4])
def test_multi_sweep_march_equals_serial_sweeps(dims, tile, ns):
    tx, ty, d = tile
    if ns > min(tile):
        pytest.skip("the skewed tiles need nt <= every tile extent")
    nx, ny, nz = dims
    u0, f0 = W.random_grid(nx, ny, nz, seed=nx + ny + ns, with_f=True)
    for f, nsweeps, pf in ((None, ns, 2), (f0, 2 * ns + 1, 1)):
        got, err = gs_column_ns(u0, f, 0.1, nsweeps, tx, ty, d, ns, pf)
        assert err is None, err
        np.testing.assert_array_equal(got, oracle.gs_lex(u0, f, 0.1, nsweeps))


@pytest.mark.parametrize("dims,tile,ns", [((13, 11, 9), (4, 4, 4), 2), ((17, 9, 10), (3, 5, 4), 3),
                                          ((9, 9, 9), (4, 4, 4), 4)])
def test_multi_sweep_march_in_dependency_orders(dims, tile, ns):
    nx, ny, nz = dims
    tx, ty, d = tile
    u0, f0 = W.random_grid(nx, ny, nz, seed=5, with_f=True)
    ref = oracle.gs_lex(u0, f0, 0.1, 2 * ns + 1)
    for seed in range(3):
        order = random_dependency_order(nx, ny, nz, tx, ty, d, ns, 2 * ns + 1, seed)
        got, err = gs_column_ns(u0, f0, 0.1, 2 * ns + 1, tx, ty, d, ns, 2, order=order)
        assert err is None, err
        np.testing.assert_array_equal(got, ref)


def test_multi_sweep_march_float32():
    u0, f0 = W.random_grid(11, 10, 9, seed=2, dtype=np.float32, with_f=True)
    got, err = gs_column_ns(u0, f0, 0.1, 5, 4, 4, 4, 2, 2)
    assert err is None
    np.testing.assert_array_equal(got, oracle.gs_lex(u0, f0, 0.1, 5))


@pytest.mark.parametrize("tile,ns,pf", [((8, 8, 30), 2, 2), ((8, 8, 30), 1, 2), ((8, 8, 30), 3, 1),
                                        ((16, 8, 30), 2, 2)])
def test_one_slot_fewer_breaks_the_multi_sweep_ring(tile, ns, pf):
    tx, ty, d = tile
    u0, _ = W.random_grid(tx + 3, ty + 3, d + 5, seed=1)
    r = ring_slots_ns(tx, ns, pf)
    _, err = gs_column_ns(u0, None, 0.1, ns, tx, ty, d, ns, pf, R=r - 1)
    assert err is not None
    got, err = gs_column_ns(u0, None, 0.1, ns, tx, ty, d, ns, pf, R=r)
    assert err is None
    np.testing.assert_array_equal(got, oracle.gs_lex(u0, None, 0.1, ns))
