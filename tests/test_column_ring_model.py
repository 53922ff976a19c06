"""The column march's shared-memory ring schedule (gs_column.cu), checked step by step on the CPU:
every update and write-back reads what it needs and no read meets a copy still in flight, for the
tile shapes the kernel instantiates and others, copy-ahead distances 1..3, chunks of 1..40 planes;
and the ring depth tx + pf + 4 is the smallest that works."""
import pytest

from tests._column_ring import check_column_ring, ring_slots


@pytest.mark.parametrize("tile", [(8, 8), (8, 16), (16, 8), (2, 2), (3, 5), (5, 2)])
@pytest.mark.parametrize("nzl", [1, 2, 3, 7, 40])
@pytest.mark.parametrize("pf", [1, 2, 3])
def test_ring_schedule_is_hazard_free(tile, nzl, pf):
    tx, ty = tile
    assert check_column_ring(tx, ty, nzl, pf) is None


@pytest.mark.parametrize("tile", [(8, 8), (16, 8), (3, 5)])
@pytest.mark.parametrize("pf", [1, 2])
def test_one_slot_fewer_breaks_it(tile, pf):
    tx, ty = tile
    err = check_column_ring(tx, ty, 40, pf, r=ring_slots(tx, pf) - 1)
    assert err is not None
