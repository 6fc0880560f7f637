"""Host logic of the sweep server (no GPU): the ring of query rows that
admits waves by memory.  A wave takes contiguous rows, never rows another
wave holds, and rows come back in admission order; a request that does not
fit waits.  Checked against a plain occupancy model over random sequences."""
import collections

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_1707_00516_gb300.serve import SweepServer  # noqa: E402


def _ring(capacity):
    """The server's ring bookkeeping alone (its device buffers are not needed)."""
    r = object.__new__(SweepServer)
    r.capacity = capacity
    r._alloc = collections.deque()
    r._head = r._tail = 0
    return r


def _used(held, capacity):
    """Rows the waves in the model hold."""
    used = np.zeros(capacity, bool)
    for off, n in held:
        used[off:off + n] = True
    return used


@pytest.mark.parametrize("capacity", [7, 64, 100, 1024])
def test_ring_rows_are_contiguous_disjoint_and_released_in_order(capacity):
    rng = np.random.default_rng(capacity)
    ring = _ring(capacity)
    held = collections.deque()  # (off, n) in admission order, the model
    admitted = refused = 0
    for _ in range(4000):
        if held and rng.random() < 0.45:
            ring._ring_release()
            held.popleft()
            continue
        n = int(rng.integers(1, capacity + 1))
        used = _used(held, capacity)
        off = ring._ring_alloc(n)
        if off is None:
            refused += 1
            # refused only when no placement the ring may use is free: after the
            # newest wave's rows, or (wrapping) from row 0 up to the oldest's
            assert held, "an empty ring refused a wave that fits"
            head, tail = held[0][0], held[-1][0] + held[-1][1]
            if tail > head:  # free: [tail, capacity) and [0, head)
                assert not (tail + n <= capacity and not used[tail:tail + n].any())
                assert not (n <= head and not used[:n].any())
            else:  # wrapped (or exactly full): free [tail, head)
                assert tail + n > head
            continue
        admitted += 1
        assert 0 <= off and off + n <= capacity  # contiguous and in range
        assert not used[off:off + n].any()  # no row another wave holds
        held.append((off, n))
        assert list(ring._alloc) == list(held)  # released in admission order
    assert admitted > 100 and refused > 10


def test_ring_empty_restarts_at_row_zero():
    ring = _ring(10)
    assert ring._ring_alloc(6) == 0
    assert ring._ring_alloc(5) is None  # 4 rows left at the end, 0 free at the start
    assert ring._ring_alloc(4) == 6
    ring._ring_release()  # rows 0-5 free again
    assert ring._ring_alloc(5) == 0  # wraps to the start
    ring._ring_release()
    ring._ring_release()
    assert not ring._alloc
    assert ring._ring_alloc(10) == 0  # an empty ring offers all its rows
