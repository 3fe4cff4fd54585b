"""Host-side logic of bench.py that needs no GPU: the bounded wait on
serving tickets must return once every ticket is done and give up, with an
error, when one never completes."""
import time

import pytest

import bench


def test_wait_tickets_returns_when_all_done():
    done_at = {t: time.perf_counter() + 0.01 * t for t in range(5)}
    bench.wait_tickets(lambda t: time.perf_counter() >= done_at[t], list(range(5)), limit_s=5.0)


def test_wait_tickets_gives_up_on_a_lost_query():
    t0 = time.perf_counter()
    with pytest.raises(bench.ServingStuck, match="1 of 3 queries unfinished"):
        bench.wait_tickets(lambda t: t != 2, [0, 1, 2], limit_s=0.2)
    assert time.perf_counter() - t0 < 5.0


def test_wait_tickets_empty():
    bench.wait_tickets(lambda t: False, [], limit_s=0.0)
