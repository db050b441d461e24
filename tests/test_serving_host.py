"""Host logic of the serving loop (no GPU): first-come-first-served admission
under an HBM byte budget."""
from collections import deque

import pytest

from paper_1903_01168_gb300.serving import Admission, Request, active_set
from paper_1903_01168_gb300.workloads import SimSpec, serving_trace


def _req(rid, arrival, nbytes):
    r = Request(rid, arrival, SimSpec(nx=8, ny=8))
    r.nbytes = nbytes
    return r


def test_admits_in_arrival_order_within_budget_with_backfill():
    a = Admission(100)
    q = deque([_req(0, 0.0, 40), _req(1, 0.1, 50), _req(2, 0.2, 20), _req(3, 0.3, 10), _req(4, 5.0, 1)])
    got = a.take(q, now=1.0, size_of=lambda r: r.nbytes)
    assert [r.rid for r in got] == [0, 1, 3]       # 2 would exceed 100; 3 fits and passes it
    assert a.resident == 100 and [r.rid for r in q] == [2, 4]
    assert a.take(q, now=1.0, size_of=lambda r: r.nbytes) == []
    a.release(40)                                   # request 0 retires
    got = a.take(q, now=1.0, size_of=lambda r: r.nbytes)
    assert [r.rid for r in got] == [2]              # 4 has not arrived yet
    got = a.take(q, now=6.0, size_of=lambda r: r.nbytes)
    assert [r.rid for r in got] == [4] and a.resident == 81


def test_active_set_keeps_the_oldest_and_backfills_to_the_cap():
    nodes = {0: 60, 1: 50, 2: 30, 3: 200, 4: 5}
    assert active_set([0, 1, 2], nodes.get, 100) == [0, 2]       # 1 would exceed; 2 fits after 0
    assert active_set([3, 0, 4], nodes.get, 100) == [3]          # the oldest runs alone when it exceeds the cap
    assert active_set([0, 3, 4], nodes.get, 100) == [0, 4]
    assert active_set([0, 1, 2], nodes.get, None) == [0, 1, 2]   # no cap: everything resident runs


def test_node_cap_never_blocks_an_idle_server():
    assert active_set([0], {0: 500}.get, 10) == [0]


def test_request_larger_than_budget_is_an_error():
    a = Admission(10)
    with pytest.raises(ValueError):
        a.take(deque([_req(0, 0.0, 11)]), now=0.0, size_of=lambda r: r.nbytes)


def test_release_never_goes_negative():
    a = Admission(10)
    with pytest.raises(AssertionError):
        a.release(1)


def test_serving_trace_is_seeded_and_shaped_like_the_open_channel_case():
    t1 = serving_trace(seed=5, n_requests=12)
    t2 = serving_trace(seed=5, n_requests=12)
    assert [(a, s.nx, s.ny, s.steps, s.storage) for a, s in t1] == \
           [(a, s.nx, s.ny, s.steps, s.storage) for a, s in t2]
    arrivals = [a for a, _ in t1]
    assert arrivals == sorted(arrivals)
    for _, s in t1:
        assert 512 <= s.nx <= 8192 and 64 <= s.ny <= 256 and s.nx % 32 == 0 and s.ny % 32 == 0
        assert 5000 <= s.steps <= 50000 and s.storage in (0, 1, 2)
        assert s.bc_x == 2 and s.bc_y == 1 and s.u_in_r > 0 and s.u_in_b > 0 and s.p_out > 0


def test_chunk_length_runs_to_the_next_completion():
    """Between admissions the server runs the batch to its next completion (at most
    max_chunk steps); it checks back after `chunk` steps only while the next
    request has yet to arrive (it may be admitted then), not while one that has
    arrived is held back by the budget or the node cap."""
    from types import SimpleNamespace as NS
    from paper_1903_01168_gb300.serving import Server

    srv = Server(budget_bytes=1e9, chunk=100, max_chunk=4000)

    def member(steps, t):
        return (NS(t=t), NS(spec=NS(steps=steps)), 0.0, 0)

    active = {0: member(5000, 1000), 1: member(20000, 0)}
    assert srv._chunk_len(active, deque(), now=1.0) == 4000                      # capped by max_chunk
    active = {0: member(1500, 1000), 1: member(20000, 0)}
    assert srv._chunk_len(active, deque(), now=1.0) == 500                       # next completion
    future = deque([Request(7, 5.0, SimSpec(nx=8, ny=8))])
    assert srv._chunk_len(active, future, now=1.0) == 100                        # an arrival is due
    arrived = deque([Request(7, 0.5, SimSpec(nx=8, ny=8))])
    assert srv._chunk_len(active, arrived, now=1.0) == 500                       # held back: run on
