"""Host logic of the serving loop (no GPU): first-come-first-served admission
under an HBM byte budget."""
from collections import deque

import pytest

from paper_1903_01168_gb300.serving import Admission, Request
from paper_1903_01168_gb300.workloads import SimSpec, serving_trace


def _req(rid, arrival, nbytes):
    r = Request(rid, arrival, SimSpec(nx=8, ny=8))
    r.nbytes = nbytes
    return r


def test_admits_in_arrival_order_within_budget():
    a = Admission(100)
    q = deque([_req(0, 0.0, 40), _req(1, 0.1, 50), _req(2, 0.2, 20), _req(3, 5.0, 1)])
    got = a.take(q, now=1.0, size_of=lambda r: r.nbytes)
    assert [r.rid for r in got] == [0, 1]          # 2 would exceed 100, and blocks 3 behind it
    assert a.resident == 90 and [r.rid for r in q] == [2, 3]
    assert a.take(q, now=1.0, size_of=lambda r: r.nbytes) == []
    a.release(40)                                   # request 0 retires
    got = a.take(q, now=1.0, size_of=lambda r: r.nbytes)
    assert [r.rid for r in got] == [2]              # 3 has not arrived yet
    got = a.take(q, now=6.0, size_of=lambda r: r.nbytes)
    assert [r.rid for r in got] == [3] and a.resident == 71


def test_active_node_cap_holds_back_later_requests():
    a = Admission(1000, max_active_nodes=100)
    q = deque([_req(0, 0.0, 1), _req(1, 0.0, 1), _req(2, 0.0, 1)])
    nodes = {0: 60, 1: 50, 2: 30}
    got = a.take(q, now=0.0, size_of=lambda r: r.nbytes, nodes_of=lambda r: nodes[r.rid])
    assert [r.rid for r in got] == [0]              # 60 + 50 > 100, and FCFS keeps 2 behind 1
    a.release(1, 60)
    got = a.take(q, now=0.0, size_of=lambda r: r.nbytes, nodes_of=lambda r: nodes[r.rid])
    assert [r.rid for r in got] == [1, 2] and a.active_nodes == 80


def test_node_cap_never_blocks_an_idle_server():
    a = Admission(1000, max_active_nodes=10)
    got = a.take(deque([_req(0, 0.0, 1)]), now=0.0, size_of=lambda r: r.nbytes, nodes_of=lambda r: 500)
    assert [r.rid for r in got] == [0]


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
