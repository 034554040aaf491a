"""Admission of the serving loop (host logic, CPU, fake jobs): first come first served
while work is in flight, eviction of idle resident systems, skip-ahead only when
nothing is in flight, and an error for a request that can never fit the budget."""
from collections import OrderedDict
from types import SimpleNamespace

import pytest

from paper_1401_7441_gb300 import serving as SV


class _FakeSystem:
    def __init__(self):
        self.closed = False

    def close(self):
        self.closed = True


def _server(budget, streams=2, resident=()):
    srv = SV.Server.__new__(SV.Server)          # no device: only the admission state
    srv.budget = float(budget)
    srv.streams = [object() for _ in range(streams)]
    srv.resident = OrderedDict()
    srv.used = 0
    for rid, nbytes, busy in resident:
        srv.resident[rid] = SimpleNamespace(bytes=nbytes, busy=busy, system=_FakeSystem(), phi=object())
        srv.used += nbytes
    return srv


def _job(rid, nbytes):
    return SimpleNamespace(req=SimpleNamespace(rid=rid), est_bytes=nbytes, stream=None, t_admit=0.0)


def test_fifo_while_work_is_in_flight():
    srv = _server(10)
    a, b, c = _job(1, 6), _job(2, 6), _job(3, 1)
    first = srv._admit([a, b, c], [], 4)
    assert first == [a]                                  # b does not fit behind a: wait (FIFO)
    assert srv.used == 6 and a.stream is srv.streams[0]
    assert srv._admit([b, c], [a], 4) == []              # a in flight: b waits, c stays behind it


def test_idle_resident_systems_are_evicted_least_recently_used_first():
    srv = _server(10, resident=[(7, 4, False), (8, 4, False)])
    j = _job(1, 5)
    assert srv._admit([j], [], 4) == [j]
    assert 7 not in srv.resident and 8 in srv.resident      # one eviction was enough
    assert srv.used == 4 + 5


def test_skip_ahead_only_when_nothing_is_in_flight():
    # a busy resident system (the parent of a prepared request) holds 8 of 10 bytes: the
    # head request (5) cannot fit until something finishes, and nothing is in flight
    srv = _server(10, resident=[(7, 8, True)])
    head, small = _job(1, 5), _job(2, 2)
    assert srv._admit([head, small], [], 4) == [small]
    assert head.stream is None and srv.used == 10


def test_streams_and_inflight_limits():
    srv = _server(100, streams=2)
    jobs = [_job(k, 1) for k in range(4)]
    got = srv._admit(jobs, [], 3)
    assert got == jobs[:2]                               # two streams
    assert len({id(j.stream) for j in got}) == 2
    srv2 = _server(100, streams=4)
    assert srv2._admit(jobs, [], 3) == jobs[:3]          # in-flight limit


def test_request_larger_than_the_budget_is_an_error():
    srv = _server(10)
    with pytest.raises(RuntimeError, match="more than the whole"):
        srv._admit([_job(1, 11)], [], 4)
