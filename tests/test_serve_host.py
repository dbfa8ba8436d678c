"""Host logic of the serving loop (serve.Server) on the CPU: admission in
arrival order under the HBM budget, one group per kind and step, each on a
free slot, at most max_group jobs and max_group_work pixels or site updates
per group (one larger job alone), and the release of memory and slots when
a group completes.  Launches and CUDA events are stubs here; the
GPU tests run the real groups."""
import collections

import numpy as np
import pytest

from paper_1105_5804_gb300 import build, serve


@pytest.fixture(scope="module", autouse=True)
def _library():
    build.build()   # label job sizes ask the library for workspace bytes (host arithmetic)


class _Event:
    def __init__(self):
        self.done = False

    def query(self):
        return self.done


class _Pool:
    """Pinned result buffers: always available here."""

    def acquire(self, nbytes):
        return object()

    def release(self, buf):
        pass


class _HostRows:
    def __init__(self, n):
        self.a = np.zeros((n, 3), dtype=np.int64)

    def numpy(self):
        return self.a


class StubServer(serve.Server):
    """serve.Server's host state without CUDA streams; launches are recorded."""

    def __init__(self, budget, slots=2, max_group=32, max_group_work=serve.MAX_GROUP_WORK):
        self.budget = int(budget)
        self.in_use = 0
        self.streams = [None] * slots
        self.free_slots = list(range(slots))
        self.max_group = max_group
        self.max_group_work = max_group_work
        self.keep_results = False
        self.queue = collections.deque()
        self.running = []
        self.done = []
        self.peak_in_use = 0
        self.max_running = 0
        self.launched = []
        self.clock = lambda: 0.0
        self.pool = _Pool()

    def _launch(self, kind, jobs):
        g = serve._Group(self.free_slots.pop(), jobs, kind)
        g.event = _Event()
        for j in jobs:
            if kind == "sw":      # the observables' host buffer (filled by the group's stream)
                j.observables = _HostRows(j.sweeps)
        self.running.append(g)
        self.max_running = max(self.max_running, len(self.running))
        self.launched.append((kind, [j.id for j in jobs]))


def _label(jid, side=64):
    return serve.Job(jid, "label", float(jid), H=side, W=side, pixels=None)


def _sw(jid, L=64):
    return serve.Job(jid, "sw", float(jid), L=L, beta=0.4, sweeps=2)


def _finish_all(server, now):
    for g in server.running:
        g.event.done = True
    server.step(now)


def test_admission_is_fifo_under_the_budget():
    small, big = _label(0), _label(4, side=512)
    budget = 3 * small.bytes + _sw(2).bytes + big.bytes - 1   # big fits the budget, not what is left
    s = StubServer(budget)
    for j in [_label(0), _label(1), _sw(2), _label(3), _label(4, side=512), _label(5)]:
        s.submit(j)
    s.step(0.0)
    # label jobs of the step form one group, sw jobs another; job 4 does not
    # fit the budget, and job 5, which would, waits behind it
    assert s.launched == [("label", [0, 1, 3]), ("sw", [2])]
    assert [j.id for j in s.queue] == [4, 5]
    assert s.in_use <= s.budget and s.peak_in_use == s.in_use
    assert all(j.t_admit == 0.0 for g in s.running for j in g.jobs)


def test_a_group_needs_a_free_slot_and_at_most_max_group_jobs(monkeypatch):
    # a completed sw group frees its batch: stub
    monkeypatch.setattr(serve.sw, "sw_batch_destroy", lambda b: None)
    s = StubServer(1 << 40, slots=1, max_group=2)
    for j in [_label(0), _label(1), _label(2), _sw(3)]:
        s.submit(j)
    s.step(0.0)
    assert s.launched == [("label", [0, 1])]      # group full at two; no second slot for the sw group
    s.step(0.1)
    assert s.launched == [("label", [0, 1])]      # the only slot is still busy
    _finish_all(s, 0.2)
    assert s.launched[-1] == ("label", [2])       # the sw job needs a second slot, which one slot cannot give
    _finish_all(s, 0.3)
    assert s.launched[-1] == ("sw", [3])
    _finish_all(s, 0.4)
    assert s.idle() and [j.id for j in s.done] == [0, 1, 2, 3]


def test_a_group_takes_jobs_while_its_work_is_within_the_bound(monkeypatch):
    monkeypatch.setattr(serve.sw, "sw_batch_destroy", lambda b: None)
    s = StubServer(1 << 40, slots=2, max_group_work=3 * 64 * 64)
    # labels of 64^2 pixels: three fit one group; a 256^2 job is larger than
    # the bound and runs as a group of its own
    for j in [_label(0), _label(1), _label(2), _label(3), _label(4, side=256), _sw(5, L=128)]:
        s.submit(j)
    s.step(0.0)
    assert s.launched == [("label", [0, 1, 2])]   # job 3 would exceed the bound; FIFO stops there
    s.step(0.1)
    assert s.launched[-1] == ("label", [3])       # the second slot; job 4 would exceed the bound
    _finish_all(s, 0.2)
    assert s.launched[-2:] == [("label", [4]), ("sw", [5])]   # larger than the bound: alone
    _finish_all(s, 0.3)
    assert s.idle() and [j.id for j in s.done] == [0, 1, 2, 3, 4, 5]


def test_completion_releases_memory_and_slots():
    a, b = _label(0, side=256), _label(1, side=256)
    s = StubServer(a.bytes + b.bytes // 2, slots=2)
    s.submit(a)
    s.submit(b)
    s.step(0.0)
    assert s.launched == [("label", [0])] and s.in_use == a.bytes
    s.step(0.5)                                   # not complete yet: nothing moves
    assert len(s.launched) == 1 and [j.id for j in s.queue] == [1]
    _finish_all(s, 1.0)                           # job 0 done, its bytes and slot back; job 1 admitted
    assert s.launched[-1] == ("label", [1]) and s.in_use == b.bytes
    assert a.t_done == 1.0 and a in s.done
    _finish_all(s, 2.0)
    assert s.in_use == 0 and sorted(s.free_slots) == [0, 1] and s.idle()
    assert s.peak_in_use <= s.budget


def test_a_job_larger_than_the_whole_budget_is_refused():
    j = _label(0, side=256)
    s = StubServer(j.bytes - 1)
    s.submit(j)
    with pytest.raises(ValueError):
        s.step(0.0)


def test_pinned_pool_is_a_buddy_system_over_one_arena():
    import torch
    arena = torch.zeros(4 << 20, dtype=torch.uint8)     # stands in for the pinned arena
    pool = serve.PinnedPool(4 << 20, arena=arena)
    assert pool.top == 22 and pool.free[22] == {0}
    a = pool.acquire(1 << 20)                 # 1 MiB block at the start, the rest split off
    b = pool.acquire((1 << 20) + 1)           # needs 2 MiB: the upper half
    c = pool.acquire(100)                     # 64 KiB from the remaining 1 MiB
    offs = [t.data_ptr() - arena.data_ptr() for t in (a, b, c)]
    assert offs == [0, 2 << 20, 1 << 20] and b.numel() == 2 << 20 and c.numel() == 64 << 10
    assert pool.acquire(2 << 20) is None      # no 2 MiB block left
    pool.release(b)
    assert pool.acquire(2 << 20).data_ptr() - arena.data_ptr() == 2 << 20
    pool.release(a)
    pool.release(c)
    # a and c's blocks merged back into the lower 2 MiB
    assert 0 in pool.free[21]
    with pytest.raises(ValueError):
        pool.acquire(8 << 20)
