"""CPU tests of the server's admission queue on its host scheduler
(tvolap_sched_submit / _pump / _admitted / _cancel / _queue): requests that
find no slot or arena piece wait, and are admitted in arrival order as
retired streams free their room, each record carrying the base ticks it
waited. Checked against a plain Python model of slots, first-fit placement and
a FIFO. No GPU is needed."""
import numpy as np
import pytest

from paper_2310_00319_gb300._lib import TvolapError
from paper_2310_00319_gb300.server import Scheduler

CAPACITY, ARG = -5, -1


def _up(v, a=256):
    return (v + a - 1) // a * a


def _footprint(L, M, n_out, F):
    spec = 2 * L * 8
    return (_up(F * n_out * M * spec) + _up(2 * M * spec) + _up(n_out * 3 * L * 4) +
            _up(L * 4))


class Model:
    """Slots (lowest free id first), first-fit arena with merging, and a FIFO
    whose head alone may be admitted."""

    def __init__(self, slots, arena):
        self.free_ids = set(range(slots))
        self.free = [(0, arena)]
        self.queue = []          # (ticket, fp, submit_tick)
        self.live = {}           # id -> (off, fp)
        self.tick = 0
        self.next_ticket = 1
        self.records = []

    def _take(self, n):
        for i, (o, s) in enumerate(self.free):
            if s >= n:
                self.free[i:i + 1] = [] if s == n else [(o + n, s - n)]
                return o
        return None

    def _give(self, o, n):
        self.free = sorted(self.free + [(o, n)])
        merged = []
        for a, s in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + s)
            else:
                merged.append((a, s))
        self.free = merged

    def submit(self, fp):
        t = self.next_ticket
        self.next_ticket += 1
        self.queue.append((t, fp, self.tick))
        self.pump()
        return t

    def pump(self):
        while self.queue and self.free_ids:
            t, fp, st = self.queue[0]
            off = self._take(fp)
            if off is None:
                return
            i = min(self.free_ids)
            self.free_ids.remove(i)
            self.live[i] = (off, fp)
            self.records.append((t, i, self.tick - st))
            self.queue.pop(0)

    def retire(self, i):
        off, fp = self.live.pop(i)
        self._give(off, fp)
        self.free_ids.add(i)


def test_fifo_admission_as_room_frees_up():
    """Three slots, five requests: three are admitted at once, the fourth and
    fifth wait and are admitted, in order, at the first pump after a stream
    retires; the wait is counted in base ticks."""
    sch = Scheduler(16, 64, 3, 2, 1 << 30)
    tickets = [sch.submit(32, 4, 2, 3) for _ in range(5)]
    assert tickets == [1, 2, 3, 4, 5]
    assert sch.admitted() == [(1, 0, 0), (2, 1, 0), (3, 2, 0)]
    assert sch.queue() == (2, 0)
    for _ in range(7):
        sch.advance()
    assert sch.queue() == (2, 7) and sch.pump() == 0
    sch.retire(1)
    assert sch.pump() == 1
    assert sch.admitted() == [(4, 1, 7)]
    sch.advance()
    sch.retire(0)
    sch.retire(2)
    assert sch.pump() == 1                  # one request was left
    assert sch.admitted() == [(5, 0, 8)]
    assert sch.queue() == (0, 0) and sch.admitted() == []


def test_nothing_overtakes_the_head():
    """A request at the head that needs more arena than is free holds back a
    smaller one behind it that would fit; both go once the room is there."""
    arena = 3 << 20
    sch = Scheduler(16, 64, 8, 2, arena)
    big_fp = _footprint(64, 200, 2, 4)
    small_fp = _footprint(16, 2, 1, 1)
    a = sch.submit(64, 120, 2, 4)                        # takes most of the arena
    assert sch.admitted() == [(a, 0, 0)]
    b = sch.submit(64, 200, 2, 4)                        # does not fit next to it
    c = sch.submit(16, 2, 1, 1)                          # would fit, but waits behind b
    assert big_fp <= arena and small_fp < arena - sch.arena()[0]
    assert sch.pump() == 0 and sch.queue()[0] == 2 and sch.admitted() == []
    sch.advance()
    sch.retire(0)
    assert sch.pump() == 2
    assert sch.admitted() == [(b, 0, 1), (c, 1, 1)]


def test_request_larger_than_the_arena_is_refused_at_submit():
    sch = Scheduler(16, 64, 4, 2, 1 << 20)
    with pytest.raises(TvolapError) as ei:
        sch.submit(64, 500, 2, 36)
    assert ei.value.status == CAPACITY
    assert sch.queue() == (0, 0)
    with pytest.raises(TvolapError) as ei:
        sch.submit(48, 2, 1, 1)                          # bad hop
    assert ei.value.status == ARG
    assert sch.submit(16, 1, 1, 1) == 1                  # tickets count accepted requests only


def test_cancel_a_waiting_request():
    sch = Scheduler(16, 64, 1, 2, 1 << 24)
    a = sch.submit(16, 2, 1, 1)
    b = sch.submit(16, 2, 1, 1)
    c = sch.submit(16, 2, 1, 1)
    sch.cancel(b)
    for t in (a, b, 99):                                 # admitted, cancelled, unknown
        with pytest.raises(TvolapError) as ei:
            sch.cancel(t)
        assert ei.value.status == ARG
    sch.retire(0)
    sch.pump()
    assert sch.admitted() == [(a, 0, 0), (c, 0, 0)]


def test_injected_failures_delay_the_queue_and_change_nothing_else():
    """TVOLAP_SERVER_OPT_FAIL_ADMITS through the queue: every refused attempt
    leaves the request at the head; it is admitted, with the placement an
    uninjected scheduler gives, once the injected failures are used up."""
    ref = Scheduler(16, 64, 4, 2, 1 << 24)
    sch = Scheduler(16, 64, 4, 2, 1 << 24)
    sch.fail_admits(3)
    t = sch.submit(32, 5, 2, 4)
    assert sch.admitted() == [] and sch.queue()[0] == 1
    for _ in range(2):
        sch.advance()
        assert sch.pump() == 0
    sch.advance()
    assert sch.pump() == 1
    assert sch.admitted() == [(t, 0, 3)]
    ref.admit(32, 5, 2, 4)
    assert sch.arena() == ref.arena()


def test_random_sequences_against_the_model():
    rng = np.random.default_rng(3)
    arena, slots = 24 << 20, 12
    sch = Scheduler(16, 128, slots, 2, arena)
    model = Model(slots, arena)
    for step in range(1500):
        u = rng.uniform()
        if u < 0.45:
            L = int(rng.choice([16, 32, 64, 128]))
            M = int(rng.integers(1, 80))
            F = int(rng.integers(1, 6))
            fp = _footprint(L, M, 2, F)
            if fp > arena:
                continue
            assert sch.submit(L, M, 2, F) == model.submit(fp)
        elif u < 0.75 and model.live:
            i = int(rng.choice(sorted(model.live)))
            sch.retire(i)
            model.retire(i)
        elif u < 0.9:
            sch.pump()
            model.pump()
        else:
            sch.advance()
            model.tick += 1
        got = sch.admitted()
        want, model.records = model.records, []
        assert got == want
        waiting = len(model.queue)
        oldest = model.tick - model.queue[0][2] if model.queue else 0
        assert sch.queue() == (waiting, oldest)
        assert sch.arena()[0] == sum(fp for _, fp in model.live.values())
