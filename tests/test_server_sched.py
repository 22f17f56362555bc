"""CPU tests of the streaming server's host scheduler (tvolap_sched_*): stream
footprints, first-fit placement with merging of freed pieces (against a
Python model), admission limits, phase choice and the due lists per base
tick. No GPU is needed."""
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


def _block_bytes(L, M, n_out):
    spec = 2 * L * 8
    return (1 + n_out) * M * spec + n_out * spec


@pytest.mark.parametrize("L,M,n_out,F", [(16, 1, 1, 1), (64, 94, 2, 36), (256, 282, 2, 36),
                                         (1024, 3, 1, 5)])
def test_footprint(L, M, n_out, F):
    assert Scheduler.footprint(L, M, n_out, F) == _footprint(L, M, n_out, F)


class FirstFit:
    """Reference placement: lowest-offset free piece that fits; freed pieces
    merge with free neighbours."""

    def __init__(self, size):
        self.free = [(0, size)]

    def take(self, n):
        for i, (o, s) in enumerate(self.free):
            if s >= n:
                if s == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (o + n, s - n)
                return o
        return None

    def give(self, o, n):
        self.free.append((o, n))
        self.free.sort()
        merged = []
        for a, s in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + s)
            else:
                merged.append((a, s))
        self.free = merged

    def largest(self):
        return max((s for _, s in self.free), default=0)


def test_first_fit_placement_against_model():
    rng = np.random.default_rng(0)
    arena = 64 << 20
    sch = Scheduler(64, 256, 64, 2, arena)
    model = FirstFit(arena)
    live = {}
    for step in range(600):
        if live and rng.uniform() < 0.45:
            i = int(rng.choice(list(live)))
            off, fp = live.pop(i)
            sch.retire(i)
            model.give(off, fp)
        else:
            L = int(rng.choice([64, 128, 256]))
            M = int(rng.integers(1, 60))
            F = int(rng.integers(1, 8))
            fp = _footprint(L, M, 2, F)
            want = model.take(fp) if len(live) < 64 else None
            if want is None:
                with pytest.raises(TvolapError) as ei:
                    sch.admit(L, M, 2, F)
                assert ei.value.status == CAPACITY
                continue
            i, off, _ = sch.admit(L, M, 2, F)
            assert off == want and i not in live
            live[i] = (off, fp)
        used, largest = sch.arena()
        assert used == sum(fp for _, fp in live.values())
        assert largest == model.largest()
    for i, (off, fp) in list(live.items()):
        sch.retire(i)
    assert sch.arena() == (0, arena)


def test_slot_limit_and_failed_admit_changes_nothing():
    sch = Scheduler(16, 64, 2, 2, 1 << 30)
    a = sch.admit(16, 3, 2, 4)
    b = sch.admit(32, 3, 1, 4)
    before = sch.arena()
    with pytest.raises(TvolapError) as ei:
        sch.admit(64, 3, 2, 4)
    assert ei.value.status == CAPACITY and sch.arena() == before
    sch.retire(a[0])
    c = sch.admit(64, 3, 2, 4)
    assert c[0] == a[0]
    sch.retire(b[0])
    sch.retire(c[0])
    assert sch.arena() == (0, (1 << 30))


def test_injected_admission_failures_change_nothing():
    """Fault injection on the host: the next n valid admissions are refused
    with TVOLAP_ERR_CAPACITY and leave the slots, the arena, the phase loads
    and the due lists as they were; invalid arguments are still reported as
    such and do not use up an injected failure; then admission resumes with
    the same placement it would have had."""
    ref = Scheduler(16, 64, 4, 2, 1 << 24)
    sch = Scheduler(16, 64, 4, 2, 1 << 24)
    for s in (ref, sch):
        a = s.admit(32, 3, 2, 4)
        s.activate(a[0])
        s.advance()
    state = (sch.arena(), sch.phase_loads().tolist(), sch.due().tolist())
    sch.fail_admits(2)
    for _ in range(2):
        with pytest.raises(TvolapError) as ei:
            sch.admit(64, 5, 2, 4)
        assert ei.value.status == CAPACITY
        with pytest.raises(TvolapError) as ei:
            sch.admit(48, 5, 2, 4)                       # bad hop: not an injected failure
        assert ei.value.status == ARG
        assert (sch.arena(), sch.phase_loads().tolist(), sch.due().tolist()) == state
    sch.fail_admits(0)                                   # clearing works too
    sch.fail_admits(1)
    with pytest.raises(TvolapError):
        sch.admit(64, 5, 2, 4)
    assert sch.admit(64, 5, 2, 4) == ref.admit(64, 5, 2, 4)
    with pytest.raises(TvolapError) as ei:
        sch.fail_admits(-1)
    assert ei.value.status == ARG


@pytest.mark.parametrize("args", [(48, 1, 1, 1), (8, 1, 1, 1), (128, 1, 1, 1), (32, 0, 1, 1),
                                  (32, 1, 3, 1), (32, 1, 1, 0)])
def test_bad_stream_arguments(args):
    sch = Scheduler(16, 64, 4, 2, 1 << 20)
    with pytest.raises(TvolapError) as ei:
        sch.admit(*args)
    assert ei.value.status == ARG


@pytest.mark.parametrize("args", [(24, 64, 4, 2), (16, 256, 4, 2), (64, 32, 4, 2),
                                  (16, 64, 0, 2), (16, 64, 4, 3)])
def test_bad_scheduler_arguments(args):
    with pytest.raises(TvolapError) as ei:
        Scheduler(*args, 1 << 20)
    assert ei.value.status == ARG


def test_phase_choice_evens_out_the_load():
    """Each new stream goes to the phase whose base ticks (those it would be
    due in) are least loaded: smallest heaviest tick, then smallest sum, then
    lowest phase. Loads add up to every stream's bytes per block in each base
    tick it is due in, and random streams end up spread evenly."""
    rng = np.random.default_rng(1)
    sch = Scheduler(64, 256, 1024, 2, 1 << 40)
    total = np.zeros(4, np.int64)
    phases = {}
    for _ in range(500):
        L = int(rng.choice([64, 128, 256]))
        M = int(rng.integers(20, 1200)) * 64 // L
        r = L // 64
        before = total.copy()
        i, _, ph = sch.admit(L, M, 2, 36)
        key = [(before[p::r].max(), before[p::r].sum(), p) for p in range(r)]
        assert ph == min(key)[2], (key, ph)
        load = _block_bytes(L, M, 2)
        total[ph::r] += load
        phases[i] = (r, ph, load)
        np.testing.assert_array_equal(sch.phase_loads(), total)
    assert (total.max() - total.min()) / total.mean() < 0.02
    # retiring takes the load back off
    for i in list(phases)[:100]:
        r, ph, load = phases.pop(i)
        sch.retire(i)
        total[ph::r] -= load
    np.testing.assert_array_equal(sch.phase_loads(), total)


def test_due_lists_follow_phases_and_activation():
    sch = Scheduler(16, 128, 32, 2, 1 << 30)
    streams = {}
    for L in (16, 32, 64, 128, 32, 64, 128, 16):
        i, _, ph = sch.admit(L, 4, 2, 2)
        streams[i] = (L // 16, ph)
    first = list(streams)[:5]
    for i in first:
        sch.activate(i)
    with pytest.raises(TvolapError):
        sch.activate(first[0])                 # already live
    seen = {i: [] for i in streams}
    for t in range(64):
        if t == 20:
            for i in list(streams)[5:]:
                sch.activate(i)
        for i in sch.due():
            seen[int(i)].append(t)
        sch.advance()
    for i, (r, ph) in streams.items():
        start = 0 if i in first else 20
        want = [t for t in range(start, 64) if t % r == ph]
        assert seen[i] == want, (i, r, ph)
