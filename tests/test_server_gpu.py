"""GPU tests of the streaming server (tvolap_server_*): every stream against the
FP64 oracle (output delayed by L), one stream alone and in a mix of streams
arriving and leaving (bit-identical), graph replay against direct launches,
admission by device footprint, a bad filter index, and the bounded input wait
running out (a flag nothing sets) with the server staying usable.

Tolerance against the oracle: rel-L2 <= 1e-5 and max-abs <= 1e-4 x peak.
"""
import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT_STATUS = -6
CAPACITY_STATUS = -5
ARG_STATUS = -1


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _server(dev, base=16, top=64, cap=16, arena=256 << 20, **kw):
    from paper_2310_00319_gb300.server import Server
    return Server(base, top, cap, max_out=2, arena_bytes=arena, device=dev, **kw)


def _irs(s, n_out, dev):
    return torch.from_numpy(np.ascontiguousarray(s.irs[:, :n_out])).to(dev)


def drive(srv, streams, starts, dev, n_outs=None, max_ticks=100000):
    """Admit stream i at tick starts[i], feed one block per due tick, retire
    it after its last block. Returns each stream's output blocks [n_out, nb, L]."""
    n_outs = n_outs or [2] * len(streams)
    outs = [np.zeros((n_outs[i], s.n_blocks, s.L), np.float32) for i, s in enumerate(streams)]
    ids = [None] * len(streams)
    given = [0] * len(streams)
    done = 0
    owner = {}
    tick = 0
    while done < len(streams) and tick < max_ticks:
        for i, s in enumerate(streams):
            if ids[i] is None and starts[i] == tick:
                ids[i] = srv.admit(s.L, _irs(s, n_outs[i], dev))
                owner[ids[i]] = i
        due = srv.due()
        for sid in due:
            i = owner[int(sid)]
            s, b = streams[i], given[i]
            assert srv.state(int(sid))[1] == b
            srv.inp[sid, :s.L] = s.x[b * s.L:(b + 1) * s.L]
            srv.sel[sid] = s.sel[b]
        srv.tick()
        srv.wait()
        for sid in due:
            i = owner[int(sid)]
            s, b = streams[i], given[i]
            outs[i][:, b, :] = srv.out[sid, :n_outs[i], :s.L]
            given[i] += 1
            if given[i] == s.n_blocks:
                srv.retire(int(sid))
                del owner[int(sid)]
                done += 1
        tick += 1
    assert done == len(streams), "streams did not finish"
    return outs


def _oracle_stream(s, n_out):
    nb, L = s.n_blocks, s.L
    F, _, ir_len = s.irs.shape
    irs = s.irs[:, :n_out].reshape(F * n_out, ir_len)
    sched = np.stack([s.sel * n_out + o for o in range(n_out)]).astype(np.int32)
    return oracle.tvolap_direct(s.x[None, :], irs, L, sched, out_len=(nb - 1) * L,
                                out_to_in=[0] * n_out)


def _assert_close(y, ref, what):
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    mx = np.max(np.abs(y - ref)) / np.max(np.abs(ref))
    assert rel <= 1e-5 and mx <= 1e-4, (what, rel, mx)


def test_streams_match_oracle():
    dev = _dev()
    S = W.serving_streams(41, 7)
    n_outs = [2, 1, 2, 2, 1, 2, 2]
    starts = [0, 0, 3, 5, 9, 14, 20]
    srv = _server(dev)
    outs = drive(srv, S, starts, dev, n_outs)
    for i, s in enumerate(S):
        ref = _oracle_stream(s, n_outs[i])
        y = outs[i].reshape(n_outs[i], -1).astype(np.float64)
        # block 0 emits samples [-L, 0): silence up to FP32 rounding
        assert np.max(np.abs(y[:, :s.L])) <= 1e-5 * np.max(np.abs(ref)), i
        _assert_close(y[:, s.L:], ref, (i, s.L))
    st = srv.stats()
    assert st["live"] == 0 and st["pending"] == 0 and st["arena_used"] == 0
    srv.close()


def test_alone_equals_mix_bitwise():
    """Continuous batching: the result of a stream does not depend on the other
    streams admitted, running or retired around it."""
    dev = _dev()
    A = W.serving_streams(42, 1, hops=(32,), blocks=(70, 70))[0]
    others = W.serving_streams(43, 9, blocks=(10, 40))
    srv = _server(dev)
    alone = drive(srv, [A], [0], dev)[0]
    srv.close()
    srv = _server(dev)
    starts = [5] + [int(v) for v in np.random.default_rng(1).integers(0, 60, len(others))]
    mix = drive(srv, [A] + others, starts, dev)[0]
    srv.close()
    np.testing.assert_array_equal(alone, mix)


def test_graph_equals_direct_launches_and_timing():
    dev = _dev()
    from paper_2310_00319_gb300.server import OPT_GRAPH, OPT_TIMING
    S = W.serving_streams(44, 5)
    starts = [0, 1, 2, 3, 4]
    runs = []
    for opt in ((OPT_GRAPH, 1), (OPT_GRAPH, 0), (OPT_TIMING, 1)):
        srv = _server(dev)
        srv.set_option(*opt)
        runs.append(drive(srv, S, starts, dev))
        st = srv.stats()
        if opt[0] == OPT_TIMING:
            assert st["timed_ticks"] == st["ticks"] > 0
            assert all(v > 0 for v in st["stage_ms"])
        srv.close()
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            np.testing.assert_array_equal(a, b)


def test_admission_by_footprint():
    dev = _dev()
    from paper_2310_00319_gb300._lib import TvolapError
    S = W.serving_streams(45, 3, hops=(64,), ir_min=1000, ir_max=1000)
    probe = _server(dev)
    fp = probe.footprint(64, -(-1000 // 128), 2, S[0].irs.shape[0])
    probe.close()
    srv = _server(dev, cap=8, arena=2 * fp)
    a = srv.admit(64, _irs(S[0], 2, dev))
    b = srv.admit(64, _irs(S[1], 2, dev))
    with pytest.raises(TvolapError) as ei:
        srv.admit(64, _irs(S[2], 2, dev))
    assert ei.value.status == CAPACITY_STATUS
    assert srv.stats()["arena_used"] == 2 * fp
    srv.retire(a)
    c = srv.admit(64, _irs(S[2], 2, dev))
    assert c == a and srv.stats()["arena_used"] == 2 * fp
    srv.retire(b)
    srv.retire(c)
    srv.wait()
    srv.close()
    # slot limit: two slots, arena to spare
    srv = _server(dev, cap=2, arena=16 * fp)
    srv.admit(64, _irs(S[0], 2, dev))
    srv.admit(64, _irs(S[1], 2, dev))
    with pytest.raises(TvolapError) as ei:
        srv.admit(64, _irs(S[2], 2, dev))
    assert ei.value.status == CAPACITY_STATUS
    srv.wait()
    srv.close()


def test_bad_filter_index_is_rejected():
    dev = _dev()
    from paper_2310_00319_gb300._lib import TvolapError
    s = W.serving_streams(46, 1)[0]
    srv = _server(dev)
    i = srv.admit(s.L, _irs(s, 2, dev))
    srv.wait()
    while len(srv.due()) == 0:
        srv.tick()
        srv.wait()
    srv.sel[i] = s.irs.shape[0]           # one past the last filter
    with pytest.raises(TvolapError) as ei:
        srv.tick()
    assert ei.value.status == ARG_STATUS
    assert srv.state(i)[1] == 0 and srv.stats()["ticks"] >= 0
    srv.close()


def test_input_wait_times_out_and_server_recovers():
    """With the input wait on, a tick whose staging is never declared written
    gives up after the limit (no fault, no hang), processes nothing and is
    rolled back; the same blocks then run normally and the outputs equal those
    of a run that never timed out."""
    dev = _dev()
    from paper_2310_00319_gb300._lib import TvolapError
    from paper_2310_00319_gb300.server import OPT_WAIT_US
    s = W.serving_streams(47, 1, hops=(16,), blocks=(30, 30))[0]
    srv = _server(dev)
    ref = drive(srv, [s], [0], dev)[0]
    srv.close()

    srv = _server(dev)
    srv.set_option(OPT_WAIT_US, 20000)                   # 20 ms
    i = srv.admit(s.L, _irs(s, 2, dev))
    srv.wait()
    due = srv.due()
    assert list(due) == [i]
    srv.inp[i, :s.L] = s.x[:s.L]
    srv.sel[i] = s.sel[0]
    srv.tick()                                           # nothing posts tick 1
    with pytest.raises(TvolapError) as ei:
        srv.wait()
    assert ei.value.status == TIMEOUT_STATUS
    assert srv.state(i)[1] == 0 and srv.stats()["ticks"] == 0
    # the same tick again, now posted: runs normally from here on
    out = np.zeros_like(ref)
    for b in range(s.n_blocks):
        assert list(srv.due()) == [i]
        srv.inp[i, :s.L] = s.x[b * s.L:(b + 1) * s.L]
        srv.sel[i] = s.sel[b]
        srv.post(srv.stats()["ticks"] + 1)              # the next tick's number
        srv.tick()
        srv.wait()
        out[:, b, :] = srv.out[i, :2, :s.L]
    np.testing.assert_array_equal(out, ref)
    srv.close()


def test_edge_streams():
    """Hop 1024 with base 128 (eight base ticks per block, 2048 bins), a single
    filter of one tap (M = 1), a mono stream, and a server of capacity 1 that
    retires a stream before it turns live and admits another."""
    dev = _dev()
    rng = np.random.default_rng(71)

    def stream(L, ir_len, F, nb):
        irs = np.stack([W.binaural_pair(rng, ir_len, 0.1) for _ in range(F)]).astype(np.float32)
        return W.ServeStream(L, irs, W.white(rng, nb * L).astype(np.float32),
                             W.head_walk(rng, nb, F))

    S = [stream(1024, 5000, 3, 12), stream(128, 1, 1, 30), stream(256, 2000, 2, 20)]
    srv = _server(dev, base=128, top=1024, cap=4, arena=512 << 20)
    outs = drive(srv, S, [0, 2, 5], dev, n_outs=[2, 2, 1])
    srv.close()
    for i, s in enumerate(S):
        n_out = [2, 2, 1][i]
        ref = _oracle_stream(s, n_out)
        y = outs[i].reshape(n_out, -1).astype(np.float64)
        _assert_close(y[:, s.L:], ref, ("edge", i, s.L))
    srv = _server(dev, cap=1)
    t = W.serving_streams(72, 2)
    i0 = srv.admit(t[0].L, _irs(t[0], 2, dev))
    srv.retire(i0)                      # before it ever turned live
    assert srv.state(i0)[0] == 0
    out = drive(srv, [t[1]], [0], dev)[0]
    ref = _oracle_stream(t[1], 2)
    _assert_close(out.reshape(2, -1).astype(np.float64)[:, t[1].L:], ref, "after early retire")
    srv.close()


def test_pipelined_ticks_equal_one_at_a_time():
    """Two ticks in flight: due() hands out the staging set of the tick two
    back (waiting for it), whose outputs are read before the set is refilled.
    Results equal those of ticks run one at a time, bit for bit."""
    dev = _dev()
    S = W.serving_streams(48, 4, hops=(16, 32, 64), blocks=(20, 40))
    srv = _server(dev)
    ref = drive(srv, S, [0, 0, 0, 0], dev)
    srv.close()

    srv = _server(dev)
    ids = [srv.admit(s.L, _irs(s, 2, dev)) for s in S]
    srv.wait()
    owner = {sid: i for i, sid in enumerate(ids)}
    given = [0] * len(S)
    outs = [np.zeros((2, s.n_blocks, s.L), np.float32) for s in S]
    inflight = {}                       # staging set -> [(stream, block)] of its last tick
    done = 0

    def collect(buf):
        for i, b in inflight.pop(buf, []):
            outs[i][:, b, :] = srv.outs(buf)[ids[i], :2, :S[i].L]

    for _ in range(100000):
        if done == len(S):
            break
        due = srv.due()                 # waits for the tick that used this set
        collect(srv.buf)
        batch = []
        for sid in due:
            i = owner[int(sid)]
            s, b = S[i], given[i]
            srv.inp[sid, :s.L] = s.x[b * s.L:(b + 1) * s.L]
            srv.sel[sid] = s.sel[b]
            batch.append((i, b))
            given[i] += 1
        inflight[srv.buf] = batch
        srv.tick()
        for i, b in batch:
            if b + 1 == S[i].n_blocks:
                srv.retire(ids[i])      # its last block is enqueued; the slot is free later
                done += 1
    srv.wait()
    for buf in list(inflight):
        collect(buf)
    srv.close()
    for a, b in zip(ref, outs):
        np.testing.assert_array_equal(a, b)


def _feed(srv, sid, s, b0, b1, extra=()):
    """Feed stream s's blocks b0 .. b1-1 to stream id sid (and silence with
    filter 0 to the extra stream ids); returns sid's output blocks [2, b1-b0, L]."""
    outs, b = [], b0
    for _ in range(100 * (b1 - b0) + 100):
        if b == b1:
            break
        due = [int(v) for v in srv.due()]
        for x in due:
            if x == sid:
                assert srv.state(sid)[1] == b
                srv.inp[x, :s.L] = s.x[b * s.L:(b + 1) * s.L]
                srv.sel[x] = s.sel[b]
            else:
                assert x in extra
                srv.inp[x, :] = 0.0
                srv.sel[x] = 0
        srv.tick()
        srv.wait()
        if sid in due:
            outs.append(np.array(srv.out[sid, :2, :s.L]))
            b += 1
    assert b == b1, "stream did not run"
    return np.stack(outs, 1)


@pytest.mark.parametrize("where", ["cuda", "cpu"])
def test_snapshot_restore_and_migration_bitwise(where):
    """A stream snapshotted after some blocks continues bit for bit when
    restored: into another slot of the same server after retiring it
    (migration), and into a fresh server with other streams around it."""
    dev = _dev()
    A = W.serving_streams(90, 1, hops=(32,), blocks=(50, 50))[0]
    B = W.serving_streams(91, 2, hops=(16, 64), blocks=(50, 50))
    srv = _server(dev)
    other = srv.admit(B[0].L, _irs(B[0], 2, dev))          # takes the first slot and piece
    sid = srv.admit(A.L, _irs(A, 2, dev))
    _feed(srv, sid, A, 0, 20, extra=(other,))
    if where == "cuda":
        snap = srv.snapshot(sid)
    else:
        n = srv.snapshot(sid).numel()
        snap = srv.snapshot(sid, torch.empty(n, dtype=torch.uint8).pin_memory())
    ref = _feed(srv, sid, A, 20, 50, extra=(other,))
    # migration: retire, then restore into the same server (another slot / piece)
    srv.retire(sid)
    srv.retire(other)
    late = [srv.admit(b.L, _irs(b, 2, dev)) for b in B]    # take the old slots first
    sid2 = srv.restore(snap)
    assert sid2 not in (sid, other)
    got = _feed(srv, sid2, A, 20, 50, extra=tuple(late))
    np.testing.assert_array_equal(got, ref)
    srv.close()
    # a fresh server
    srv2 = _server(dev)
    sid3 = srv2.restore(snap)
    got2 = _feed(srv2, sid3, A, 20, 50)
    np.testing.assert_array_equal(got2, ref)
    srv2.close()


def test_restore_rejects_a_foreign_buffer():
    from paper_2310_00319_gb300 import TvolapError
    dev = _dev()
    srv = _server(dev)
    with pytest.raises(TvolapError):
        srv.restore(torch.zeros(4096, dtype=torch.uint8, device=dev))
    srv.close()
