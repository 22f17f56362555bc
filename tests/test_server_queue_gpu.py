"""GPU tests of the server's admission queue and of the server at the serving
size.

* Requests submitted while every slot is taken wait in the queue and are
  admitted, oldest first, as streams retire; each stream's output still
  equals the FP64 oracle (delayed by L), and equals, bit for bit, the same
  stream run alone on an empty server.
* Admissions refused by host-side fault injection (TVOLAP_SERVER_OPT_FAIL_ADMITS)
  leave the requests in the queue; they are admitted at later ticks and their
  outputs are unchanged.
* About 1000 binaural streams with serving-size banks (36 pairs of 12000 to
  144000 taps, hops 64/128/256) run a few hundred base ticks; 16 sampled
  streams, both ears, are compared with the oracle element by element.

Tolerance against the oracle: rel-L2 <= 1e-5 and max-abs <= 1e-4 x the
oracle's peak.
"""
import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _server(dev, base=16, top=64, cap=16, arena=256 << 20):
    from paper_2310_00319_gb300.server import Server
    return Server(base, top, cap, max_out=2, arena_bytes=arena, device=dev)


def _irs(s, dev):
    return torch.from_numpy(np.ascontiguousarray(s.irs)).to(dev)


def _oracle_stream(s):
    F, _, ir_len = s.irs.shape
    sched = np.stack([s.sel * 2, s.sel * 2 + 1]).astype(np.int32)
    return oracle.tvolap_direct(s.x[None, :], s.irs.reshape(F * 2, ir_len), s.L, sched,
                                out_len=(s.n_blocks - 1) * s.L, out_to_in=[0, 0])


def _assert_close(y, ref, what):
    peak = np.max(np.abs(ref))
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    mx = np.max(np.abs(y - ref)) / peak
    assert rel <= 1e-5 and mx <= 1e-4, (what, rel, mx)


def drive_queue(srv, streams, submit_at, dev, max_ticks=20000):
    """Submit stream i at tick submit_at[i]; once admitted (admitted() names its
    id) feed it one block per due tick and retire it after its last block.
    Returns the outputs [2, nb, L] per stream and the waits in base ticks."""
    outs = [np.zeros((2, s.n_blocks, s.L), np.float32) for s in streams]
    ticket_of, owner, given, waits = {}, {}, [0] * len(streams), [None] * len(streams)
    done, tick = 0, 0
    while done < len(streams) and tick < max_ticks:
        for i, s in enumerate(streams):
            if submit_at[i] == tick:
                ticket_of[srv.submit(s.L, _irs(s, dev))] = i
        due = srv.due()
        for t, sid, w in srv.admitted():
            i = ticket_of.pop(t)
            owner[sid] = i
            waits[i] = w
        for sid in due:
            i = owner[int(sid)]
            s, b = streams[i], given[i]
            srv.inp[sid, :s.L] = s.x[b * s.L:(b + 1) * s.L]
            srv.sel[sid] = s.sel[b]
        srv.tick()
        srv.wait()
        for sid in due:
            i = owner[int(sid)]
            s, b = streams[i], given[i]
            outs[i][:, b, :] = srv.out[sid, :2, :s.L]
            given[i] += 1
            if given[i] == s.n_blocks:
                srv.retire(int(sid))
                del owner[int(sid)]
                done += 1
        tick += 1
    assert done == len(streams), "streams did not finish"
    return outs, waits


def test_queued_streams_are_admitted_in_order_and_match_oracle():
    dev = _dev()
    S = W.serving_streams(51, 7, blocks=(12, 30))
    submit_at = [0, 0, 0, 1, 2, 2, 9]
    srv = _server(dev, cap=3)
    outs, waits = drive_queue(srv, S, submit_at, dev)
    q = srv.queue()
    assert q["waiting"] == 0 and q["admitted_total"] == len(S)
    assert waits[:3] == [0, 0, 0] and max(waits) > 0 and q["max_wait_ticks"] == max(waits)
    srv.close()
    for i, s in enumerate(S):
        ref = _oracle_stream(s)
        y = outs[i].reshape(2, -1).astype(np.float64)
        _assert_close(y[:, s.L:], ref, i)
    # each stream alone on an empty server gives the same bits
    for i in (3, 6):
        srv = _server(dev, cap=3)
        alone, w = drive_queue(srv, [S[i]], [0], dev)
        assert w == [0]
        srv.close()
        np.testing.assert_array_equal(alone[0], outs[i])


def test_injected_admission_failures_wait_in_the_queue():
    """Host-side fault injection through the real server: the next three
    admissions are refused as if the arena were full; the requests stay queued
    (nothing is dropped), are admitted at later ticks, and give the outputs of
    an uninjected run bit for bit."""
    dev = _dev()
    from paper_2310_00319_gb300.server import OPT_FAIL_ADMITS
    S = W.serving_streams(52, 2, blocks=(15, 20))
    ref_srv = _server(dev)
    ref, ref_w = drive_queue(ref_srv, S, [0, 0], dev)
    ref_srv.close()
    assert ref_w == [0, 0]
    srv = _server(dev)
    srv.set_option(OPT_FAIL_ADMITS, 3)
    outs, waits = drive_queue(srv, S, [0, 0], dev)
    assert min(waits) >= 1, waits                  # both waited behind the refusals
    assert srv.queue()["admitted_total"] == 2 and srv.queue()["waiting"] == 0
    srv.close()
    for a, b in zip(outs, ref):
        np.testing.assert_array_equal(a, b)


def test_serving_size_sampled_streams_match_oracle():
    """About 1000 binaural streams at the serving workload's sizes: hops 64,
    128 and 256 on a 64-sample base tick, 36 response pairs per stream of
    12000..144000 taps (16 distinct banks, each stream transforming its own
    copy), a head-orientation walk choosing the pair of every block, white
    input. 320 base ticks; 16 streams spread over the slots, both ears, are
    compared with the oracle over their first blocks."""
    dev = _dev()
    from paper_2310_00319_gb300.server import Server
    rng = np.random.default_rng(53)
    n_streams, base, top, n_pairs, ticks, rec = 1000, 64, 256, 36, 320, 80
    lens = rng.integers(12000, 144001, 16)
    banks_np = [W.serving_bank(rng, int(n), n_pairs) for n in lens]
    banks = [torch.from_numpy(b).to(dev) for b in banks_np]
    hop_of = rng.choice([64, 128, 256], n_streams)
    bank_of = rng.integers(0, 16, n_streams)
    free = torch.cuda.mem_get_info(dev)[0]
    arena = int(min(0.6 * free, n_streams * 90e6))
    srv = Server(base, top, n_streams, max_out=2, arena_bytes=arena, device=dev)
    ticket_of = {srv.submit(int(hop_of[k]), banks[bank_of[k]]): k for k in range(n_streams)}
    srv.due()
    owner = {}
    for t, sid, w in srv.admitted():
        owner[sid] = ticket_of.pop(t)
    assert not ticket_of, "every stream fits the arena"
    sampled = {sid for sid in list(owner)[::len(owner) // 16][:16]}
    rec_x = {sid: [] for sid in sampled}
    rec_sel = {sid: [] for sid in sampled}
    rec_y = {sid: [] for sid in sampled}
    pool = (0.1 * rng.standard_normal((4096, top))).astype(np.float32)
    sel = rng.integers(0, n_pairs, n_streams).astype(np.int32)
    for tick in range(ticks):
        ids = srv.due()
        k = np.array([owner[int(i)] for i in ids], np.int64)
        srv.inp[ids] = pool[(ids * 7 + tick) % 4096]
        sel[k] = (sel[k] + rng.integers(-1, 2, k.shape[0])) % n_pairs
        srv.sel[ids] = sel[k]
        for sid in ids:
            if int(sid) in sampled and len(rec_x[int(sid)]) < rec:
                L = int(hop_of[owner[int(sid)]])
                rec_x[int(sid)].append(srv.inp[sid, :L].copy())
                rec_sel[int(sid)].append(int(srv.sel[sid]))
        srv.tick()
        srv.wait()
        for sid in ids:
            if int(sid) in sampled and len(rec_y[int(sid)]) < len(rec_x[int(sid)]):
                L = int(hop_of[owner[int(sid)]])
                rec_y[int(sid)].append(srv.out[sid, :2, :L].copy())
    st = srv.stats()
    assert st["live"] == n_streams and st["pending"] == 0
    srv.close()
    assert len({int(hop_of[owner[s]]) for s in sampled}) == 3
    for sid in sorted(sampled):
        k = owner[sid]
        L, nb = int(hop_of[k]), len(rec_y[sid])
        assert nb >= 40
        s = W.ServeStream(L, banks_np[bank_of[k]], np.concatenate(rec_x[sid][:nb]),
                          np.array(rec_sel[sid][:nb], np.int32))
        ref = _oracle_stream(s)
        y = np.concatenate(rec_y[sid][:nb], axis=1).astype(np.float64)
        assert np.max(np.abs(y[:, :L])) <= 1e-5 * np.max(np.abs(ref))   # block 0: silence
        _assert_close(y[:, L:], ref, (sid, L))
