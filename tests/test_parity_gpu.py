"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance for FP32 results against the FP64 oracle: relative L2 error
<= 1e-5 and max-abs error <= 1e-4 times the reference peak, per output.
"""
import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
MAX_ABS = 1e-4


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _plan(wl, dev, n_slots=None):
    from paper_2310_00319_gb300 import Plan
    p = Plan(wl.L, wl.M, n_in=wl.n_in, n_out=wl.n_out, out_to_in=wl.out_to_in,
             n_slots=n_slots or wl.irs.shape[0], device=dev)
    p.load_bank(0, torch.from_numpy(wl.irs).to(dev))
    return p


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _errors(y, ref):
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    rel = np.linalg.norm(y - ref) / max(np.linalg.norm(ref), 1e-30)
    mx = np.max(np.abs(y - ref)) / max(np.max(np.abs(ref)), 1e-30) if ref.size else 0.0
    return rel, mx


def _assert_close(y, ref, what=""):
    y = np.atleast_2d(y)
    ref = np.atleast_2d(ref)
    for o in range(ref.shape[0]):
        if not np.any(ref[o]):
            assert np.max(np.abs(y[o])) < 1e-6, f"{what} out {o} should be silent"
            continue
        rel, mx = _errors(y[o], ref[o])
        assert rel <= REL_L2 and mx <= MAX_ABS, f"{what} out {o}: rel-L2 {rel:.3e}, max {mx:.3e}"


def _run_signal(wl, dev, plan=None):
    plan = plan or _plan(wl, dev)
    y = plan.process_signal(_t(wl.x, dev), _t(wl.sched_a, dev), _t(wl.sched_b, dev),
                            _t(wl.sched_alpha, dev), out_len=wl.out_len)
    plan.check()
    return y.cpu().numpy()


def _ref(wl):
    return oracle.tvolap_direct(wl.x, wl.irs, wl.L, wl.sched_a, wl.sched_b, wl.sched_alpha,
                                out_len=wl.out_len, out_to_in=wl.out_to_in)


# ------------------------------------------------------------------ stage parity
@pytest.mark.parametrize("L", [16, 64, 128, 256, 512, 1024])
def test_forward_spectra_match_oracle(L):
    """Kernel (a): windowed, zero-padded block spectra on the half-bin grid
    (Eqs. 1, 3, 5), for every block including the pre-roll block l = -1 and
    blocks that run past the signal end."""
    dev = _dev()
    wl = W.random_case(1000 + L, L=L, ir_len=2 * L, N=7 * L + L // 2 + 3, n_slots=1)
    from paper_2310_00319_gb300 import Plan
    nb = W.blocks_for(wl.N + 2 * L, L)
    plan = Plan(L, 1, device=dev)
    X = plan.forward_spectra(_t(wl.x, dev), nb).cpu().numpy()[0]
    ref = oracle.block_spectra(wl.x[0], L, list(range(-1, nb - 1)), grid="halfbin")[:, :2 * L]
    rel, mx = _errors(np.concatenate([X.real, X.imag]), np.concatenate([ref.real, ref.imag]))
    assert rel < 1e-6 and mx < 1e-5, (rel, mx)


@pytest.mark.parametrize("L,ir_len", [(16, 100), (128, 4096), (256, 1000), (1024, 5000)])
def test_bank_spectra_match_oracle(L, ir_len):
    """Kernel (b): partition spectra (Eqs. 2, 4, 6), ragged last partition."""
    dev = _dev()
    rng = np.random.default_rng(L + ir_len)
    irs = rng.standard_normal((2, ir_len)).astype(np.float32)
    M = oracle.n_partitions(ir_len, L)
    from paper_2310_00319_gb300 import Plan
    plan = Plan(L, M, n_slots=2, device=dev)
    plan.load_bank(0, _t(irs, dev))
    for s in range(2):
        H = plan.bank_spectra(s).cpu().numpy()
        ref = oracle.partition_spectra(irs[s], L, M, grid="halfbin")[:, :2 * L]
        rel, mx = _errors(np.concatenate([H.real, H.imag]), np.concatenate([ref.real, ref.imag]))
        assert rel < 1e-6 and mx < 1e-5, (s, rel, mx)


@pytest.mark.parametrize("n_slots,interp", [(3, True), (8, True), (8, False), (1, False)])
def test_mac_stage_matches_eq7(n_slots, interp):
    """Kernel (c) alone: Y(t) = sum_m H_t(m) X(t - 2m) from oracle spectra.
    Random slots and weights per block make runs mix up to 2R distinct slots,
    which exercises the run splitting down to single blocks."""
    dev = _dev()
    L = 32
    wl = W.random_case(77 + n_slots, L=L, ir_len=9 * 2 * L - 5, N=60 * L, n_in=2, n_out=2,
                       n_slots=n_slots, interp=interp)
    M, P, nb = wl.M, 2 * L, wl.n_blocks
    X = np.stack([oracle.block_spectra(wl.x[c], L, list(range(-1, nb - 1)), grid="halfbin")[:, :P]
                  for c in range(2)])
    H = np.stack([oracle.partition_spectra(wl.irs[s], L, M, grid="halfbin")[:, :P]
                  for s in range(n_slots)])
    plan = _plan(wl, dev)
    Y = plan.mac(_t(X.astype(np.complex64), dev), _t(wl.sched_a, dev), _t(wl.sched_b, dev),
                 _t(wl.sched_alpha, dev)).cpu().numpy()
    for o in range(2):
        c = wl.out_to_in[o]
        ref = np.zeros((nb, P), np.complex128)
        for t in range(nb):
            a, b, al = wl.sched_a[o, t], wl.sched_b[o, t], np.float64(wl.sched_alpha[o, t])
            Ht = (1 - al) * H[a] + al * H[b]
            for m in range(M):
                if t - 2 * m >= 0:
                    ref[t] += Ht[m] * X[c, t - 2 * m]
        rel, mx = _errors(np.concatenate([Y[o].real, Y[o].imag]),
                          np.concatenate([ref.real, ref.imag]))
        assert rel < 2e-6 and mx < 2e-5, (o, rel, mx)


# ------------------------------------------------------------------ end to end
CASES = [
    # seed, L, ir_len, N, n_in, n_out, n_slots, out_tail, interp, routing
    (1, 16, 150, 1000, 1, 1, 3, 0, True, None),
    (2, 64, 64 * 2, 5000, 1, 1, 2, 0, True, None),           # M = 1 (WOLA case)
    (3, 64, 2000, 4321, 2, 2, 4, 0, False, None),             # ragged N, no mixing
    (4, 128, 4096, 9000, 1, 2, 4, 4096, True, [0, 0]),        # binaural routing, full tail
    (5, 256, 3000, 7777, 3, 3, 5, 513, True, None),
    (6, 512, 6000, 9000, 1, 1, 2, 0, True, None),
    (7, 1024, 4100, 12000, 1, 1, 2, 2048, True, None),        # L = 1024, 2 partitions + ragged
    (8, 32, 70, 20, 1, 1, 2, 40, True, None),                 # signal shorter than a hop
]


@pytest.mark.parametrize("case", CASES, ids=[f"L{c[1]}_ir{c[2]}_N{c[3]}" for c in CASES])
def test_process_signal_matches_oracle(case):
    dev = _dev()
    seed, L, ir_len, N, n_in, n_out, n_slots, tail, interp, routing = case
    wl = W.random_case(seed, L=L, ir_len=ir_len, N=N, n_in=n_in, n_out=n_out, n_slots=n_slots,
                       out_len=N + tail, interp=interp, out_to_in=routing)
    _assert_close(_run_signal(wl, dev), _ref(wl), f"case {seed}")


def test_plain_mono_full_size():
    """Mono, L=128, 96000 samples, 4 IRs of 4096 taps switched every 16 blocks:
    the whole output against the oracle."""
    dev = _dev()
    wl = W.plain_mono()
    y = _run_signal(wl, dev)
    ref = _ref(wl)
    _assert_close(y, ref, "plain mono")
    rel, mx = _errors(y, ref)
    print(f"plain_mono: rel-L2 {rel:.3e} max-abs/peak {mx:.3e}")


def test_plain_at_scale_sampled():
    """64 channels, L=256, 480000 samples, 48000-tap IRs, a new mixed filter
    every block, run whole on the GPU in the benchmark's launch configuration;
    compared with the oracle at 4096 sampled output samples (random positions
    plus the first and last samples of every channel)."""
    dev = _dev()
    wl = W.plain_at_scale()
    y = _run_signal(wl, dev)
    rng = np.random.default_rng(99)
    oc = np.concatenate([rng.integers(0, wl.n_out, 3840), np.repeat(np.arange(wl.n_out), 4)])
    ni = np.concatenate([rng.integers(0, wl.out_len, 3840),
                         np.tile([0, 1, wl.out_len - 2, wl.out_len - 1], wl.n_out)])
    ref = oracle.tvolap_samples(wl.x, wl.irs, wl.L, wl.sched_a, wl.sched_b, wl.sched_alpha,
                                oc, ni, out_to_in=wl.out_to_in)
    got = y[oc, ni].astype(np.float64)
    peak = np.max(np.abs(ref))                   # the oracle's, not the GPU output's
    err = np.abs(got - ref)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"plain_at_scale sampled: rel-L2 {rel:.3e} max-abs/peak {err.max() / peak:.3e}")
    assert rel <= REL_L2 and err.max() <= MAX_ABS * peak
    assert np.all(np.isfinite(y))


def test_empty_and_zero_inputs():
    dev = _dev()
    from paper_2310_00319_gb300 import Plan
    plan = Plan(64, 3, n_slots=1, device=dev)
    plan.load_bank(0, torch.randn(1, 300, device=dev))
    sa = torch.zeros((1, 10), dtype=torch.int32, device=dev)
    # N = 0: output is silence
    y = plan.process_signal(torch.zeros((1, 0), device=dev), sa, out_len=400)
    assert torch.count_nonzero(y).item() == 0
    # out_len = 0: nothing to do
    y = plan.process_signal(torch.randn((1, 100), device=dev), sa, out_len=0)
    assert y.shape == (1, 0)
    plan.check()


def test_invalid_slot_is_silenced_and_reported():
    dev = _dev()
    wl = W.random_case(12, L=64, ir_len=500, N=3000, n_slots=2, interp=False)
    bad = wl.sched_a.copy()
    bad[0, 10:20] = 57
    plan = _plan(wl, dev)
    y = plan.process_signal(_t(wl.x, dev), _t(bad, dev), out_len=wl.out_len)
    from paper_2310_00319_gb300 import TvolapError
    with pytest.raises(TvolapError):
        plan.check()
    plan.check()                                      # record cleared
    irs0 = np.concatenate([wl.irs, np.zeros((1, wl.ir_len), np.float32)])
    fixed = wl.sched_a.copy()
    fixed[0, 10:20] = 2                               # the zero response
    ref = oracle.tvolap_direct(wl.x, irs0, wl.L, fixed, out_len=wl.out_len)
    _assert_close(y.cpu().numpy(), ref, "invalid slot")


@pytest.mark.parametrize("L,n_slots,interp", [(16, 6, True), (256, 6, True), (128, 3, False),
                                               (512, 2, True)])
def test_mac_staging_variants_agree_bitwise(L, n_slots, interp):
    """The persistent and the one-group-per-CTA TMA kernels (one or two bins
    per thread) and the cp.async kernel run the same arithmetic in the same
    order: their outputs are identical. L = 16 (32 bins) has no 64-bin tiles;
    six random slots per block send most groups to the overflow kernel, two or
    three keep them in the group kernels."""
    dev = _dev()
    wl = W.random_case(14 + L, L=L, ir_len=80 * L, N=200 * L, n_in=2, n_out=3, n_slots=n_slots,
                       out_to_in=[0, 1, 1], interp=interp)
    plan = _plan(wl, dev)
    y0 = _run_signal(wl, dev, plan)
    for staging in (1, 3, 4):
        plan.set_option(1, staging)
        np.testing.assert_array_equal(_run_signal(wl, dev, plan), y0)
    _assert_close(y0, _ref(wl), "variants")


@pytest.mark.parametrize("L", [16, 64, 256, 512, 1024])
def test_transform_cta_size_changes_no_result(L):
    """TVOLAP_OPT_XFORM_THREADS (256, 128, 64 threads per CTA of the offline
    transforms) only regroups transforms into CTAs: outputs, block spectra and
    bank spectra are the same bit for bit."""
    dev = _dev()
    from paper_2310_00319_gb300.tvolap import OPT_XFORM_THREADS
    wl = W.random_case(230 + L, L=L, ir_len=3 * L + 7, N=40 * L + 3, n_in=2, n_out=3,
                       n_slots=3, out_len=41 * L, out_to_in=[0, 1, 1])
    from paper_2310_00319_gb300 import Plan
    runs = []
    for th in (0, 128, 64):
        plan = Plan(wl.L, wl.M, n_in=wl.n_in, n_out=wl.n_out, out_to_in=wl.out_to_in,
                    n_slots=wl.irs.shape[0], device=dev)
        plan.set_option(OPT_XFORM_THREADS, th)             # before the bank transform
        plan.load_bank(0, _t(wl.irs, dev))
        y = _run_signal(wl, dev, plan)
        X = plan.block_spectra(_t(wl.x, dev), 0, wl.n_blocks).cpu().numpy()
        H = plan.bank_spectra(1).cpu().numpy()
        runs.append((y, X, H))
        plan.close()
    for r in runs[1:]:
        for a, b in zip(r, runs[0]):
            np.testing.assert_array_equal(a, b)


def test_staging_option_range():
    """TVOLAP_OPT_MAC_STAGING takes 0 .. 5, TVOLAP_OPT_STAGE_TIMING 0 or 1;
    other values and options are refused."""
    from paper_2310_00319_gb300 import TvolapError
    dev = _dev()
    wl = W.random_case(3, L=64, ir_len=300, N=2000, n_slots=2)
    plan = _plan(wl, dev)
    for v in range(6):
        plan.set_option(1, v)
    for v in (1, 0):
        plan.set_option(2, v)
    for v in (0, 64, 128, 256):
        plan.set_option(3, v)
    for opt, v in [(1, -1), (1, 6), (2, 2), (2, -1), (3, 32), (3, 512), (4, 0), (0, 0)]:
        with pytest.raises(TvolapError):
            plan.set_option(opt, v)


@pytest.mark.parametrize("k", [1, 2, 3, 8])
def test_mac_four_filter_groups(k):
    """Staging option 2 stages up to four filters per group of 64 blocks: a
    schedule cycling four filters every k blocks then runs without the
    overflow path. Against the oracle, and against option 0 up to rounding."""
    dev = _dev()
    rng = np.random.default_rng(60 + k)
    L, N, ir_len = 128, 40000, 6000
    nb = W.blocks_for(N, L)
    a = W.cyclic_schedule(nb, 4, k)[None, :].astype(np.int32)
    a = np.concatenate([a, (a + 1) % 4 + 4])                 # output 1: filters 4..7
    wl = W.Workload(f"cyclic4_k{k}", L, W.white(rng, (2, N)).astype(np.float32),
                    (rng.standard_normal((8, ir_len)) / np.sqrt(ir_len)).astype(np.float32),
                    a, a.copy(), np.zeros(a.shape, np.float32), np.arange(2, dtype=np.int32), N)
    plan = _plan(wl, dev)
    y0 = _run_signal(wl, dev, plan)
    plan.set_option(1, 2)
    y2 = _run_signal(wl, dev, plan)
    plan.set_option(1, 5)                                    # persistent, four filters
    np.testing.assert_array_equal(_run_signal(wl, dev, plan), y2)
    _assert_close(y2, _ref(wl), f"four-filter groups k={k}")
    rel = np.linalg.norm(y2 - y0) / np.linalg.norm(y0)
    assert rel <= 1e-6, rel


def test_deterministic_bitwise():
    dev = _dev()
    wl = W.random_case(13, L=128, ir_len=3000, N=20000, n_in=2, n_out=2, n_slots=3)
    plan = _plan(wl, dev)
    y1 = _run_signal(wl, dev, plan)
    y2 = _run_signal(wl, dev, plan)
    np.testing.assert_array_equal(y1, y2)


# ------------------------------------------------------------------ streaming
@pytest.mark.parametrize("L,ir_len,n_in,n_out,routing", [(64, 700, 1, 1, None),
                                                         (128, 2000, 2, 3, [0, 1, 1]),
                                                         (256, 4096, 1, 1, None)])
def test_streaming_equals_offline_delayed_by_L(L, ir_len, n_in, n_out, routing):
    """process_block, one hop at a time with this tick's selection passed as
    device arrays, equals the offline output delayed by exactly L samples."""
    dev = _dev()
    N = 40 * L + L // 2
    wl = W.random_case(200 + L, L=L, ir_len=ir_len, N=N, n_in=n_in, n_out=n_out, n_slots=3,
                       out_len=N, out_to_in=routing)
    plan = _plan(wl, dev)
    n_ticks = wl.n_blocks
    xpad = np.zeros((n_in, n_ticks * L), np.float32)
    xpad[:, :N] = wl.x
    xd = _t(xpad, dev)
    outs = []
    sa, sb, sal = _t(wl.sched_a.T.copy(), dev), _t(wl.sched_b.T.copy(), dev), \
        _t(wl.sched_alpha.T.copy(), dev)
    for t in range(n_ticks):
        outs.append(plan.process_block(xd[:, t * L:(t + 1) * L].contiguous(), None,
                                       sa[t], sb[t], sal[t]).clone())
    plan.check()
    y = torch.cat(outs, dim=1).cpu().numpy()
    ref = _ref(wl)
    # tick 0 emits samples [-L, 0): silence up to FP32 rounding
    assert np.max(np.abs(y[:, :L])) <= 1e-5 * np.max(np.abs(ref))
    _assert_close(y[:, L:L + N], ref[:, :min(N, y.shape[1] - L)], "stream")


def test_stage_timing_changes_no_output():
    """TVOLAP_OPT_STAGE_TIMING: the three stages of every tick are timed (all
    times positive, one count per tick) and the outputs are those of the
    untimed ticks, bit for bit."""
    dev = _dev()
    from paper_2310_00319_gb300.tvolap import OPT_STAGE_TIMING
    L, N = 64, 64 * 25
    wl = W.random_case(210, L=L, ir_len=700, N=N, n_in=2, n_out=3, n_slots=3, out_len=N,
                       out_to_in=[0, 1, 1])
    xd = _t(wl.x, dev)
    sa, sb, sal = _t(wl.sched_a.T.copy(), dev), _t(wl.sched_b.T.copy(), dev), \
        _t(wl.sched_alpha.T.copy(), dev)
    runs = []
    for timing in (0, 1):
        plan = _plan(wl, dev)
        plan.set_option(OPT_STAGE_TIMING, timing)
        outs = [plan.process_block(xd[:, t * L:(t + 1) * L].contiguous(), None, sa[t], sb[t],
                                   sal[t]).clone() for t in range(N // L)]
        ms, n = plan.stage_times()
        if timing:
            assert n == N // L and all(v > 0 for v in ms), (ms, n)
        else:
            assert n == 0 and ms == [0.0, 0.0, 0.0]
        plan.check()
        runs.append(torch.cat(outs, dim=1).cpu().numpy())
        plan.close()
    np.testing.assert_array_equal(runs[0], runs[1])


def test_streaming_set_filter_and_select():
    """set_filter exchanges all partitions at once; select mixes two slots."""
    dev = _dev()
    L, N = 64, 64 * 30
    rng = np.random.default_rng(5)
    x = rng.standard_normal((1, N)).astype(np.float32)
    irs = rng.standard_normal((2, 500)).astype(np.float32)
    from paper_2310_00319_gb300 import Plan
    M = oracle.n_partitions(500, L)
    plan = Plan(L, M, n_slots=2, device=dev)
    plan.load_bank(0, _t(irs, dev))
    assert plan.slot_count == 3                       # slot 2 is output 0's private slot
    nb = W.blocks_for(N, L)
    # schedule: ticks < 10 silent (private slot still zero), 10..19 set_filter(irs[1]),
    # 20.. select a mix of slots 0 and 1 with alpha 0.25
    plan.reset()
    xd = _t(np.concatenate([x, np.zeros((1, nb * L - N), np.float32)], 1), dev)
    outs = []
    for t in range(nb):
        if t == 10:
            plan.set_filter(0, _t(irs[1], dev))
        if t == 20:
            plan.select(0, 0, 1, 0.25)
        outs.append(plan.process_block(xd[:, t * L:(t + 1) * L].contiguous()).clone())
    plan.check()
    y = torch.cat(outs, 1).cpu().numpy()[:, L:L + N]
    irs_o = np.concatenate([irs, np.zeros((1, 500), np.float32)])
    sa = np.full((1, nb), 2, np.int32)
    sb = np.full((1, nb), 2, np.int32)
    al = np.zeros((1, nb), np.float32)
    sa[0, 10:20] = sb[0, 10:20] = 1
    sa[0, 20:], sb[0, 20:], al[0, 20:] = 0, 1, 0.25
    ref = oracle.tvolap_direct(x, irs_o, L, sa, sb, al)
    _assert_close(y, ref, "set_filter/select")


# ------------------------------------------------------------------ state snapshot
@pytest.mark.parametrize("where", ["cuda", "cpu"])
def test_state_snapshot_resumes_bitwise(where):
    """A snapshot taken after some ticks and restored, into the same plan and
    into a fresh plan of the same shape, continues with the same outputs bit
    for bit (host or device snapshot buffer); a plan of another shape refuses it."""
    from paper_2310_00319_gb300 import TvolapError
    dev = _dev()
    L = 128
    N = 30 * L
    wl = W.random_case(80, L=L, ir_len=1500, N=N, n_in=2, n_out=3, n_slots=3,
                       out_to_in=[0, 1, 1])
    plan = _plan(wl, dev)
    xd = _t(wl.x, dev)
    sa, sb, sal = _t(wl.sched_a.T.copy(), dev), _t(wl.sched_b.T.copy(), dev), \
        _t(wl.sched_alpha.T.copy(), dev)

    def tick(p, t):
        return p.process_block(xd[:, t * L:(t + 1) * L].contiguous(), None, sa[t], sb[t],
                               sal[t]).clone()

    for t in range(12):
        tick(plan, t)
    buf = torch.empty(plan.state_bytes(), dtype=torch.uint8,
                      device=dev if where == "cuda" else "cpu")
    if where == "cpu":
        buf = buf.pin_memory()
    plan.get_state(buf)
    first = torch.cat([tick(plan, t) for t in range(12, 20)], dim=1).cpu().numpy()
    plan.set_state(buf)
    again = torch.cat([tick(plan, t) for t in range(12, 20)], dim=1).cpu().numpy()
    np.testing.assert_array_equal(again, first)
    other = _plan(wl, dev)
    other.set_state(buf)
    moved = torch.cat([tick(other, t) for t in range(12, 20)], dim=1).cpu().numpy()
    np.testing.assert_array_equal(moved, first)
    plan.check()
    from paper_2310_00319_gb300 import Plan
    wrong = Plan(L, wl.M + 1, n_in=2, n_out=3, out_to_in=[0, 1, 1], n_slots=3, device=dev)
    with pytest.raises(TvolapError):
        wrong.set_state(buf)
