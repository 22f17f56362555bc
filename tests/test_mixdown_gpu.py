"""GPU parity of the frequency-domain mixdown (several outputs summed per mix
output before one inverse transform per mix output) against the FP64 oracle.

Tolerance as in test_parity_gpu.py: relative L2 error <= 1e-5 and max-abs
error <= 1e-4 times the reference peak, per mix output.
"""
import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_parity_gpu import _assert_close, _dev, _plan, _run_signal, _t  # noqa: E402


def _binaural(seed, S, L, ir_len, N, n_slots=6, out_len=None):
    """S sources, two ears: plan output o = 2s + e reads source s through its
    own time-variant schedule; ear e mixes outputs e, e + 2, e + 4, ..."""
    wl = W.random_case(seed, L=L, ir_len=ir_len, N=N, n_in=S, n_out=2 * S, n_slots=n_slots,
                       out_len=out_len, out_to_in=[o // 2 for o in range(2 * S)])
    return wl, [o % 2 for o in range(2 * S)]


def _mix_ref(wl, mix):
    ref = oracle.tvolap_direct(wl.x, wl.irs, wl.L, wl.sched_a, wl.sched_b, wl.sched_alpha,
                               out_len=wl.out_len, out_to_in=wl.out_to_in)
    return oracle.mixdown(ref, mix)


@pytest.mark.parametrize("S,L,ir_len,N", [(3, 64, 1000, 9000), (5, 256, 9000, 30000),
                                          (2, 16, 200, 1500), (4, 512, 20000, 40000)])
def test_process_signal_mix_matches_oracle(S, L, ir_len, N):
    """Ear e's output is the sum of its paths' TVOLAP outputs (oracle), here
    formed in the frequency domain before one inverse transform per ear."""
    dev = _dev()
    wl, mix = _binaural(40 + S, S, L, ir_len, N, out_len=N + L // 2)
    plan = _plan(wl, dev)
    plan.set_mix(mix)
    y = plan.process_signal_mix(_t(wl.x, dev), _t(wl.sched_a, dev), _t(wl.sched_b, dev),
                                _t(wl.sched_alpha, dev), out_len=wl.out_len)
    plan.check()
    assert tuple(y.shape) == (2, wl.out_len)
    _assert_close(y.cpu().numpy(), _mix_ref(wl, mix), "mixdown")


def test_single_member_mix_equals_plain_outputs_bitwise():
    """A mix output with one member copies its spectrum exactly, so the
    identity map gives the plain outputs bit for bit."""
    dev = _dev()
    wl = W.random_case(50, L=128, ir_len=3000, N=12000, n_in=2, n_out=3, n_slots=4,
                       out_to_in=[0, 1, 1])
    plan = _plan(wl, dev)
    y_plain = _run_signal(wl, dev, plan)
    plan.set_mix([0, 1, 2])
    y_mix = plan.process_signal_mix(_t(wl.x, dev), _t(wl.sched_a, dev), _t(wl.sched_b, dev),
                                    _t(wl.sched_alpha, dev), out_len=wl.out_len).cpu().numpy()
    np.testing.assert_array_equal(y_mix, y_plain)


def test_mix_stage_sums_in_output_order():
    """tvolap_mix: each mix output is the FP32 sum of its members' spectra in
    increasing output order (bitwise), an empty mix output is zero."""
    dev = _dev()
    from paper_2310_00319_gb300 import Plan
    plan = Plan(64, 4, n_in=1, n_out=5, out_to_in=[0] * 5, n_slots=1, device=dev)
    mix = [2, 0, 2, 0, 2]
    plan.set_mix(mix, n_mix=4)
    rng = np.random.default_rng(5)
    Y = (rng.standard_normal((5, 7, 128)) + 1j * rng.standard_normal((5, 7, 128))).astype(np.complex64)
    got = plan.mix(_t(Y, dev)).cpu().numpy()
    want = np.zeros((4, 7, 128), np.complex64)
    for o in range(5):
        want[mix[o]] = want[mix[o]] + Y[o]
    np.testing.assert_array_equal(got, want)


def test_streaming_mix_equals_offline_mix_delayed_by_L():
    """process_block_mix, one hop at a time with this tick's selection, equals
    the offline mixdown delayed by exactly L samples."""
    dev = _dev()
    L, S = 128, 3
    N = 40 * L + L // 2
    wl, mix = _binaural(60, S, L, 2000, N, n_slots=3)
    plan = _plan(wl, dev)
    plan.set_mix(mix)
    n_ticks = wl.n_blocks
    xpad = np.zeros((S, n_ticks * L), np.float32)
    xpad[:, :N] = wl.x
    xd = _t(xpad, dev)
    sa, sb, sal = _t(wl.sched_a.T.copy(), dev), _t(wl.sched_b.T.copy(), dev), \
        _t(wl.sched_alpha.T.copy(), dev)
    outs = [plan.process_block_mix(xd[:, t * L:(t + 1) * L].contiguous(), None, sa[t], sb[t],
                                   sal[t]).clone() for t in range(n_ticks)]
    plan.check()
    y = torch.cat(outs, dim=1).cpu().numpy()
    ref = _mix_ref(wl, mix)
    assert np.max(np.abs(y[:, :L])) <= 1e-5 * np.max(np.abs(ref))
    _assert_close(y[:, L:L + N], ref[:, :min(N, y.shape[1] - L)], "streaming mixdown")


def test_set_mix_rejects_invalid_maps():
    from paper_2310_00319_gb300 import TvolapError
    dev = _dev()
    wl, mix = _binaural(70, 2, 64, 300, 2000)
    plan = _plan(wl, dev)
    for bad, n in [([0, 1, 2, 0], 2), ([0, -1, 0, 1], 2), ([0, 1, 0, 1], 5)]:
        with pytest.raises(TvolapError):
            plan.set_mix(bad, n_mix=n)
    with pytest.raises(TvolapError):                           # no mixdown defined
        plan.process_signal_mix(_t(wl.x, dev), _t(wl.sched_a, dev))
    plan.set_mix(mix)
    plan.set_mix(None)
    with pytest.raises(TvolapError):
        plan.mix(torch.zeros((4, 3, 128), dtype=torch.complex64, device=dev))
