"""GPU parity of two-level non-uniform partitions (tvolap_nu_*) against the
FP64 oracle's definition (oracle.tvolap_nonuniform: head at hop La, tail at
hop ratio * La added D samples later), offline and streaming.

Tolerance as in test_parity_gpu.py: relative L2 <= 1e-5 and max-abs <= 1e-4
times the reference peak, per output.
"""
import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_parity_gpu import _assert_close, _dev, _t  # noqa: E402


def _nu(dev, La, Ma, ratio, Mb, n_in, n_out, out_to_in, irs):
    from paper_2310_00319_gb300.nonuniform import NonUniform
    h = NonUniform(La, Ma, ratio, Mb, n_in=n_in, n_out=n_out, out_to_in=out_to_in,
                   n_slots=irs.shape[0], device=dev)
    h.load_bank(0, _t(irs, dev))
    return h


def _case(seed, La, Ma, ratio, Mb, n_in=2, n_out=3, out_to_in=(0, 1, 1), N=None, n_slots=4,
          ir_len=None):
    D, Lb = 2 * La * Ma, ratio * La
    ir_len = ir_len or D + 2 * Lb * Mb - 7
    N = N or 20 * Lb + La // 2
    wl = W.random_case(seed, L=La, ir_len=ir_len, N=N, n_in=n_in, n_out=n_out, n_slots=n_slots,
                       out_to_in=list(out_to_in))
    return wl


def _ref(wl, La, Ma, ratio, Mb):
    return oracle.tvolap_nonuniform(wl.x, wl.irs, La, Ma, ratio, Mb, wl.sched_a, wl.sched_b,
                                    wl.sched_alpha, out_len=wl.out_len, out_to_in=wl.out_to_in)


@pytest.mark.parametrize("La,Ma,ratio,Mb", [(32, 4, 4, 6), (16, 7, 8, 3), (64, 2, 2, 9),
                                            (128, 3, 4, 2)])
def test_offline_matches_oracle(La, Ma, ratio, Mb):
    dev = _dev()
    wl = _case(100 + La, La, Ma, ratio, Mb)
    h = _nu(dev, La, Ma, ratio, Mb, wl.n_in, wl.n_out, wl.out_to_in, wl.irs)
    y = h.process_signal(_t(wl.x, dev), _t(wl.sched_a, dev), _t(wl.sched_b, dev),
                         _t(wl.sched_alpha, dev), out_len=wl.out_len)
    h.check()
    _assert_close(y.cpu().numpy(), _ref(wl, La, Ma, ratio, Mb), "non-uniform")


def test_fixed_long_response_is_its_convolution():
    """One fixed 2-second-class response split over the two levels equals its
    full convolution (numpy)."""
    dev = _dev()
    La, Ma, ratio, Mb = 64, 15, 16, 5
    D, Lb = 2 * La * Ma, ratio * La
    rng = np.random.default_rng(7)
    N = 30000
    x = rng.standard_normal((1, N)).astype(np.float32)
    h = (rng.standard_normal((1, D + 2 * Lb * Mb)) * np.exp(-np.arange(D + 2 * Lb * Mb) / 3000.0)
         ).astype(np.float32)
    nu = _nu(dev, La, Ma, ratio, Mb, 1, 1, None, h)
    nb = oracle.n_out_blocks(N, La)
    y = nu.process_signal(_t(x, dev), _t(np.zeros((1, nb), np.int32), dev), out_len=N)
    nu.check()
    ref = np.convolve(x[0].astype(np.float64), h[0].astype(np.float64))[:N]
    _assert_close(y.cpu().numpy(), ref[None], "fixed response")


@pytest.mark.parametrize("La,Ma,ratio,Mb", [(32, 4, 4, 6), (16, 3, 4, 5)])
def test_streaming_equals_offline_delayed_by_La(La, Ma, ratio, Mb):
    """process_block one head hop at a time, with this tick's selection,
    gives the offline result delayed by exactly La samples."""
    dev = _dev()
    wl = _case(200 + La, La, Ma, ratio, Mb, n_slots=3)
    h = _nu(dev, La, Ma, ratio, Mb, wl.n_in, wl.n_out, wl.out_to_in, wl.irs)
    n_ticks = wl.n_blocks
    N = wl.x.shape[1]
    xpad = np.zeros((wl.n_in, n_ticks * La), np.float32)
    xpad[:, :N] = wl.x
    xd = _t(xpad, dev)
    sa, sb, sal = _t(wl.sched_a.T.copy(), dev), _t(wl.sched_b.T.copy(), dev), \
        _t(wl.sched_alpha.T.copy(), dev)
    outs = [h.process_block(xd[:, t * La:(t + 1) * La].contiguous(), None, sa[t], sb[t],
                            sal[t]).clone() for t in range(n_ticks)]
    h.check()
    y = torch.cat(outs, dim=1).cpu().numpy()
    ref = _ref(wl, La, Ma, ratio, Mb)
    assert np.max(np.abs(y[:, :La])) <= 1e-5 * np.max(np.abs(ref))
    n = min(N, y.shape[1] - La)
    _assert_close(y[:, La:La + n], ref[:, :n], "non-uniform stream")


def test_create_rejects_bad_levels():
    from paper_2310_00319_gb300 import TvolapError
    from paper_2310_00319_gb300.nonuniform import NonUniform
    dev = _dev()
    for args in [(32, 4, 3, 2), (32, 2, 4, 2), (32, 4, 1, 2), (256, 8, 8, 2)]:
        with pytest.raises(TvolapError):
            NonUniform(*args, device=dev)
