"""Pins for the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a textbook
routine (numpy.convolve), a closed form (the polarity switch of Section 3,
Fig. 3), a number the paper prints (Tables 1-2, tests/golden/), an
independent implementation (pure-Python tap sum, numpy WOLA), or a planted
mistake that must be caught. CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from synth import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _const_sched(nb, slot=0):
    return np.full((1, nb), slot, np.int32)


# --------------------------------------------------------------------- time-invariant
@pytest.mark.parametrize("L,ir_len,N", [(4, 24, 50), (8, 13, 61), (16, 96, 333), (32, 64, 257),
                                        (3, 11, 40)])
def test_time_invariant_equals_linear_convolution(L, ir_len, N):
    """A filter that never changes must give plain linear convolution: the
    hop-L Hann windows sum to one and the 4L padding prevents wrap-around
    (Section 2, Eqs. 1-4)."""
    rng = np.random.default_rng(L * 1000 + ir_len)
    x = rng.standard_normal(N)
    h = rng.standard_normal(ir_len)
    full = N + ir_len - 1
    nb = oracle.n_out_blocks(full, L)
    y = oracle.tvolap_direct(x, h[None], L, _const_sched(nb), out_len=full)
    ref = np.convolve(x, h)
    assert _rel(y, ref) < 1e-13
    assert np.max(np.abs(y - ref)) < 1e-12 * np.max(np.abs(ref))


def test_interpolated_filter_is_tap_mix():
    """A constant mix (1 - a) h0 + a h1 equals convolution with the mixed taps."""
    rng = np.random.default_rng(5)
    L, N = 8, 150
    irs = rng.standard_normal((2, 40))
    alpha = 0.3125
    nb = oracle.n_out_blocks(N, L)
    x = rng.standard_normal(N)
    y = oracle.tvolap_direct(x, irs, L, np.zeros((1, nb)), np.ones((1, nb)),
                             np.full((1, nb), alpha))
    ref = np.convolve(x, (1 - alpha) * irs[0] + alpha * irs[1])[:N]
    assert _rel(y, ref) < 1e-13


@pytest.mark.parametrize("d", [0, 1, 7, 16, 45])
def test_delta_ir_returns_delayed_input(d):
    """h = delta at tap d returns x delayed by d samples."""
    L, N = 8, 200
    rng = np.random.default_rng(d)
    x = rng.standard_normal(N)
    h = np.zeros(48)
    h[d] = 1.0
    nb = oracle.n_out_blocks(N, L)
    y = oracle.tvolap_direct(x, h[None], L, _const_sched(nb))
    ref = np.concatenate([np.zeros(d), x])[:N]
    assert np.max(np.abs(y - ref)) < 1e-14


def test_linearity_in_x_and_h():
    """Linear in the input and in the stored impulse responses, for a
    time-variant schedule with mixing."""
    wl = W.random_case(11, L=8, ir_len=37, N=123, n_slots=3)
    x1, irs1 = wl.x.astype(np.float64), wl.irs.astype(np.float64)
    rng = np.random.default_rng(12)
    x2 = rng.standard_normal(x1.shape)
    irs2 = rng.standard_normal(irs1.shape)
    args = (wl.L, wl.sched_a, wl.sched_b, wl.sched_alpha)
    y11 = oracle.tvolap_direct(x1, irs1, *args)
    y21 = oracle.tvolap_direct(x2, irs1, *args)
    y12 = oracle.tvolap_direct(x1, irs2, *args)
    ya = oracle.tvolap_direct(2.5 * x1 - 0.75 * x2, irs1, *args)
    yb = oracle.tvolap_direct(x1, 1.5 * irs1 + 2.0 * irs2, *args)
    assert _rel(ya, 2.5 * y11 - 0.75 * y21) < 1e-13
    assert _rel(yb, 1.5 * y11 + 2.0 * y12) < 1e-13


def test_channels_are_independent():
    """c channels run side by side (Section 2): each output equals the mono
    result of its own input channel, and routing one input to two outputs
    gives both outputs from that input."""
    wl = W.random_case(21, L=4, ir_len=20, N=70, n_in=2, n_out=3, n_slots=4,
                       out_to_in=[1, 0, 1])
    y = oracle.tvolap_direct(wl.x, wl.irs, wl.L, wl.sched_a, wl.sched_b, wl.sched_alpha,
                             out_to_in=wl.out_to_in)
    for o in range(3):
        c = wl.out_to_in[o]
        ym = oracle.tvolap_direct(wl.x[c], wl.irs, wl.L, wl.sched_a[o:o + 1],
                                  wl.sched_b[o:o + 1], wl.sched_alpha[o:o + 1])
        np.testing.assert_array_equal(y[o], ym)


def test_mixdown_of_paths_equals_one_path_with_summed_taps():
    """Mixdown (the sum of outputs per mix output): two paths reading the same
    input through fixed responses h1 and h2 and mixed together equal one path
    with the response h1 + h2 (linearity of convolution), and paths with h and
    -h cancel exactly; each is checked against numpy.convolve as well."""
    rng = np.random.default_rng(31)
    L, N, ir_len = 8, 150, 40
    x = rng.standard_normal(N)
    h1, h2 = rng.standard_normal(ir_len), rng.standard_normal(ir_len)
    irs = np.stack([h1, h2, -h1])
    nb = oracle.n_out_blocks(N, L)
    sched = np.array([[0] * nb, [1] * nb, [2] * nb], np.int32)
    y = oracle.tvolap_direct(x, irs, L, sched, out_to_in=[0, 0, 0])
    mixed = oracle.mixdown(y, [0, 0, 1], n_mix=3)
    ref = np.convolve(x, h1 + h2)[:N]
    assert _rel(mixed[0], ref) < 1e-12
    assert _rel(mixed[1], -np.convolve(x, h1)[:N]) < 1e-12
    assert not mixed[2].any()                                   # no member: silent
    # h and -h routed to one mix output cancel to rounding
    cancel = oracle.mixdown(y[[0, 2]], [0, 0])
    assert np.max(np.abs(cancel)) <= 1e-12 * np.max(np.abs(y[0]))


def test_nonuniform_fixed_response_is_full_convolution():
    """Two-level non-uniform partitions with one fixed response: head (small
    hop) plus tail (hop ratio * La, added D samples later) equal numpy's full
    linear convolution; a response no longer than D leaves the tail silent."""
    rng = np.random.default_rng(33)
    La, Ma, ratio, Mb = 4, 3, 4, 2
    D, Lb = 2 * La * Ma, ratio * La
    N = 300
    x = rng.standard_normal(N)
    h = rng.standard_normal(D + 2 * Lb * Mb - 5)
    nb = oracle.n_out_blocks(N, La)
    y = oracle.tvolap_nonuniform(x, h[None], La, Ma, ratio, Mb, _const_sched(nb), out_len=N)
    assert _rel(y[0], np.convolve(x, h)[:N]) < 1e-12
    short = h[:D - 3]
    ys = oracle.tvolap_nonuniform(x, short[None], La, Ma, ratio, Mb, _const_sched(nb), out_len=N)
    yp = oracle.tvolap_direct(x, short[None], La, _const_sched(nb), out_len=N, M=Ma)
    np.testing.assert_array_equal(ys, np.atleast_2d(yp))


def test_nonuniform_tail_takes_the_head_entry_of_its_hop():
    """The filter switches from response 0 to 1 at head block ts; an input
    that starts at sample (ts + 1) La meets response 1 in every block of both
    levels only if the tail's entry t maps to head entry (t + 1) ratio - 1 or
    later: the output is then exactly x * h1. A tail reading the entry at the
    start of its hop instead would still use response 0 and is caught."""
    rng = np.random.default_rng(34)
    La, Ma, ratio, Mb = 4, 3, 4, 2
    D, Lb = 2 * La * Ma, ratio * La
    N = 400
    h = rng.standard_normal((2, D + 2 * Lb * Mb))
    ts = 37
    x = np.zeros(N)
    S = (ts + 1) * La
    x[S:] = rng.standard_normal(N - S)
    nb = oracle.n_out_blocks(N, La)
    sched = np.zeros((1, nb), np.int32)
    sched[0, ts:] = 1
    y = oracle.tvolap_nonuniform(x, h, La, Ma, ratio, Mb, sched, out_len=N)
    assert _rel(y[0], np.convolve(x, h[1])[:N]) < 1e-12
    # planted: the tail reading the head entry t * ratio (start of its hop)
    tail_len = N - D
    idx = np.arange(oracle.n_out_blocks(tail_len, Lb)) * ratio
    yt = oracle.tvolap_direct(x, h[:, D:], Lb, sched[:, np.minimum(idx, nb - 1)],
                              out_len=tail_len, M=Mb)
    yh = oracle.tvolap_direct(x, h[:, :D], La, sched, out_len=N, M=Ma)
    wrong = np.atleast_2d(yh).copy()
    wrong[:, D:] += np.atleast_2d(yt)
    assert _rel(wrong[0], np.convolve(x, h[1])[:N]) > 1e-3


# --------------------------------------------------------------------- closed form, Fig. 3
@pytest.mark.parametrize("L,M,d,A", [(8, 4, 3, 10), (8, 4, 21, 12), (16, 2, 40, 9), (4, 3, 17, 15)])
def test_polarity_switch_closed_form(L, M, d, A):
    """Section 3, Fig. 3: a run of ones through a single tap whose sign flips
    from + to - at output block A. With the 1/2-Hann and the output-time filter
    convention the output is +1 before n0 = A*L + (d mod 2L), exactly
    cos(pi (n - n0) / L) on [n0, n0 + L) and -1 afterwards."""
    N = (A + 8) * L + d
    x = np.ones(N)
    ir = np.zeros((2, 2 * L * M))
    ir[0, d] = 1.0
    ir[1, d] = -1.0
    nb = oracle.n_out_blocks(N, L)
    t = np.arange(nb)
    sched = (t - 1 >= A).astype(np.int32)[None, :]        # block l = t - 1
    y = oracle.tvolap_direct(x, ir, L, sched)
    n0 = A * L + (d % (2 * L))
    n = np.arange(N)
    expect = np.where(n < n0, 1.0, -1.0)
    sl = (n >= n0) & (n < n0 + L)
    expect[sl] = np.cos(np.pi * (n[sl] - n0) / L)
    expect[n < d] = 0.0                                   # before the first input reaches tap d
    assert np.max(np.abs(y - expect)) < 1e-13


def test_switching_latency_matches_table1():
    """Table 1 prints a TVOLAP switching latency of 256 samples for N_IR = 2048,
    2L = 512, M = 4, i.e. N_IR / (2M) = L (Section 3). The oracle's transition
    from +1 to -1 lasts exactly that many samples."""
    g = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))["table1"]
    L, M = g["L"], g["M"]
    assert g["N_IR"] == 2 * L * M
    d, A = 5, 12
    N = (A + 6) * L
    ir = np.zeros((2, g["N_IR"]))
    ir[0, d], ir[1, d] = 1.0, -1.0
    nb = oracle.n_out_blocks(N, L)
    sched = (np.arange(nb) - 1 >= A).astype(np.int32)[None, :]
    y = oracle.tvolap_direct(np.ones(N), ir, L, sched)
    settled = np.abs(np.abs(y) - 1.0) < 1e-12
    moving = np.flatnonzero(~settled[d:]) + d
    # the first transition sample is exactly +1 (cos 0); the last is the one before -1
    transition = (moving.max() - moving.min() + 2)
    assert transition == g["tvolap"]["switching_latency"] == g["N_IR"] // (2 * M)


# --------------------------------------------------------------------- independent implementations
@pytest.mark.parametrize("L,ir_len,N,tail", [(1, 3, 9, 0), (2, 7, 14, 5), (4, 24, 30, 24),
                                             (2, 12, 11, 12), (4, 5, 21, 3)])
def test_bruteforce_matches_direct(L, ir_len, N, tail):
    """Pure-Python per-sample tap sum (tiny sizes) equals the C oracle, with a
    random slot pair and mix weight at every block."""
    wl = W.random_case(100 + L * 7 + ir_len, L=L, ir_len=ir_len, N=N, n_slots=3,
                       out_len=N + tail)
    y = oracle.tvolap_direct(wl.x, wl.irs, L, wl.sched_a, wl.sched_b, wl.sched_alpha,
                             out_len=wl.out_len)
    yb = oracle.tvolap_bruteforce(wl.x[0], wl.irs, L, wl.sched_a[0], wl.sched_b[0],
                                  wl.sched_alpha[0], wl.out_len)
    assert np.max(np.abs(y - yb)) < 1e-13 * max(1.0, np.max(np.abs(yb)))


def _wola_hann_rect(x, irs, L, sched_a, out_len):
    """Independent M = 1 reference: Hann analysis window, per-block linear
    convolution with that block's 2L-tap filter, rectangular synthesis,
    overlap-add at hop L (the WOLA reading of Section 3)."""
    N = x.shape[0]
    w = 0.5 - 0.5 * np.cos(np.pi * np.arange(2 * L) / L)
    y = np.zeros(out_len + 8 * L)
    xp = np.concatenate([np.zeros(L), x, np.zeros(4 * L)])
    for t in range(len(sched_a)):
        l = t - 1
        seg = xp[l * L + L: l * L + 3 * L] * w
        c = np.convolve(seg, irs[sched_a[t]])
        start = l * L
        for i, v in enumerate(c):
            if 0 <= start + i < out_len:
                y[start + i] += v
    return y[:out_len]


def test_single_partition_is_wola_hann_rect():
    """Section 3: with one partition TVOLAP is WOLA with a Hann analysis and a
    rectangular synthesis window."""
    rng = np.random.default_rng(31)
    L, N = 8, 300
    irs = rng.standard_normal((3, 2 * L))
    nb = oracle.n_out_blocks(N, L)
    sa = rng.integers(0, 3, nb)
    x = np.sin(np.arange(N) * 0.37) + 0.1 * rng.standard_normal(N)
    y = oracle.tvolap_direct(x, irs, L, sa[None, :])
    ref = _wola_hann_rect(x, irs, L, sa, N)
    assert np.max(np.abs(y - ref)) < 1e-13


# --------------------------------------------------------------------- spectral forms
@pytest.mark.parametrize("grid", ["regular", "halfbin"])
def test_spectral_literal_equals_direct(grid):
    """Eqs. 5-12 evaluated with 4L-point DFTs (regular grid as printed, and the
    half-bin grid) give the time-domain result, for a time-variant schedule."""
    wl = W.random_case(41, L=8, ir_len=45, N=170, n_slots=3, out_len=170 + 30)
    y = oracle.tvolap_direct(wl.x, wl.irs, wl.L, wl.sched_a, wl.sched_b, wl.sched_alpha,
                             out_len=wl.out_len)[0]
    ys = oracle.tvolap_spectral(wl.x[0], wl.irs, wl.L, wl.sched_a[0], wl.sched_b[0],
                                wl.sched_alpha[0], out_len=wl.out_len, grid=grid)
    assert _rel(ys, y) < 1e-12


def test_eq9_printed_predecessor_breaks_time_invariance():
    """Planted mistake: Eq. 9 as printed (block l - 1) does not reproduce
    linear convolution, the same-parity reading (l - 2) does."""
    rng = np.random.default_rng(3)
    L, N = 8, 200
    x, h = rng.standard_normal(N), rng.standard_normal(40)
    nb = oracle.n_out_blocks(N, L)
    ref = np.convolve(x, h)[:N]
    good = oracle.tvolap_spectral(x, h[None], L, np.zeros(nb, np.int32), pr_lag=2)
    bad = oracle.tvolap_spectral(x, h[None], L, np.zeros(nb, np.int32), pr_lag=1)
    assert _rel(good, ref) < 1e-12
    assert _rel(bad, ref) > 0.1


def test_literal_window_amplitude_doubles_output():
    """Planted mistake: the window exactly as printed, 1 - cos(...), makes the
    hop-L windows sum to 2, so a time-invariant filter returns twice the
    convolution; the 1/2-Hann returns it exactly."""
    L = 16
    w_half = oracle.hann_half(L)
    w_printed = 1.0 - np.cos(2 * np.pi * np.arange(2 * L) / (2 * L))
    # hop-L sums over one period
    s_half = w_half[:L] + w_half[L:]
    s_printed = w_printed[:L] + w_printed[L:]
    assert np.max(np.abs(s_half - 1.0)) < 1e-15
    assert np.max(np.abs(s_printed - 2.0)) < 1e-15


def test_halfbin_spectra_match_definition():
    """The half-bin spectra (sum_n v(n) e^{-j 2 pi n (k + 1/2) / 4L}) of the
    oracle equal the definition summed directly; they are conjugate-symmetric
    about the middle, so 2L complex values describe a real block; and their
    product is the spectrum of the LINEAR convolution (no wrap within 4L)."""
    rng = np.random.default_rng(8)
    L = 8
    x = rng.standard_normal(80)
    blocks = [-1, 0, 3, 8]
    X = oracle.block_spectra(x, L, blocks, grid="halfbin")
    w = oracle.hann_half(L)
    for r, l in enumerate(blocks):
        v = np.zeros(4 * L)
        for i in range(2 * L):
            if 0 <= l * L + i < 80:
                v[i] = x[l * L + i] * w[i]
        Xd = oracle.halfbin_dft(v, 4 * L)
        assert np.max(np.abs(X[r] - Xd)) < 1e-12
        k = np.arange(2 * L)
        assert np.max(np.abs(X[r][4 * L - 1 - k] - np.conj(X[r][k]))) < 1e-12
    h = rng.standard_normal(2 * L)
    H = oracle.partition_spectra(h, L, 1, grid="halfbin")[0]
    Hd = oracle.halfbin_dft(np.concatenate([h, np.zeros(2 * L)]), 4 * L)
    assert np.max(np.abs(H - Hd)) < 1e-12
    seg = x[:2 * L] * w
    prod = oracle.halfbin_dft(np.concatenate([seg, np.zeros(2 * L)]), 4 * L) * Hd
    n = np.arange(4 * L)
    back = np.fft.ifft(prod) * np.exp(1j * np.pi * n / (4 * L))
    full = np.convolve(seg, h)
    assert np.max(np.abs(back[:4 * L - 1] - full)) < 1e-12
    assert abs(back[4 * L - 1]) < 1e-12


def test_output_time_convention_differs_from_input_time():
    """Planted mistake: filtering each input block with ITS OWN filter (instead
    of the filter current at the output block, Eq. 7) moves the Fig. 3
    transition from A*L + (d mod 2L) to A*L + d; the oracle's transition sits at
    the former."""
    L, M, d, A = 8, 4, 37, 10
    N = (A + 10) * L
    ir = np.zeros((2, 2 * L * M))
    ir[0, d], ir[1, d] = 1.0, -1.0
    nb = oracle.n_out_blocks(N, L)
    sched = (np.arange(nb) - 1 >= A).astype(np.int32)[None, :]
    y = oracle.tvolap_direct(np.ones(N), ir, L, sched)
    first_change = int(np.flatnonzero(np.abs(y[d:] - 1.0) > 1e-12)[0]) + d
    assert first_change == A * L + (d % (2 * L)) + 1
    assert first_change != A * L + d + 1


# --------------------------------------------------------------------- sampled form
def test_samples_match_full():
    wl = W.random_case(51, L=16, ir_len=100, N=400, n_in=2, n_out=3, n_slots=4,
                       out_to_in=[0, 1, 1], out_len=450)
    y = oracle.tvolap_direct(wl.x, wl.irs, wl.L, wl.sched_a, wl.sched_b, wl.sched_alpha,
                             out_len=wl.out_len, out_to_in=wl.out_to_in)
    rng = np.random.default_rng(0)
    oc = rng.integers(0, 3, 64)
    ni = rng.integers(0, 450, 64)
    ys = oracle.tvolap_samples(wl.x, wl.irs, wl.L, wl.sched_a, wl.sched_b, wl.sched_alpha,
                               oc, ni, out_to_in=wl.out_to_in)
    np.testing.assert_array_equal(ys, y[oc, ni])


def test_partition_count():
    assert oracle.n_partitions(4096, 128) == 16       # plain mono workload
    assert oracle.n_partitions(48000, 256) == 94      # ceil(48000 / 512)
    assert oracle.n_partitions(2048, 256) == 4        # Table 1
    assert oracle.n_partitions(1, 256) == 1
    assert math.isclose(oracle.hann_half(4)[4], 1.0)
