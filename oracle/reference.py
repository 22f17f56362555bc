"""FP64 CPU oracle for time-variant overlap-add in partitions (TVOLAP).

TEST INFRASTRUCTURE ONLY. Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this module. It
shares no code, table or helper with the CUDA library and never imports it.

Functions and the passages of arxiv 2310.00319 they follow:

* ``hann_half``            -- Section 2, Eq. "w_hann", read with the factor 1/2
                              (the 50%-overlapped periodic windows then sum to 1).
* ``tvolap_direct``        -- Section 2, Eqs. 1-12 restated in the time domain
                              (C, FP64, OpenMP; ``tvolap_direct.c``).
* ``tvolap_samples``       -- the same arithmetic for a list of (channel, n).
* ``tvolap_bruteforce``    -- the same definition as a pure-Python per-sample
                              tap sum; a second, independent implementation for
                              tiny cases.
* ``tvolap_spectral``      -- Eqs. 1-12 taken literally in the frequency domain:
                              4L-point DFTs (Eqs. 5-6), every-second-spectrum MAC
                              (Eq. 7), inverse DFT (Eq. 8), two-step overlap-add
                              (Eqs. 9-12). ``grid='regular'`` is the paper's DFT
                              grid; ``grid='halfbin'`` evaluates the same spectra
                              on the frequencies (k + 1/2) / 4L.
* ``block_spectra``        -- Eqs. 1, 3, 5 for chosen blocks (input spectra X).
* ``partition_spectra``    -- Eqs. 2, 4, 6 (transfer-function partitions H).
* ``halfbin_dft``          -- the definition of the half-bin DFT, by summation.
* ``params_forward``       -- Eqs. 5, 7, 8-12 with free per-block partition
                              spectra P[t, m, k] in place of transforms of
                              impulse responses (the trainable model).
* ``params_grad``          -- the hand-derived adjoint of ``params_forward``
                              (gradients w.r.t. P and x, PyTorch's convention
                              dL/dRe + i dL/dIm for complex parameters); pinned
                              against FP64 finite differences in
                              tests/test_oracle_grad_pins.py.
* ``params_grad_sampled``  -- chosen entries of the same gradients, each from
                              the definitions on its own (full-size checks).
* ``tvolap_nonuniform``    -- two-level non-uniform partitions: TVOLAP of the
                              first D = 2 La Ma taps at hop La plus TVOLAP of
                              the remaining taps at hop ratio * La, added D
                              samples later (the tail's schedule entry t is
                              the head's entry (t + 1) ratio - 1); each level is
                              ``tvolap_direct``.
* ``mixdown``              -- the sum of the outputs routed to each mix output
                              (Section 2's c channels summed per ear for the
                              binaural rendering of Section 5; by linearity of
                              Eq. 8 and Eqs. 9-12 the library sums spectra).

Readings of the paper that these functions take (each is pinned by a test in
tests/test_oracle_pins.py):

* the Hann window carries a factor 1/2;
* Eq. 2's partition offset is m * 2L (the printed l * 2L is a typo);
* Eq. 9's predecessor is block l - 2, the previous block of the same parity;
* the filter current at OUTPUT block l multiplies every partition (Eq. 7);
* the first block is l = -1 (L zeros before the signal), schedules are indexed
  by t = l + 1;
* a filter that is a mix (1 - alpha) * ir[a] + alpha * ir[b] is that mix of taps.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tvolap_direct.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libtvolap_oracle.so")
_lib = None
_lock = threading.Lock()


# --------------------------------------------------------------------------- build
def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lp = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_tvolap_direct.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, dp,
                ctypes.c_int, ctypes.c_int, dp,
                ctypes.c_int, ip, ctypes.c_int, ip, ip, dp,
                ctypes.c_int64, dp]
            lib.oracle_tvolap_direct.restype = None
            lib.oracle_tvolap_samples.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, dp,
                ctypes.c_int, ctypes.c_int, dp,
                ctypes.c_int, ip, ctypes.c_int, ip, ip, dp,
                ctypes.c_int, ip, lp, dp]
            lib.oracle_tvolap_samples.restype = None
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the C oracle uses."""
    return int(_load().oracle_num_threads())


# --------------------------------------------------------------------------- helpers
def n_partitions(ir_len: int, L: int) -> int:
    """M = ceil(N_IR / 2L): partitions of length 2L (Section 2, Eq. 2)."""
    return max(1, -(-int(ir_len) // (2 * int(L))))


def n_out_blocks(out_len: int, L: int) -> int:
    """Schedule entries needed for output samples [0, out_len): t = l + 1 for
    l = -1 .. floor((out_len - 1) / L)."""
    if out_len <= 0:
        return 0
    return (int(out_len) - 1) // int(L) + 2


def hann_half(L: int) -> np.ndarray:
    """w(i) = (1 - cos(2 pi i / 2L)) / 2, 0 <= i < 2L (Section 2, Eq. "w_hann";
    the factor 1/2 is the reading under which the hop-L windows sum to one)."""
    i = np.arange(2 * L, dtype=np.float64)
    return 0.5 * (1.0 - np.cos(2.0 * np.pi * i / (2 * L)))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _sched(n_out, n_blocks, sched_a, sched_b, sched_alpha):
    a = _i32(sched_a).reshape(n_out, -1)
    b = a if sched_b is None else _i32(sched_b).reshape(n_out, -1)
    al = (np.zeros(a.shape) if sched_alpha is None
          else _f64(np.asarray(sched_alpha, dtype=np.float64)).reshape(n_out, -1))
    if a.shape[1] < n_blocks or b.shape[1] < n_blocks or al.shape[1] < n_blocks:
        raise ValueError(f"schedule has {a.shape[1]} entries per channel, need {n_blocks}")
    return (np.ascontiguousarray(a[:, :n_blocks]), np.ascontiguousarray(b[:, :n_blocks]),
            np.ascontiguousarray(al[:, :n_blocks]))


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


# --------------------------------------------------------------------------- direct (C)
def tvolap_direct(x, irs, L, sched_a, sched_b=None, sched_alpha=None, out_len=None,
                  M=None, out_to_in=None):
    """TVOLAP output by the time-domain restatement of Eqs. 1-12 (FP64, C).

    x          [n_in, N] (or [N]) input, any float dtype (upcast to FP64)
    irs        [n_slots, ir_len] stored impulse responses
    sched_a/b  [n_out, n_blocks] slot indices; block l = t - 1 uses
               (1 - alpha) * irs[a] + alpha * irs[b]  (sched_b defaults to a)
    sched_alpha [n_out, n_blocks] mixing weights (default 0)
    out_len    output samples per channel (default N)
    M          partitions (default ceil(ir_len / 2L))
    out_to_in  [n_out] input channel of each output (default identity)
    returns    [n_out, out_len] FP64
    """
    lib = _load()
    x = _f64(x)
    squeeze = x.ndim == 1
    x = x.reshape(-1, x.shape[-1])
    n_in, N = x.shape
    irs = _f64(irs).reshape(-1, np.asarray(irs).shape[-1])
    n_slots, ir_len = irs.shape
    if M is None:
        M = n_partitions(ir_len, L)
    if ir_len > 2 * L * M:
        raise ValueError("ir_len exceeds 2*L*M")
    if out_len is None:
        out_len = N
    sa = _i32(sched_a)
    n_out = 1 if sa.ndim == 1 else sa.shape[0]
    if out_to_in is None:
        out_to_in = np.arange(n_out) if n_in == n_out else np.zeros(n_out)
    o2i = _i32(out_to_in)
    nb = n_out_blocks(out_len, L)
    a, b, al = _sched(n_out, nb, sched_a, sched_b, sched_alpha)
    if a.size and (a.min() < 0 or a.max() >= n_slots or b.min() < 0 or b.max() >= n_slots):
        raise ValueError("schedule slot out of range")
    y = np.zeros((n_out, int(out_len)), dtype=np.float64)
    lib.oracle_tvolap_direct(int(L), int(M), int(n_in), int(N), _ptr(x, ctypes.c_double),
                             int(n_slots), int(ir_len), _ptr(irs, ctypes.c_double),
                             int(n_out), _ptr(o2i, ctypes.c_int), int(nb),
                             _ptr(a, ctypes.c_int), _ptr(b, ctypes.c_int),
                             _ptr(al, ctypes.c_double), int(out_len), _ptr(y, ctypes.c_double))
    return y[0] if (squeeze and n_out == 1) else y


def tvolap_nonuniform(x, irs, La, Ma, ratio, Mb, sched_a, sched_b=None, sched_alpha=None,
                      out_len=None, out_to_in=None):
    """Two-level non-uniform partitioned TVOLAP (FP64).

    Head: taps [0, D), D = 2 La Ma, TVOLAP at hop La with Ma partitions and the
    given schedules (per head block). Tail: taps [D, D + 2 Lb Mb), Lb = ratio La,
    TVOLAP at hop Lb with Mb partitions; its schedule entry t is the head's
    entry min((t + 1) ratio - 1, last); its aligned output is added at n + D.
    A fixed response gives its full linear convolution.
    """
    irs = _f64(irs).reshape(-1, np.asarray(irs).shape[-1])
    x = _f64(x)
    N = x.reshape(-1, x.shape[-1]).shape[1]
    out_len = N if out_len is None else int(out_len)
    D, Lb = 2 * La * Ma, ratio * La
    if irs.shape[1] > D + 2 * Lb * Mb:
        raise ValueError("responses longer than D + 2 Lb Mb")
    head = np.zeros((irs.shape[0], D))
    head[:, :min(D, irs.shape[1])] = irs[:, :D]
    sa = np.atleast_2d(_i32(sched_a))
    sb = sa if sched_b is None else np.atleast_2d(_i32(sched_b))
    sal = np.zeros(sa.shape) if sched_alpha is None else np.atleast_2d(_f64(sched_alpha))
    y = tvolap_direct(x, head, La, sa, sb, sal, out_len=out_len, M=Ma, out_to_in=out_to_in)
    y = np.atleast_2d(y)
    if irs.shape[1] > D and out_len > D:
        tail = irs[:, D:]
        nb_head = n_out_blocks(out_len, La)
        tail_len = out_len - D
        idx = np.minimum((np.arange(n_out_blocks(tail_len, Lb)) + 1) * ratio - 1, nb_head - 1)
        yt = tvolap_direct(x, tail, Lb, sa[:, idx], sb[:, idx], sal[:, idx], out_len=tail_len,
                           M=Mb, out_to_in=out_to_in)
        y[:, D:] += np.atleast_2d(yt)
    return y


def mixdown(y, mix_of_out, n_mix=None):
    """Mix outputs as sums of plan outputs (FP64): row e of the result is the
    sum of the rows o of y with mix_of_out[o] == e, added in increasing o.

    y          [n_out, n] outputs (any float dtype, upcast to FP64)
    mix_of_out [n_out] mix output of each plan output, in [0, n_mix)
    n_mix      mix outputs (default max(mix_of_out) + 1)
    returns    [n_mix, n] FP64
    """
    y = _f64(y)
    m = np.asarray(mix_of_out, dtype=np.int64)
    if m.shape != (y.shape[0],):
        raise ValueError("mix_of_out must have one entry per output")
    n_mix = int(m.max()) + 1 if n_mix is None else int(n_mix)
    out = np.zeros((n_mix, y.shape[1]), np.float64)
    for o in range(y.shape[0]):
        out[m[o]] += y[o]
    return out


def tvolap_samples(x, irs, L, sched_a, sched_b, sched_alpha, out_ch, n_idx, M=None,
                   out_to_in=None, n_blocks=None):
    """y[out_ch[k], n_idx[k]] for every k, with the arithmetic of tvolap_direct.
    ``n_blocks`` is the schedule length per channel (default: its width)."""
    lib = _load()
    x = _f64(x)
    x = x.reshape(-1, x.shape[-1])
    n_in, N = x.shape
    irs = _f64(irs).reshape(-1, np.asarray(irs).shape[-1])
    n_slots, ir_len = irs.shape
    if M is None:
        M = n_partitions(ir_len, L)
    sa = _i32(sched_a)
    sa = sa.reshape(-1, sa.shape[-1])
    n_out = sa.shape[0]
    if n_blocks is None:
        n_blocks = sa.shape[1]
    a, b, al = _sched(n_out, n_blocks, sched_a, sched_b, sched_alpha)
    if out_to_in is None:
        out_to_in = np.arange(n_out) if n_in == n_out else np.zeros(n_out)
    o2i = _i32(out_to_in)
    oc = _i32(out_ch)
    ni = np.ascontiguousarray(np.asarray(n_idx, dtype=np.int64))
    out = np.zeros(oc.shape[0], dtype=np.float64)
    lib.oracle_tvolap_samples(int(L), int(M), int(n_in), int(N), _ptr(x, ctypes.c_double),
                              int(n_slots), int(ir_len), _ptr(irs, ctypes.c_double),
                              int(n_out), _ptr(o2i, ctypes.c_int), int(n_blocks),
                              _ptr(a, ctypes.c_int), _ptr(b, ctypes.c_int),
                              _ptr(al, ctypes.c_double), int(oc.shape[0]),
                              _ptr(oc, ctypes.c_int), _ptr(ni, ctypes.c_int64),
                              _ptr(out, ctypes.c_double))
    return out


# --------------------------------------------------------------------------- brute force
def tvolap_bruteforce(x, irs, L, sched_a, sched_b, sched_alpha, out_len, M=None):
    """Pure-Python per-sample tap form of the same definition (mono, tiny sizes).

    y(n) = sum_s x(s) sum_{q : 0 <= s - qL < 2L} w(s - qL) h_{q + 2*floor(d/2L)}(d),
    d = n - s, 0 <= d < 2LM: input sample s sits in input block q at window
    position s - qL; tap d lies in partition m = floor(d / 2L), so it reaches the
    output through output block l = q + 2m (Eq. 7), whose filter is used.
    """
    x = [float(v) for v in np.asarray(x, dtype=np.float64).ravel()]
    irs = np.asarray(irs, dtype=np.float64)
    irs = [[float(v) for v in row] for row in irs.reshape(-1, irs.shape[-1])]
    ir_len = len(irs[0])
    if M is None:
        M = n_partitions(ir_len, L)
    sa = [int(v) for v in np.asarray(sched_a).ravel()]
    sb = sa if sched_b is None else [int(v) for v in np.asarray(sched_b).ravel()]
    sal = ([0.0] * len(sa) if sched_alpha is None
           else [float(v) for v in np.asarray(sched_alpha, dtype=np.float64).ravel()])
    import math
    w = [0.5 * (1.0 - math.cos(2.0 * math.pi * i / (2 * L))) for i in range(2 * L)]
    N = len(x)
    y = [0.0] * out_len
    for n in range(out_len):
        acc = 0.0
        for s in range(max(0, n - 2 * L * M + 1), min(N, n + 1)):
            d = n - s
            if d >= ir_len:
                continue
            m = d // (2 * L)
            for q in range(-1, s // L + 1):
                i = s - q * L
                if not (0 <= i < 2 * L):
                    continue
                t = q + 2 * m + 1
                h = (1.0 - sal[t]) * irs[sa[t]][d] + sal[t] * irs[sb[t]][d]
                acc += x[s] * w[i] * h
        y[n] = acc
    return np.array(y)


# --------------------------------------------------------------------------- spectra
def halfbin_dft(v, n_fft):
    """sum_n v(n) exp(-j 2 pi n (k + 1/2) / n_fft), k = 0 .. n_fft-1, by direct
    summation (the definition; O(n_fft^2), for pinning small cases)."""
    v = np.asarray(v, dtype=np.complex128)
    n = np.arange(v.shape[-1])
    k = np.arange(n_fft)
    E = np.exp(-2j * np.pi * np.outer(k + 0.5, n) / n_fft)
    return v @ E.T


def _dft4l(v, grid):
    """4L-point forward transform of the last axis (length 4L, zero padded)."""
    n4 = v.shape[-1]
    if grid == "regular":
        return np.fft.fft(v, axis=-1)                     # Eq. 5 / Eq. 6
    if grid == "halfbin":
        n = np.arange(n4)
        return np.fft.fft(v * np.exp(-1j * np.pi * n / n4), axis=-1)
    raise ValueError(grid)


def _idft4l(V, grid):
    """Inverse of _dft4l, including the 1/4L of Eq. 8."""
    n4 = V.shape[-1]
    if grid == "regular":
        return np.fft.ifft(V, axis=-1)
    if grid == "halfbin":
        n = np.arange(n4)
        return np.fft.ifft(V, axis=-1) * np.exp(1j * np.pi * n / n4)
    raise ValueError(grid)


def block_spectra(x, L, blocks, grid="halfbin"):
    """X(k, l) for the listed blocks l (Eqs. 1, 3, 5): window 2L samples from
    l*L, append 2L zeros, 4L-point DFT. Returns complex [len(blocks), 4L]."""
    x = np.asarray(x, dtype=np.float64).ravel()
    N = x.shape[0]
    w = hann_half(L)
    out = np.zeros((len(blocks), 4 * L), dtype=np.float64)
    for r, l in enumerate(blocks):
        for i in range(2 * L):
            s = l * L + i
            if 0 <= s < N:
                out[r, i] = x[s] * w[i]
    return _dft4l(out, grid)


def partition_spectra(ir, L, M=None, grid="halfbin"):
    """H(k, m) (Eqs. 2, 4, 6): partition m holds taps [2mL, 2mL + 2L), then 2L
    zeros, then the 4L-point DFT. Returns complex [M, 4L]."""
    ir = np.asarray(ir, dtype=np.float64).ravel()
    if M is None:
        M = n_partitions(ir.shape[0], L)
    p = np.zeros((M, 4 * L), dtype=np.float64)
    for m in range(M):
        seg = ir[2 * m * L: 2 * m * L + 2 * L]
        p[m, :seg.shape[0]] = seg
    return _dft4l(p, grid)


def tvolap_spectral(x, irs, L, sched_a, sched_b=None, sched_alpha=None, out_len=None,
                    M=None, grid="regular", pr_lag=2):
    """Eqs. 1-12 taken literally in the frequency domain (mono, FP64, numpy FFT).

    pr_lag is the block whose right half Eq. 9 adds to the current left half;
    the paper prints l - 1, the reading taken here is l - 2 (pr_lag=2).
    """
    x = np.asarray(x, dtype=np.float64).ravel()
    N = x.shape[0]
    irs = np.asarray(irs, dtype=np.float64)
    irs = irs.reshape(-1, irs.shape[-1])
    ir_len = irs.shape[1]
    if M is None:
        M = n_partitions(ir_len, L)
    if out_len is None:
        out_len = N
    nb = n_out_blocks(out_len, L)
    sa = np.asarray(sched_a).ravel()
    sb = sa if sched_b is None else np.asarray(sched_b).ravel()
    sal = np.zeros(sa.shape) if sched_alpha is None else np.asarray(sched_alpha, np.float64).ravel()
    # input spectra X(k, l) for l = -1 .. nb-2 (Eq. 5)
    ls = list(range(-1, nb - 1))
    X = block_spectra(x, L, ls, grid)                       # row r <-> block l = r - 1
    # intermediate outputs y(n', l), length 4L (Eqs. 7, 8)
    ylist = []
    for r, l in enumerate(ls):
        t = l + 1
        h = (1.0 - sal[t]) * irs[sa[t]] + sal[t] * irs[sb[t]]
        H = partition_spectra(h, L, M, grid)
        Y = np.zeros(4 * L, dtype=np.complex128)
        for m in range(M):
            q = l - 2 * m
            if q >= -1:
                Y += H[m] * X[q + 1]
        ylist.append(np.real(_idft4l(Y, grid)))
    # two-step overlap-add (Eqs. 9-12)
    out = np.zeros(out_len + 4 * L, dtype=np.float64)
    for r, l in enumerate(ls):
        yhat = ylist[r][:2 * L].copy()                       # Eq. 10
        if r - pr_lag >= 0:
            yhat += ylist[r - pr_lag][2 * L:]                # Eq. 9
        for i in range(2 * L):                               # Eq. 12
            n = l * L + i
            if 0 <= n < out_len:
                out[n] += yhat[i]
    return out[:out_len]


# --------------------------------------------------------------------------- spectral parameters
# A model whose filter partitions are free per-block spectra P[t, m, k] (k < 2L,
# half-bin grid) instead of transforms of impulse responses: Eqs. 5, 7, 8-12 with
# H_l(k, m) = P[t = l + 1, m, k]. A real block's spectrum on this grid is
# determined by its 2L lower bins (X(4L-1-k) = conj X(k)); a parameter spectrum
# is read the same way, so the inverse transform of each output block is real.

def _halfbin_full(V):
    """Extend lower-half bins [.., 2L] to the conjugate-symmetric 4L bins."""
    return np.concatenate([V, np.conj(V[..., ::-1])], axis=-1)


def params_forward(x, Pspec, L, out_len=None, pr_lag=2):
    """y = TVOLAP of one channel x with per-block spectra Pspec[t, m, k]
    (t = l + 1 < n_blocks, m < M, k < 2L), FP64, literal Eqs. 5, 7, 8-12."""
    x = np.asarray(x, np.float64).ravel()
    N = x.shape[0]
    Pspec = np.asarray(Pspec, np.complex128)
    nb, M, P2 = Pspec.shape
    assert P2 == 2 * L
    if out_len is None:
        out_len = N
    assert nb >= n_out_blocks(out_len, L)
    X = block_spectra(x, L, list(range(-1, nb - 1)), grid="halfbin")[:, :2 * L]
    out = np.zeros(out_len + 4 * L)
    for t in range(nb):
        Y = np.zeros(2 * L, np.complex128)
        for m in range(M):
            if t - 2 * m >= 0:
                Y += Pspec[t, m] * X[t - 2 * m]
        yb = np.real(_idft4l(_halfbin_full(Y), "halfbin"))       # Eq. 8, length 4L
        l = t - 1
        for i in range(4 * L):                                  # Eqs. 9-12: add at l*L
            n = l * L + i
            if 0 <= n < out_len:
                out[n] += yb[i]
    return out[:out_len]


def params_grad(x, Pspec, L, g):
    """Hand adjoint of params_forward for a real loss with dL/dy = g:
    returns (dP, dx) with dP = dL/dRe P + i dL/dIm P.

      G(t) = (1/2L) sum_{n<4L} g(l*L + n) e^{-i pi n (2k+1) / 4L}     (adjoint of Eq. 8)
      dP(t, m) = G(t) conj X(t - 2m)                                  (adjoint of Eq. 7)
      dX(q) = sum_m G(q + 2m) conj P(q + 2m, m)
      dx(l*L + n) += w(n) Re sum_{k<2L} dX_q(k) e^{+i pi n (2k+1) / 4L}, n < 2L  (Eqs. 1, 5)
    """
    x = np.asarray(x, np.float64).ravel()
    g = np.asarray(g, np.float64).ravel()
    N, out_len = x.shape[0], g.shape[0]
    Pspec = np.asarray(Pspec, np.complex128)
    nb, M, _ = Pspec.shape
    X = block_spectra(x, L, list(range(-1, nb - 1)), grid="halfbin")[:, :2 * L]
    n4 = np.arange(4 * L)
    k2 = np.arange(2 * L)
    E = np.exp(-1j * np.pi * np.outer(n4, 2 * k2 + 1) / (4 * L))      # [4L, 2L]
    G = np.zeros((nb, 2 * L), np.complex128)
    for t in range(nb):
        seg = np.zeros(4 * L)
        for i in range(4 * L):
            n = (t - 1) * L + i
            if 0 <= n < out_len:
                seg[i] = g[n]
        G[t] = (seg @ E) / (2 * L)
    dP = np.zeros_like(Pspec)
    dX = np.zeros((nb, 2 * L), np.complex128)
    for t in range(nb):
        for m in range(M):
            q = t - 2 * m
            if q >= 0:
                dP[t, m] = G[t] * np.conj(X[q])
                dX[q] += G[t] * np.conj(Pspec[t, m])
    w = hann_half(L)
    dx = np.zeros(N)
    Einv = np.exp(1j * np.pi * np.outer(np.arange(2 * L), 2 * k2 + 1) / (4 * L))   # [2L, 2L]
    for q in range(nb):
        dxw = np.real(Einv @ dX[q])
        l = q - 1
        for i in range(2 * L):
            s = l * L + i
            if 0 <= s < N:
                dx[s] += w[i] * dxw[i]
    return dP, dx


def params_grad_sampled(x, Pspec, L, g, dP_idx, dx_idx):
    """Selected entries of params_grad, each computed on its own from the same
    definitions: dP[t, m, k] for the (t, m, k) triples in dP_idx and
    dx[s] for s in dx_idx, for one channel (x [N], Pspec [nb, M, 2L], g [out_len])."""
    x = np.asarray(x, np.float64).ravel()
    g = np.asarray(g, np.float64).ravel()
    N, out_len = x.shape[0], g.shape[0]
    nb, M = Pspec.shape[0], Pspec.shape[1]
    k2 = np.arange(2 * L)
    n4 = np.arange(4 * L)
    E = np.exp(-1j * np.pi * np.outer(n4, 2 * k2 + 1) / (4 * L))
    cacheG, cacheX = {}, {}

    def G(t):
        if t not in cacheG:
            seg = np.zeros(4 * L)
            for i in range(4 * L):
                n = (t - 1) * L + i
                if 0 <= n < out_len:
                    seg[i] = g[n]
            cacheG[t] = (seg @ E) / (2 * L)
        return cacheG[t]

    def X(q):
        if q not in cacheX:
            cacheX[q] = block_spectra(x, L, [q - 1], grid="halfbin")[0, :2 * L]
        return cacheX[q]

    dP = np.array([G(t)[k] * np.conj(X(t - 2 * m)[k]) if t - 2 * m >= 0 else 0.0
                   for (t, m, k) in dP_idx], dtype=np.complex128)
    w = hann_half(L)
    dx = np.zeros(len(dx_idx))
    for j, s in enumerate(dx_idx):
        acc = 0.0
        for q in (s // L, s // L + 1):
            n = s - (q - 1) * L
            if not (0 <= n < 2 * L) or q >= nb:
                continue
            dXq = np.zeros(2 * L, np.complex128)
            for m in range(M):
                t = q + 2 * m
                if t < nb:
                    dXq += G(t) * np.conj(np.asarray(Pspec[t, m], np.complex128))
            acc += w[n] * np.real(np.sum(dXq * np.exp(1j * np.pi * n * (2 * k2 + 1) / (4 * L))))
        dx[j] = acc
    return dP, dx
