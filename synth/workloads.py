"""Seeded synthetic inputs shaped like the paper's auralization workloads.

All values are drawn in FP64 with ``numpy.random.default_rng(seed)`` and
rounded to FP32; both the CUDA path and the FP64 oracle consume the same FP32
arrays. The paper's own measurements use KEMAR HRIRs and Salford-BBC BRIRs
(Section 3, Section 4); exponentially decaying Gaussian impulse responses of
comparable length and reverberation time stand in for them.

A ``Workload`` carries
  x           [n_in, N] float32 input channels
  irs         [n_slots, ir_len] float32 stored impulse responses
  sched_a/b   [n_out, n_blocks] int32 slot indices per output block
  sched_alpha [n_out, n_blocks] float32 mix weight: block filter is
              (1 - alpha) * irs[a] + alpha * irs[b]
  out_to_in   [n_out] int32 input channel feeding each output
Schedules are indexed by t = l + 1 (block l = -1 is entry 0) and have
n_blocks = floor((out_len - 1) / L) + 2 entries.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FS = 48000


@dataclass
class Workload:
    name: str
    L: int
    x: np.ndarray
    irs: np.ndarray
    sched_a: np.ndarray
    sched_b: np.ndarray
    sched_alpha: np.ndarray
    out_to_in: np.ndarray
    out_len: int
    fs: int = FS
    meta: dict = field(default_factory=dict)

    @property
    def n_in(self):
        return self.x.shape[0]

    @property
    def N(self):
        return self.x.shape[1]

    @property
    def n_out(self):
        return self.sched_a.shape[0]

    @property
    def ir_len(self):
        return self.irs.shape[1]

    @property
    def M(self):
        return max(1, -(-self.ir_len // (2 * self.L)))

    @property
    def n_blocks(self):
        return blocks_for(self.out_len, self.L)


def blocks_for(out_len: int, L: int) -> int:
    """Schedule entries covering output samples [0, out_len)."""
    return 0 if out_len <= 0 else (out_len - 1) // L + 2


def decaying_ir(rng, n: int, t60: float, fs: int = FS) -> np.ndarray:
    """Gaussian noise times a 60 dB-per-T60 exponential decay, unit energy."""
    k = np.arange(n, dtype=np.float64)
    h = rng.standard_normal(n) * 10.0 ** (-3.0 * k / (fs * t60))
    return h / np.sqrt(np.sum(h * h))


def white(rng, shape, sigma=0.1):
    return sigma * rng.standard_normal(shape)


def pinkish(rng, shape, sigma=0.1, a=0.95):
    """White Gaussian noise through the one-pole lowpass v[n] = a v[n-1] + e[n]."""
    from scipy.signal import lfilter
    e = white(rng, shape, sigma)
    return lfilter([1.0], [1.0, -a], e, axis=-1)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def cyclic_schedule(n_blocks: int, n_filters: int, period: int, first_slot: int = 0):
    """Slot (t // period) mod n_filters at schedule entry t."""
    t = np.arange(n_blocks)
    return first_slot + (t // period) % n_filters


def random_walk_schedule(rng, n_blocks: int, n_filters: int, step_sigma: float,
                         first_slot: int = 0):
    """Position p <- (p + N(0, step^2)) mod n_filters per block; the block mixes
    filters floor(p) and floor(p)+1 (cyclic) with weight frac(p) on the second."""
    p0 = rng.uniform(0, n_filters)
    steps = rng.normal(0.0, step_sigma, size=n_blocks)
    steps[0] = 0.0
    p = np.mod(p0 + np.cumsum(steps), n_filters)
    alpha = (p - np.floor(p)).astype(np.float32)
    a = np.floor(p).astype(np.int64) % n_filters
    b = (a + 1) % n_filters
    return first_slot + a, first_slot + b, alpha


# ----------------------------------------------------------------------------- configs
def plain_mono(seed=1, N=96000, L=128, ir_len=4096, n_ir=4, t60=0.3, period=16):
    """Plain TVOLAP, mono, fs 48 kHz, L=128: Gaussian white noise (sigma 0.1),
    4 decaying IRs of 4096 taps (T60 0.3 s), filter switched every 16 blocks in
    cyclic order."""
    rng = np.random.default_rng(seed)
    x = white(rng, (1, N))
    irs = np.stack([decaying_ir(rng, ir_len, t60) for _ in range(n_ir)])
    out_len = N
    nb = blocks_for(out_len, L)
    a = cyclic_schedule(nb, n_ir, period)[None, :]
    return Workload("plain_mono_L128", L, _f32(x), _f32(irs), _i32(a), _i32(a),
                    np.zeros(a.shape, np.float32), _i32([0]), out_len,
                    meta=dict(seed=seed, t60=t60, period=period))


def plain_at_scale(seed=2, n_ch=64, N=480000, L=256, ir_len=48000, n_ir=8,
                   step_sigma=0.05):
    """Plain TVOLAP at scale: n_ch independent channels, L=256, pink-ish noise
    (one-pole lowpass a=0.95 of white noise, sigma 0.1), per channel n_ir
    decaying IRs (T60 ~ U(0.2, 1.0) s) and a new filter every block from a
    random walk between them with linear interpolation of taps.

    Stored IR i of channel c sits in slot c * n_ir + i."""
    rng = np.random.default_rng(seed)
    x = pinkish(rng, (n_ch, N))
    irs = np.empty((n_ch * n_ir, ir_len), dtype=np.float64)
    for s in range(n_ch * n_ir):
        irs[s] = decaying_ir(rng, ir_len, rng.uniform(0.2, 1.0))
    out_len = N
    nb = blocks_for(out_len, L)
    A = np.empty((n_ch, nb), np.int64)
    B = np.empty((n_ch, nb), np.int64)
    AL = np.empty((n_ch, nb), np.float32)
    for c in range(n_ch):
        A[c], B[c], AL[c] = random_walk_schedule(rng, nb, n_ir, step_sigma, c * n_ir)
    return Workload(f"plain_at_scale_{n_ch}ch_L{L}", L, _f32(x), _f32(irs), _i32(A), _i32(B),
                    _f32(AL), _i32(np.arange(n_ch)), out_len,
                    meta=dict(seed=seed, n_ir=n_ir, step_sigma=step_sigma))


def random_case(seed, L, ir_len, N, n_in=1, n_out=None, n_slots=3, out_len=None,
                interp=True, out_to_in=None):
    """Small random time-variant case for parity and pin tests: white input,
    random slots per block, random mix weights (or none)."""
    rng = np.random.default_rng(seed)
    n_out = n_in if n_out is None else n_out
    x = white(rng, (n_in, N), 1.0)
    irs = rng.standard_normal((n_slots, ir_len)) / np.sqrt(max(ir_len, 1))
    out_len = N if out_len is None else out_len
    nb = blocks_for(out_len, L)
    a = rng.integers(0, n_slots, size=(n_out, nb))
    b = rng.integers(0, n_slots, size=(n_out, nb)) if interp else a.copy()
    al = rng.uniform(0, 1, size=(n_out, nb)) if interp else np.zeros((n_out, nb))
    if out_to_in is None:
        out_to_in = np.arange(n_out) % n_in
    return Workload(f"random_s{seed}_L{L}", L, _f32(x), _f32(irs), _i32(a), _i32(b),
                    _f32(al), _i32(out_to_in), out_len, meta=dict(seed=seed))


def differentiable(seed=4, n_ch=16, N=240000, L=256, ir_len=24000, scale=None, with_target=False):
    """Trainable-spectra workload: n_ch channels of white noise (sigma 0.1),
    L = 256, partitions of a 24000-tap response (M = 47), per-block parameter
    spectra P [n_ch, n_blocks, M, 2L] drawn complex Gaussian with standard
    deviation `scale` (default 1/sqrt(M) per component), and the weights r of
    a linear loss sum(r * y) (dL/dy = r). With with_target, also a target bank
    of 4 decaying responses of ir_len taps switched every 32 blocks."""
    rng = np.random.default_rng(seed)
    M = max(1, -(-ir_len // (2 * L)))
    nb = blocks_for(N, L)
    x = white(rng, (n_ch, N))
    s = (1.0 / np.sqrt(M)) if scale is None else scale
    P = np.empty((n_ch, nb, M, 2 * L), dtype=np.complex64)
    for c in range(n_ch):
        re = rng.standard_normal((nb, M, 2 * L), dtype=np.float32)
        im = rng.standard_normal((nb, M, 2 * L), dtype=np.float32)
        P[c] = (re + 1j * im) * np.float32(s)
    r = rng.standard_normal((n_ch, N)).astype(np.float32)
    out = dict(x=_f32(x), P=P, r=_f32(r), L=L, M=M, n_blocks=nb)
    if with_target:
        irs = np.stack([decaying_ir(rng, ir_len, rng.uniform(0.2, 1.0)) for _ in range(4)])
        out["target_irs"] = _f32(irs)
        out["target_sched"] = _i32(np.tile(cyclic_schedule(nb, 4, 32)[None, :], (n_ch, 1)))
    return out


@dataclass
class Source:
    """One independent source of a batched workload: hop L, input x [N],
    stored responses irs [n_ir, ir_len], per-block filter index sched [n_blocks]
    (into irs), output length out_len."""
    L: int
    x: np.ndarray
    irs: np.ndarray
    sched: np.ndarray
    out_len: int

    @property
    def M(self):
        return max(1, -(-self.irs.shape[1] // (2 * self.L)))


def batched_uneven(seed=3, n_src=512, hops=(64, 128, 256, 512), ir_min=4800, ir_max=96000,
                   sec_min=1.0, sec_max=20.0, n_ir=4, switch_max=8, fs=FS):
    """Batched uneven sources: hop L uniform over `hops`, impulse-response
    length log-uniform in [ir_min, ir_max] (decaying Gaussian, T60 = length / 3
    samples-to-seconds), signal length uniform in [sec_min, sec_max] s of white
    noise (sigma 0.1), n_ir stored responses per source and a switch to the next
    one every k ~ U{1..switch_max} blocks."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_src):
        L = int(rng.choice(hops))
        ir_len = int(round(np.exp(rng.uniform(np.log(ir_min), np.log(ir_max)))))
        N = int(round(rng.uniform(sec_min, sec_max) * fs))
        t60 = ir_len / (3.0 * fs)
        irs = np.stack([decaying_ir(rng, ir_len, t60, fs) for _ in range(n_ir)])
        x = white(rng, N)
        nb = blocks_for(N, L)
        k = int(rng.integers(1, switch_max + 1))
        sched = cyclic_schedule(nb, n_ir, k)
        out.append(Source(L, _f32(x), _f32(irs), _i32(sched), N))
    return out


# ----------------------------------------------------------------------------- serving
def binaural_pair(rng, n: int, t60: float, rho: float = 0.5, fs: int = FS) -> np.ndarray:
    """[2, n]: left = Gaussian noise g_l, right = rho g_l + sqrt(1 - rho^2) g_r
    (correlation rho), both times the same 60 dB-per-T60 decay, each scaled to
    unit energy."""
    k = np.arange(n, dtype=np.float64)
    env = 10.0 ** (-3.0 * k / (fs * t60))
    gl = rng.standard_normal(n)
    gr = rho * gl + np.sqrt(1.0 - rho * rho) * rng.standard_normal(n)
    out = np.stack([gl * env, gr * env])
    return out / np.sqrt(np.sum(out * out, axis=1, keepdims=True))


def serving_bank(rng, ir_len: int, n_pairs: int = 36, fs: int = FS) -> np.ndarray:
    """[n_pairs, 2, ir_len] float32 binaural pairs, T60 = ir_len / 3 samples
    expressed in seconds (as for the batched sources)."""
    t60 = ir_len / (3.0 * fs)
    return _f32(np.stack([binaural_pair(rng, ir_len, t60, fs=fs) for _ in range(n_pairs)]))


def head_walk(rng, n_blocks: int, n_pairs: int = 36) -> np.ndarray:
    """Pair index per block: a start uniform over the pairs, then steps of -1, 0
    or +1 (equally likely) modulo n_pairs."""
    p0 = int(rng.integers(0, n_pairs))
    steps = rng.integers(-1, 2, size=n_blocks)
    steps[0] = 0
    return _i32(np.mod(p0 + np.cumsum(steps), n_pairs))


@dataclass
class ServeStream:
    """One stream of the serving workload: hop L, binaural bank irs
    [n_pairs, 2, ir_len], input x [n_blocks * L] and pair index per block."""
    L: int
    irs: np.ndarray
    x: np.ndarray
    sel: np.ndarray

    @property
    def n_blocks(self):
        return self.sel.shape[0]


def serving_streams(seed: int, n: int, hops=(16, 32, 64), ir_min=200, ir_max=1500,
                    n_pairs=6, blocks=(20, 60)) -> list:
    """Small streams for parity checks: hop uniform over `hops`, response length
    uniform in [ir_min, ir_max], white input (sigma 0.1) of a block count
    uniform in `blocks`, head walk over n_pairs pairs."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        L = int(rng.choice(hops))
        ir_len = int(rng.integers(ir_min, ir_max + 1))
        nb = int(rng.integers(blocks[0], blocks[1] + 1))
        irs = serving_bank(rng, ir_len, n_pairs)
        out.append(ServeStream(L, irs, _f32(white(rng, nb * L)), head_walk(rng, nb, n_pairs)))
    return out


def serving_arrivals(seed=5, duration_s=13.0, rate=50.0, life_min=2.0, life_max=30.0,
                     prefill=1000, base_hop=64, fs=FS):
    """Arrival and departure times, in base ticks of base_hop samples, of the
    serving workload: `prefill` streams present at tick 0, then Poisson arrivals
    at `rate` per second; every lifetime uniform in [life_min, life_max] s.
    Returns an int64 array [n, 2] of (arrive, leave) sorted by arrival."""
    rng = np.random.default_rng(seed)
    tick_s = base_hop / fs
    n_new = int(rng.poisson(rate * duration_s))
    t_new = np.sort(rng.uniform(0.0, duration_s, n_new))
    arrive = np.concatenate([np.zeros(prefill), t_new])
    life = rng.uniform(life_min, life_max, arrive.shape[0])
    ev = np.stack([np.floor(arrive / tick_s), np.floor((arrive + life) / tick_s)], axis=1)
    return ev.astype(np.int64)
