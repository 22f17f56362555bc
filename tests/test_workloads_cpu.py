"""The seeded input generators follow the recipe the design notes state for
the paper's workloads: decaying Gaussian responses (60 dB per T60, unit
energy), pink-ish input (one-pole lowpass, a = 0.95), the random-walk and
cyclic schedules, the batched-source distributions, binaural pairs of
correlation 0.5, the head walk and the serving arrivals. The statistical
checks are seeded (deterministic) and their tolerances are at least three
standard errors wide."""
import inspect

import numpy as np

from synth import workloads as W


def test_decaying_ir_has_unit_energy_and_60_db_per_t60():
    rng = np.random.default_rng(0)
    fs, t60 = 48000, 0.5
    h = W.decaying_ir(rng, 48000, t60, fs)
    assert abs(np.sum(h * h) - 1.0) < 1e-12
    win, gap = 4000, 12000                     # energy of two windows 0.25 s apart
    e0 = np.sum(h[:win] ** 2)
    e1 = np.sum(h[gap:gap + win] ** 2)
    want = 10.0 ** (-6.0 * gap / (fs * t60))   # power falls 60 dB per T60
    assert abs(e1 / e0 / want - 1.0) < 0.15


def test_pinkish_input_is_the_stated_one_pole_lowpass():
    rng = np.random.default_rng(1)
    v = W.pinkish(rng, (1, 400000), sigma=0.1, a=0.95)[0]
    rho1 = np.dot(v[1:], v[:-1]) / np.dot(v, v)
    assert abs(rho1 - 0.95) < 0.01                        # AR(1): lag-1 correlation = a
    assert abs(np.var(v) / (0.01 / (1 - 0.95 ** 2)) - 1) < 0.1


def test_random_walk_schedule():
    rng = np.random.default_rng(2)
    a, b, al = W.random_walk_schedule(rng, 20000, 8, 0.05, first_slot=16)
    assert a.min() >= 16 and a.max() <= 23
    np.testing.assert_array_equal(b - 16, (a - 16 + 1) % 8)
    assert al.dtype == np.float32 and al.min() >= 0 and al.max() < 1
    p = (a - 16) + al.astype(np.float64)
    d = np.diff(p)
    d = (d + 4) % 8 - 4                                   # unwrap the modulo
    assert abs(np.std(d) - 0.05) < 0.005


def test_cyclic_schedule_and_plain_configs():
    np.testing.assert_array_equal(W.cyclic_schedule(10, 4, 3), [0, 0, 0, 1, 1, 1, 2, 2, 2, 3])
    mono = W.plain_mono()
    assert mono.x.shape == (1, 96000) and mono.irs.shape == (4, 4096) and mono.L == 128
    assert mono.M == 16
    assert abs(np.std(mono.x) - 0.1) < 0.002
    sig = inspect.signature(W.plain_at_scale).parameters
    assert (sig["n_ch"].default, sig["N"].default, sig["L"].default, sig["ir_len"].default,
            sig["n_ir"].default) == (64, 480000, 256, 48000, 8)
    small = W.plain_at_scale(n_ch=3, N=4000, ir_len=600)
    for c in range(3):                                    # channel c uses slots 8c .. 8c + 7
        assert small.sched_a[c].min() >= 8 * c and small.sched_a[c].max() <= 8 * c + 7


def test_batched_sources_follow_their_distributions():
    S = W.batched_uneven(seed=3, n_src=300, sec_min=0.01, sec_max=0.02)
    hops = np.array([s.L for s in S])
    assert set(hops) == {64, 128, 256, 512}
    lens = np.array([s.irs.shape[1] for s in S])
    assert lens.min() >= 4800 and lens.max() <= 96000
    logs = np.log(lens)                                   # log-uniform: uniform log length
    assert abs(np.mean(logs) - 0.5 * (np.log(4800) + np.log(96000))) < 0.15
    for s in S:
        assert s.irs.shape[0] == 4
        assert 480 <= s.x.shape[0] <= 960
        runs = np.diff(np.flatnonzero(np.diff(s.sched)))  # blocks between switches
        if runs.size:
            assert runs.min() == runs.max() and 1 <= runs[0] <= 8
        d = np.diff(s.sched)
        assert np.all(d[d != 0] % 4 == 1)                 # cyclic: the next response


def test_binaural_pairs_and_head_walk():
    rng = np.random.default_rng(4)
    pair = W.binaural_pair(rng, 200000, 10.0)             # long T60: nearly flat envelope
    assert np.allclose(np.sum(pair ** 2, axis=1), 1.0)
    r = np.dot(pair[0], pair[1]) / np.sqrt(np.dot(pair[0], pair[0]) * np.dot(pair[1], pair[1]))
    assert abs(r - 0.5) < 0.01
    w = W.head_walk(rng, 5000, 36)
    assert w.min() >= 0 and w.max() < 36
    steps = (np.diff(w.astype(np.int64)) + 1) % 36 - 1
    assert set(np.unique(steps)) == {-1, 0, 1}


def test_serving_arrivals():
    ev = W.serving_arrivals(seed=5)
    assert np.sum(ev[:, 0] == 0) >= 1000                  # the prefill is present at tick 0
    tick_s = 64 / 48000
    new = ev[1000:]
    assert abs(new.shape[0] - 50 * 13.0) < 4 * np.sqrt(50 * 13.0)   # Poisson count
    life = (ev[:, 1] - ev[:, 0]) * tick_s
    assert life.min() >= 2.0 - 2 * tick_s and life.max() <= 30.0 + tick_s
    assert np.all(np.diff(ev[:, 0]) >= 0)
