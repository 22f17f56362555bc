"""Pins for the oracle's spectral-parameter model and its hand adjoint.

The forward is pinned to the impulse-response model (parameters that are the
spectra of 2L-tap partitions reproduce tvolap_direct) and the adjoint to FP64
central finite differences of the forward (the loss sum(r * y) is linear, so
the differences are exact up to rounding). CPU only.
"""
import numpy as np
import pytest

import oracle


def _case(seed, L=4, M=3, N=40, out_len=None):
    rng = np.random.default_rng(seed)
    out_len = N if out_len is None else out_len
    nb = oracle.n_out_blocks(out_len, L)
    x = rng.standard_normal(N)
    P = rng.standard_normal((nb, M, 2 * L)) + 1j * rng.standard_normal((nb, M, 2 * L))
    r = rng.standard_normal(out_len)
    return x, P, r, out_len


def test_params_of_ir_partitions_equal_direct_model():
    """Per-block spectra that are the half-bin transforms of 2L-tap partitions
    of a time-variant filter reproduce the time-domain oracle."""
    rng = np.random.default_rng(3)
    L, N = 8, 200
    irs = rng.standard_normal((3, 40))
    M = oracle.n_partitions(40, L)
    nb = oracle.n_out_blocks(N, L)
    sa = rng.integers(0, 3, nb)
    x = rng.standard_normal(N)
    H = np.stack([oracle.partition_spectra(irs[s], L, M, grid="halfbin")[:, :2 * L]
                  for s in range(3)])
    P = H[sa]                                              # [nb, M, 2L]
    y = oracle.params_forward(x, P, L)
    ref = oracle.tvolap_direct(x, irs, L, sa[None, :])
    assert np.max(np.abs(y - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("seed,L,M,N,tail", [(1, 4, 3, 40, 0), (2, 2, 4, 25, 9), (3, 8, 2, 70, 5)])
def test_adjoint_matches_finite_differences(seed, L, M, N, tail):
    x, P, r, out_len = _case(seed, L, M, N, N + tail)
    dP, dx = oracle.params_grad(x, P, L, r)

    def loss(xx, PP):
        return float(np.dot(r, oracle.params_forward(xx, PP, L, out_len)))

    rng = np.random.default_rng(seed + 100)
    h = 1e-6
    for _ in range(12):
        t, m, k = rng.integers(0, P.shape[0]), rng.integers(0, M), rng.integers(0, 2 * L)
        for unit, comp in ((1.0, np.real), (1j, np.imag)):
            Pp, Pm = P.copy(), P.copy()
            Pp[t, m, k] += unit * h
            Pm[t, m, k] -= unit * h
            fd = (loss(x, Pp) - loss(x, Pm)) / (2 * h)
            assert abs(fd - comp(dP[t, m, k])) < 1e-7 * max(1.0, abs(fd)), (t, m, k)
    for s in rng.integers(0, N, 12):
        xp, xm = x.copy(), x.copy()
        xp[s] += h
        xm[s] -= h
        fd = (loss(xp, P) - loss(xm, P)) / (2 * h)
        assert abs(fd - dx[s]) < 1e-7 * max(1.0, abs(fd)), s


def test_adjoint_planted_mistake_fails():
    """Planted mistake: the gradient without the conjugate on X is not the
    derivative (finite differences disagree)."""
    x, P, r, out_len = _case(5)
    dP, _ = oracle.params_grad(x, P, 4, r)
    X = oracle.block_spectra(x, 4, list(range(-1, P.shape[0] - 1)), grid="halfbin")[:, :8]
    G = dP[2, 0] / np.conj(X[2])
    wrong = G * X[2]
    h = 1e-6
    Pp, Pm = P.copy(), P.copy()
    Pp[2, 0, 1] += h
    Pm[2, 0, 1] -= h
    fd = (np.dot(r, oracle.params_forward(x, Pp, 4, out_len))
          - np.dot(r, oracle.params_forward(x, Pm, 4, out_len))) / (2 * h)
    assert abs(fd - dP[2, 0, 1].real) < 1e-7
    assert abs(fd - wrong[1].real) > 1e-3


def test_sampled_gradient_entries_equal_full_adjoint():
    x, P, r, out_len = _case(9, L=4, M=3, N=50, out_len=57)
    dP, dx = oracle.params_grad(x, P, 4, r)
    rng = np.random.default_rng(1)
    idx = [(int(rng.integers(0, P.shape[0])), int(rng.integers(0, 3)), int(rng.integers(0, 8)))
           for _ in range(20)]
    sidx = [int(v) for v in rng.integers(0, 50, 15)] + [0, 49]
    sP, sx = oracle.params_grad_sampled(x, P, 4, r, idx, sidx)
    for j, (t, m, k) in enumerate(idx):
        assert abs(sP[j] - dP[t, m, k]) < 1e-12
    assert np.max(np.abs(sx - dx[sidx])) < 1e-12
