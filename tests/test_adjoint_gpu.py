"""GPU parity of the differentiable model (free per-block partition spectra):
forward against oracle.params_forward, gradients against oracle.params_grad
(itself pinned to FP64 finite differences), segment recomputation, the
autograd Function, and the full-size workload on sampled gradient entries.

Tolerances: forward rel-L2 <= 1e-5 and max-abs <= 1e-4 x peak; gradients rel
1e-3 (relative L2 over the checked entries, and max-abs <= 1e-3 x peak).
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


def _rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)), \
        float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


def _small(seed=11, C=2, L=32, ir_len=300, N=2500):
    d = W.differentiable(seed=seed, n_ch=C, N=N, L=L, ir_len=ir_len)
    return d


def _plan(d, dev):
    from paper_2310_00319_gb300 import Plan
    C = d["x"].shape[0]
    return Plan(d["L"], d["M"], n_in=C, n_out=C, n_slots=1, device=dev)


@pytest.mark.parametrize("segment", [None, 7])
def test_params_forward_matches_oracle(segment):
    dev = _dev()
    from paper_2310_00319_gb300.autograd import spectral_tvolap
    d = _small()
    plan = _plan(d, dev)
    x = torch.from_numpy(d["x"]).to(dev)
    P = torch.from_numpy(d["P"]).to(dev)
    with torch.no_grad():
        y = spectral_tvolap(x, P, plan, fwd_segment=segment).cpu().numpy()
    for c in range(d["x"].shape[0]):
        ref = oracle.params_forward(d["x"][c], d["P"][c], d["L"])
        rel, mx = _rel(y[c], ref)
        assert rel <= 1e-5 and mx <= 1e-4, (c, rel, mx)


@pytest.mark.parametrize("segment", [None, 5])
def test_params_gradients_match_oracle(segment):
    """Linear loss sum(r * y): dL/dy = r exactly, so the GPU gradients are
    compared with the oracle's adjoint for the same g."""
    dev = _dev()
    from paper_2310_00319_gb300.autograd import spectral_tvolap
    d = _small(seed=12)
    plan = _plan(d, dev)
    x = torch.from_numpy(d["x"]).to(dev).requires_grad_(True)
    P = torch.from_numpy(d["P"]).to(dev).requires_grad_(True)
    r = torch.from_numpy(d["r"]).to(dev)
    y = spectral_tvolap(x, P, plan, segment=segment)
    (y * r).sum().backward()
    for c in range(d["x"].shape[0]):
        dP, dx = oracle.params_grad(d["x"][c], d["P"][c], d["L"], d["r"][c])
        relP, mxP = _rel(P.grad[c].cpu().numpy(), dP)
        relx, mxx = _rel(x.grad[c].cpu().numpy(), dx)
        assert relP <= 1e-3 and mxP <= 1e-3, (c, relP, mxP)
        assert relx <= 1e-3 and mxx <= 1e-3, (c, relx, mxx)


def test_segments_give_identical_results():
    dev = _dev()
    from paper_2310_00319_gb300.autograd import spectral_tvolap
    d = _small(seed=13, N=4000)
    plan = _plan(d, dev)
    outs = []
    for seg in (None, 4, 13):
        x = torch.from_numpy(d["x"]).to(dev).requires_grad_(True)
        P = torch.from_numpy(d["P"]).to(dev).requires_grad_(True)
        y = spectral_tvolap(x, P, plan, segment=seg, fwd_segment=seg)
        (y * torch.from_numpy(d["r"]).to(dev)).sum().backward()
        outs.append((y.detach().cpu().numpy(), x.grad.cpu().numpy(), P.grad.cpu().numpy()))
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            np.testing.assert_array_equal(a, b)


def test_mse_training_step_against_oracle():
    """MSE against a target made by the oracle from a hidden time-variant bank;
    the oracle's gradient uses its own forward output."""
    dev = _dev()
    from paper_2310_00319_gb300.autograd import spectral_tvolap
    d = W.differentiable(seed=14, n_ch=2, N=2000, L=32, ir_len=200, with_target=True)
    L, C = d["L"], 2
    target = oracle.tvolap_direct(d["x"], d["target_irs"], L, d["target_sched"],
                                  out_to_in=[0, 1])
    plan = _plan(d, dev)
    x = torch.from_numpy(d["x"]).to(dev)
    P = torch.from_numpy(d["P"]).to(dev).requires_grad_(True)
    tgt = torch.from_numpy(target.astype(np.float32)).to(dev)
    y = spectral_tvolap(x, P, plan)
    loss = ((y - tgt) ** 2).mean()
    loss.backward()
    n = target.size
    for c in range(C):
        y_or = oracle.params_forward(d["x"][c], d["P"][c], L)
        g = 2.0 * (y_or - target[c].astype(np.float32).astype(np.float64)) / n
        dP, _ = oracle.params_grad(d["x"][c], d["P"][c], L, g)
        rel, mx = _rel(P.grad[c].cpu().numpy(), dP)
        assert rel <= 1e-3 and mx <= 1e-3, (c, rel, mx)


def test_full_size_sampled_gradients():
    """16 channels, L = 256, M = 47, 240000 samples: parameters 2.9 GB. Forward
    and backward run whole on the GPU (the backward recomputing every input
    spectrum inside the adjoint kernel); gradient entries are checked against
    the oracle computed entry by entry."""
    dev = _dev()
    from paper_2310_00319_gb300.autograd import spectral_tvolap
    d = W.differentiable(seed=4)
    L, M, nb = d["L"], d["M"], d["n_blocks"]
    plan = _plan(d, dev)
    x = torch.from_numpy(d["x"]).to(dev).requires_grad_(True)
    P = torch.from_numpy(d["P"]).to(dev).requires_grad_(True)
    r = torch.from_numpy(d["r"]).to(dev)
    y = spectral_tvolap(x, P, plan)                 # backward recomputes X inside the kernel
    (y * r).sum().backward()
    assert torch.isfinite(y).all() and torch.isfinite(P.grad).all() and torch.isfinite(x.grad).all()
    rng = np.random.default_rng(5)
    for c in (0, 7, 15):
        idx = [(int(rng.integers(0, nb)), int(rng.integers(0, M)), int(rng.integers(0, 2 * L)))
               for _ in range(24)] + [(nb - 1, M - 1, 5), (3, M - 1, 0)]
        sidx = [int(v) for v in rng.integers(0, d["x"].shape[1], 6)] + [0, d["x"].shape[1] - 1]
        sP, sx = oracle.params_grad_sampled(d["x"][c], d["P"][c], L, d["r"][c], idx, sidx)
        gP = np.array([P.grad[c, t, m, k].item() for (t, m, k) in idx])
        gx = x.grad[c, sidx].cpu().numpy()
        peakP = float(P.grad[c].abs().max())
        assert np.max(np.abs(gP - sP)) <= 1e-3 * peakP, c
        relx, _ = _rel(gx, sx)
        assert relx <= 1e-3, (c, relx)


@pytest.mark.parametrize("L,q_first,q_count", [(32, 0, None), (64, 0, 37), (64, 9, 23)])
def test_adjoint_mac_x_equals_two_step(L, q_first, q_count):
    """tvolap_adjoint_mac_x (input spectra recomputed in the kernel) gives the
    same dP and dX, bit for bit, as tvolap_block_spectra + tvolap_adjoint_mac,
    for the whole range and for ranges that start inside the signal."""
    dev = _dev()
    d = W.differentiable(seed=15, n_ch=3, N=40 * L + 7, L=L, ir_len=9 * L)
    plan = _plan(d, dev)
    nb = d["n_blocks"]
    qc = nb - q_first if q_count is None else q_count
    x = torch.from_numpy(d["x"]).to(dev)
    Pm = torch.from_numpy(d["P"]).to(dev)
    r = torch.from_numpy(d["r"]).to(dev)
    G = plan.adjoint_output(r, 0, nb)
    dP1 = torch.zeros_like(Pm)
    dP2 = torch.zeros_like(Pm)
    X = plan.block_spectra(x, q_first, qc)
    dX1 = plan.adjoint_mac(G, 0, X, q_first, Pm, q_first, qc, dP1)
    dX2 = plan.adjoint_mac_x(G, 0, x, Pm, q_first, qc, dP2)
    torch.cuda.synchronize()
    assert torch.equal(dX1, dX2)
    assert torch.equal(dP1, dP2)
