"""TVOLAP with trainable per-block partition spectra, as a torch.autograd.Function.

The forward and backward passes are the library's kernels (Eq. 7 with free
spectra P, its adjoint, and the adjoints of the transforms) called through the
C ABI; this module only orders the calls and holds the tensors.

    y = spectral_tvolap(x, P, plan)          # x [C, N], P [C, n_blocks, M, 2L] complex64
    loss = ((y - target) ** 2).mean(); loss.backward()

The input spectra X are not kept from the forward to the backward: the
backward recomputes them. By default each block's spectrum is recomputed
inside the adjoint kernel where it is used (tvolap_adjoint_mac_x: no X stored
at all, one launch); with ``segment=K`` they are recomputed per segment of K
blocks by the transform kernel, so that at most K blocks of X are held (the
adjoint of Eq. 7 at block q reads only X(q)). With ``fwd_segment=K`` the forward too
holds X for at most K blocks plus the 2(M-1)-block history a segment reads.
Results are the same with and without segments.
"""
from __future__ import annotations

import torch

from .tvolap import Plan, n_blocks_for


class SpectralTvolap(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, Pspec, plan: Plan, out_len: int, segment: int | None,
                fwd_segment: int | None):
        C, N = x.shape
        nb = n_blocks_for(out_len, plan.L)
        if Pspec.shape != (plan.n_out, nb, plan.M, plan.P):
            raise ValueError(f"P must be [{plan.n_out}, {nb}, {plan.M}, {plan.P}]")
        x = x.contiguous()
        Pspec = Pspec.contiguous()
        K = 0 if not segment else int(segment)          # 0: recompute inside the kernel
        Kf = nb if not fwd_segment else int(fwd_segment)
        if Kf >= nb:
            X = plan.block_spectra(x, 0, nb)
            Y = plan.mac_params(X, 0, Pspec, 0, nb)
        else:
            Y = torch.empty((plan.n_out, nb, plan.P), dtype=torch.complex64, device=x.device)
            for t0 in range(0, nb, Kf):
                tc = min(Kf, nb - t0)
                x0 = max(0, t0 - 2 * (plan.M - 1))
                X = plan.block_spectra(x, x0, t0 + tc - x0)
                plan.mac_params(X, x0, Pspec, t0, tc, out=Y, out_row=t0)
        del X
        y = plan.inverse_ola(Y, out_len)
        ctx.save_for_backward(x, Pspec)
        ctx.plan, ctx.nb, ctx.K = plan, nb, K
        return y

    @staticmethod
    def backward(ctx, gy):
        x, Pspec = ctx.saved_tensors
        plan, nb, K = ctx.plan, ctx.nb, ctx.K
        G = plan.adjoint_output(gy.contiguous(), 0, nb)
        dP = torch.empty_like(Pspec)
        dX = torch.empty((plan.n_out, nb, plan.P), dtype=torch.complex64, device=x.device)
        if K == 0:
            plan.adjoint_mac_x(G, 0, x, Pspec, 0, nb, dP, dX=dX, dx_row=0)
        else:
            for q0 in range(0, nb, K):
                qc = min(K, nb - q0)
                X = plan.block_spectra(x, q0, qc)
                plan.adjoint_mac(G, 0, X, q0, Pspec, q0, qc, dP, dX=dX, dx_row=q0)
        dx = None
        if ctx.needs_input_grad[0]:
            dx = torch.zeros_like(x)
            plan.adjoint_input(dX, 0, dx)
        return dx, dP, None, None, None, None


def spectral_tvolap(x, Pspec, plan: Plan, out_len: int | None = None, segment: int | None = None,
                    fwd_segment: int | None = None):
    """y [C, out_len] from x [C, N] and per-block spectra Pspec [C, n_blocks, M, 2L]."""
    return SpectralTvolap.apply(x, Pspec, plan, x.shape[1] if out_len is None else out_len,
                                segment, fwd_segment)
