"""Python face of the TVOLAP C ABI (include/tvolap.h).

Thin: it checks tensor devices, dtypes and shapes, passes raw device
pointers and the plan's CUDA stream to the C library, and returns tensors.
PyTorch only supplies device memory and streams; every step of the method runs
in the library's kernels. Spectra are complex64 tensors of P = 2L bins on the
half-bin grid (k + 1/2) / 4L.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _need(t, dtype, device, name, ndim=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, got {t.device}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dims, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _dims(t, name, *dims):
    """t.shape must be dims (None: any extent); the kernels index every listed
    extent, so a smaller tensor would be read or written out of bounds."""
    if t.dim() != len(dims) or any(d is not None and n != d for n, d in zip(t.shape, dims)):
        want = ", ".join("*" if d is None else str(d) for d in dims)
        raise ValueError(f"{name} must be [{want}], got {list(t.shape)}")
    return t


def n_blocks_for(out_len: int, L: int) -> int:
    """Schedule entries for output samples [0, out_len): t = l + 1, l = -1 ..
    floor((out_len - 1) / L)."""
    return 0 if out_len <= 0 else (out_len - 1) // L + 2


OPT_MAC_STAGING, OPT_STAGE_TIMING, OPT_XFORM_THREADS = 1, 2, 3


class Plan:
    """One TVOLAP plan: hop L, M partitions, n_in inputs, n_out outputs,
    n_slots stored filters. Calls run on ``stream`` (default: the current
    torch stream of ``device`` at creation)."""

    def __init__(self, L: int, M: int, n_in: int = 1, n_out: int | None = None,
                 out_to_in=None, n_slots: int = 1, device=None, stream=None):
        self.lib = _lib.load()
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise ValueError("TVOLAP plans live on a CUDA device")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        n_out = n_in if n_out is None else n_out
        self.L, self.M, self.P = int(L), int(M), 2 * int(L)
        self.n_in, self.n_out, self.n_slots = int(n_in), int(n_out), int(n_slots)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            o2i = None
            if out_to_in is not None:
                vals = [int(v) for v in out_to_in]
                if len(vals) != n_out:
                    raise ValueError("out_to_in must have n_out entries")
                o2i = (ctypes.c_int32 * n_out)(*vals)
            h = ctypes.c_void_p()
            st = self.lib.tvolap_create(ctypes.byref(h), self.L, self.M, 4 * self.L, self.n_in,
                                        self.n_out, o2i, self.n_slots,
                                        ctypes.c_void_p(self.stream.cuda_stream))
            _lib.check(st, "tvolap_create")
        self.h = h
        self.out_to_in = list(out_to_in) if out_to_in is not None else list(range(n_out))
        self.n_mix = 0

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            with torch.cuda.device(self.device):
                _lib.check(self.lib.tvolap_destroy(self.h), "tvolap_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _call(self, name, *args):
        with torch.cuda.device(self.device):
            return _lib.check(getattr(self.lib, name)(self.h, *args), name)

    @property
    def slot_count(self) -> int:
        return self._call("tvolap_slot_count")

    def reset(self):
        self._call("tvolap_reset")

    def set_option(self, option: int, value: int):
        """TVOLAP_OPT_MAC_STAGING (1): 0 = persistent TMA groups of up to four
        filters, runs of up to three (default), 1 = cp.async, 2 = TMA groups
        and runs of up to four filters, 3 = one TMA group per CTA, 4 = as 3
        with two bins per thread, 5 = as 0 with runs of up to four filters. TVOLAP_OPT_STAGE_TIMING (2): 1 = time the three
        stages of process_block (see stage_times). TVOLAP_OPT_XFORM_THREADS
        (3): threads per CTA of the offline transforms, 0 (256), 128 or 64."""
        self._call("tvolap_set_option", int(option), int(value))

    def stage_times(self):
        """(forward, multiply-accumulate, inverse) milliseconds summed over the
        ticks timed since TVOLAP_OPT_STAGE_TIMING was set, and that tick count."""
        ms = (ctypes.c_double * 3)()
        n = ctypes.c_int64()
        self._call("tvolap_stage_times", ms, ctypes.byref(n))
        return list(ms), n.value

    def check(self):
        """Synchronise and raise if a kernel met an invalid slot index."""
        self._call("tvolap_check")

    # ------------------------------------------------------------------ filters
    def load_bank(self, first_slot: int, irs: torch.Tensor):
        """Transform irs [count, ir_len] (float32, on device) into slots
        first_slot .. first_slot + count - 1."""
        irs = _need(irs, torch.float32, self.device, "irs", 2)
        self._call("tvolap_load_bank", int(first_slot), irs.shape[0], _ptr(irs), irs.shape[1],
                   irs.shape[1])

    def set_filter(self, out_ch: int, ir: torch.Tensor):
        ir = _need(ir, torch.float32, self.device, "ir", 1)
        self._call("tvolap_set_filter", int(out_ch), _ptr(ir), ir.shape[0])

    def select(self, out_ch: int, slot_a: int, slot_b: int | None = None, alpha: float = 0.0):
        slot_b = slot_a if slot_b is None else slot_b
        self._call("tvolap_select", int(out_ch), int(slot_a), int(slot_b), float(alpha))

    def bank_spectra(self, slot: int) -> torch.Tensor:
        out = torch.empty((self.M, self.P), dtype=torch.complex64, device=self.device)
        self._call("tvolap_bank_spectra", int(slot), _ptr(out))
        return out

    # ------------------------------------------------------------------ streaming
    def process_block(self, x: torch.Tensor, out: torch.Tensor | None = None, sel_a=None,
                      sel_b=None, sel_alpha=None) -> torch.Tensor:
        """One hop: x [n_in, L] -> [n_out, L] (the offline output delayed by L)."""
        x = _need(x, torch.float32, self.device, "x", 2)
        if tuple(x.shape) != (self.n_in, self.L):
            raise ValueError(f"x must be [{self.n_in}, {self.L}]")
        if out is None:
            out = torch.empty((self.n_out, self.L), dtype=torch.float32, device=self.device)
        _dims(_need(out, torch.float32, self.device, "out", 2), "out", self.n_out, self.L)
        for t, nm, dt in ((sel_a, "sel_a", torch.int32), (sel_b, "sel_b", torch.int32),
                          (sel_alpha, "sel_alpha", torch.float32)):
            if t is not None:
                _need(t, dt, self.device, nm, 1)
                if t.shape[0] != self.n_out:
                    raise ValueError(f"{nm} must have n_out entries")
        self._call("tvolap_process_block", _ptr(x), _ptr(out), _ptr(sel_a), _ptr(sel_b),
                   _ptr(sel_alpha))
        return out

    # ------------------------------------------------------------------ state
    def state_bytes(self) -> int:
        n = int(self.lib.tvolap_state_bytes(self.h))
        if n < 0:
            _lib.check(n, "tvolap_state_bytes")
        return n

    def get_state(self, out: torch.Tensor | None = None) -> torch.Tensor:
        """Snapshot of the streaming state into a uint8 tensor (device by
        default; a CPU tensor works too)."""
        n = self.state_bytes()
        if out is None:
            out = torch.empty(n, dtype=torch.uint8, device=self.device)
        if out.dtype != torch.uint8 or not out.is_contiguous() or out.numel() < n:
            raise ValueError(f"out must be a contiguous uint8 tensor of >= {n} bytes")
        self._call("tvolap_get_state", ctypes.c_void_p(out.data_ptr()), out.numel())
        return out

    def set_state(self, state: torch.Tensor):
        """Restore a snapshot from get_state (same plan shape)."""
        if state.dtype != torch.uint8 or not state.is_contiguous():
            raise ValueError("state must be a contiguous uint8 tensor")
        self._call("tvolap_set_state", ctypes.c_void_p(state.data_ptr()), state.numel())

    # ------------------------------------------------------------------ mixdown
    def set_mix(self, mix_of_out, n_mix: int | None = None):
        """Sum plan outputs into n_mix mix outputs before the inverse transform:
        mix_of_out[o] in [0, n_mix) (sequence of n_out ints); None removes it."""
        if mix_of_out is None:
            self._call("tvolap_set_mix", 0, None)
            self.n_mix = 0
            return
        vals = [int(v) for v in mix_of_out]
        if len(vals) != self.n_out:
            raise ValueError(f"mix_of_out must have {self.n_out} entries")
        n_mix = max(vals) + 1 if n_mix is None else int(n_mix)
        self._call("tvolap_set_mix", n_mix, (ctypes.c_int32 * self.n_out)(*vals))
        self.n_mix = n_mix

    def mix(self, Y: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Mixdown stage: Y complex64 [n_out, n_blocks, 2L] -> [n_mix, n_blocks, 2L]."""
        Y = _dims(_need(Y, torch.complex64, self.device, "Y", 3), "Y", self.n_out, None, self.P)
        nb = Y.shape[1]
        if out is None:
            out = torch.empty((self.n_mix, nb, self.P), dtype=torch.complex64, device=self.device)
        _dims(_need(out, torch.complex64, self.device, "out", 3), "out", self.n_mix, nb, self.P)
        self._call("tvolap_mix", _ptr(Y), nb, _ptr(out))
        return out

    def process_signal_mix(self, x: torch.Tensor, sched_a, sched_b=None, sched_alpha=None,
                           out_len: int | None = None, out: torch.Tensor | None = None):
        """Offline TVOLAP with the mixdown: x [n_in, N] -> y [n_mix, out_len]."""
        x = _need(x, torch.float32, self.device, "x", 2)
        if x.shape[0] != self.n_in:
            raise ValueError(f"x must have {self.n_in} rows")
        N = x.shape[1]
        out_len = N if out_len is None else int(out_len)
        nb = n_blocks_for(out_len, self.L)
        sa, sb, sal, stride = self._sched(sched_a, sched_b, sched_alpha, nb)
        if out is None:
            out = torch.empty((self.n_mix, out_len), dtype=torch.float32, device=self.device)
        _need(out, torch.float32, self.device, "out", 2)
        if out.shape[0] != self.n_mix or out.shape[1] < out_len:
            raise ValueError("out too small")
        self._call("tvolap_process_signal_mix", _ptr(x), N, N, _ptr(sa), _ptr(sb), _ptr(sal),
                   stride, _ptr(out), out_len, out.shape[1])
        return out

    def process_block_mix(self, x: torch.Tensor, out: torch.Tensor | None = None, sel_a=None,
                          sel_b=None, sel_alpha=None) -> torch.Tensor:
        """One hop with the mixdown: x [n_in, L] -> [n_mix, L] (delayed by L)."""
        x = _need(x, torch.float32, self.device, "x", 2)
        if tuple(x.shape) != (self.n_in, self.L):
            raise ValueError(f"x must be [{self.n_in}, {self.L}]")
        if out is None:
            out = torch.empty((self.n_mix, self.L), dtype=torch.float32, device=self.device)
        _dims(_need(out, torch.float32, self.device, "out", 2), "out", self.n_mix, self.L)
        for t, nm, dt in ((sel_a, "sel_a", torch.int32), (sel_b, "sel_b", torch.int32),
                          (sel_alpha, "sel_alpha", torch.float32)):
            if t is not None:
                _need(t, dt, self.device, nm, 1)
                if t.shape[0] != self.n_out:
                    raise ValueError(f"{nm} must have n_out entries")
        self._call("tvolap_process_block_mix", _ptr(x), _ptr(out), _ptr(sel_a), _ptr(sel_b),
                   _ptr(sel_alpha))
        return out

    # ------------------------------------------------------------------ offline
    def _sched(self, sched_a, sched_b, sched_alpha, nb):
        sched_a = _need(sched_a, torch.int32, self.device, "sched_a", 2)
        if sched_a.shape[0] != self.n_out or sched_a.shape[1] < nb:
            raise ValueError(f"sched_a must be [{self.n_out}, >= {nb}]")
        stride = sched_a.shape[1]
        for t, nm, dt in ((sched_b, "sched_b", torch.int32),
                          (sched_alpha, "sched_alpha", torch.float32)):
            if t is not None:
                _need(t, dt, self.device, nm, 2)
                if tuple(t.shape) != tuple(sched_a.shape):
                    raise ValueError(f"{nm} must match sched_a's shape")
        return sched_a, sched_b, sched_alpha, stride

    def process_signal(self, x: torch.Tensor, sched_a, sched_b=None, sched_alpha=None,
                       out_len: int | None = None, out: torch.Tensor | None = None):
        """Offline TVOLAP of x [n_in, N] -> y [n_out, out_len] (aligned with x)."""
        x = _need(x, torch.float32, self.device, "x", 2)
        if x.shape[0] != self.n_in:
            raise ValueError(f"x must have {self.n_in} rows")
        N = x.shape[1]
        out_len = N if out_len is None else int(out_len)
        nb = n_blocks_for(out_len, self.L)
        sa, sb, sal, stride = self._sched(sched_a, sched_b, sched_alpha, nb)
        if out is None:
            out = torch.empty((self.n_out, out_len), dtype=torch.float32, device=self.device)
        _need(out, torch.float32, self.device, "out", 2)
        if out.shape[0] != self.n_out or out.shape[1] < out_len:
            raise ValueError("out too small")
        self._call("tvolap_process_signal", _ptr(x), N, N, _ptr(sa), _ptr(sb), _ptr(sal),
                   stride, _ptr(out), out_len, out.shape[1])
        return out

    def process_ragged(self, x: torch.Tensor, n: torch.Tensor, out_len: torch.Tensor,
                       parts: torch.Tensor, max_out_len: int, sched_a, sched_b=None,
                       sched_alpha=None, out: torch.Tensor | None = None):
        """Channels of different lengths and partition counts in one call:
        x [C, x_stride] (channel c holds n[c] samples), n/out_len int64 [C],
        parts int32 [C]; returns y [C, max_out_len] (channel c valid up to
        out_len[c])."""
        x = _dims(_need(x, torch.float32, self.device, "x", 2), "x", self.n_in, None)
        _dims(_need(n, torch.int64, self.device, "n", 1), "n", self.n_in)
        _dims(_need(out_len, torch.int64, self.device, "out_len", 1), "out_len", self.n_out)
        _dims(_need(parts, torch.int32, self.device, "parts", 1), "parts", self.n_out)
        nb = n_blocks_for(max_out_len, self.L)
        sa, sb, sal, stride = self._sched(sched_a, sched_b, sched_alpha, nb)
        if out is None:
            out = torch.empty((self.n_out, max_out_len), dtype=torch.float32, device=self.device)
        _dims(_need(out, torch.float32, self.device, "out", 2), "out", self.n_out, None)
        self._call("tvolap_process_ragged", _ptr(x), x.shape[1], _ptr(n), _ptr(out_len),
                   _ptr(parts), int(max_out_len), _ptr(sa), _ptr(sb), _ptr(sal), stride,
                   _ptr(out), out.shape[1])
        return out

    def workspace_bytes(self, out_len: int) -> int:
        return self._call("tvolap_signal_workspace_bytes", int(out_len))

    def forward_spectra(self, x: torch.Tensor, n_blocks: int) -> torch.Tensor:
        """X [n_in, n_blocks, P] of input blocks l = -1 .. n_blocks - 2."""
        x = _dims(_need(x, torch.float32, self.device, "x", 2), "x", self.n_in, None)
        X = torch.empty((self.n_in, n_blocks, self.P), dtype=torch.complex64, device=self.device)
        self._call("tvolap_forward_spectra", _ptr(x), x.shape[1], x.shape[1], int(n_blocks),
                   _ptr(X))
        return X

    def mac(self, X: torch.Tensor, sched_a, sched_b=None, sched_alpha=None) -> torch.Tensor:
        X = _dims(_need(X, torch.complex64, self.device, "X", 3), "X", self.n_in, None, self.P)
        nb = X.shape[1]
        sa, sb, sal, stride = self._sched(sched_a, sched_b, sched_alpha, nb)
        Y = torch.empty((self.n_out, nb, self.P), dtype=torch.complex64, device=self.device)
        self._call("tvolap_mac", _ptr(X), nb, _ptr(sa), _ptr(sb), _ptr(sal), stride, _ptr(Y))
        return Y

    def inverse_ola(self, Y: torch.Tensor, out_len: int) -> torch.Tensor:
        Y = _dims(_need(Y, torch.complex64, self.device, "Y", 3), "Y", self.n_out, None, self.P)
        y = torch.empty((self.n_out, out_len), dtype=torch.float32, device=self.device)
        self._call("tvolap_inverse_ola", _ptr(Y), Y.shape[1], _ptr(y), int(out_len), int(out_len))
        return y

    # ------------------------------------------------------------------ differentiable model
    def block_spectra(self, x: torch.Tensor, t_first: int, t_count: int) -> torch.Tensor:
        """X [n_in, t_count, P]: spectra of blocks t_first .. t_first + t_count - 1."""
        x = _dims(_need(x, torch.float32, self.device, "x", 2), "x", self.n_in, None)
        X = torch.empty((self.n_in, t_count, self.P), dtype=torch.complex64, device=self.device)
        self._call("tvolap_block_spectra", _ptr(x), x.shape[1], x.shape[1], int(t_first),
                   int(t_count), _ptr(X))
        return X

    def mac_params(self, X: torch.Tensor, x_first: int, Pspec: torch.Tensor, t_first: int,
                   t_count: int, out: torch.Tensor | None = None, out_row: int = 0) -> torch.Tensor:
        """Eq. 7 with per-block parameter spectra Pspec [n_out, p_blocks, M, P] for
        blocks t_first .. t_first + t_count - 1, written to rows out_row .. of
        out [n_out, rows, P] (default: a new [n_out, t_count, P])."""
        X = _dims(_need(X, torch.complex64, self.device, "X", 3), "X", self.n_in, None, self.P)
        Pspec = _dims(_need(Pspec, torch.complex64, self.device, "Pspec", 4), "Pspec", self.n_out,
                      None, self.M, self.P)
        if out is None:
            out = torch.empty((self.n_out, t_count, self.P), dtype=torch.complex64,
                              device=self.device)
        _dims(_need(out, torch.complex64, self.device, "out", 3), "out", self.n_out, None, self.P)
        if out_row < 0 or out_row + t_count > out.shape[1]:
            raise ValueError("out rows out of range")
        ptr = ctypes.c_void_p(out.data_ptr() + out_row * self.P * 8)
        self._call("tvolap_mac_params", _ptr(X), int(x_first), X.shape[1], _ptr(Pspec),
                   Pspec.shape[1], int(t_first), int(t_count), ptr, out.shape[1])
        return out

    def adjoint_output(self, g: torch.Tensor, t_first: int, t_count: int) -> torch.Tensor:
        """G [n_out, t_count, P] = dL/dY of blocks t_first .. from g = dL/dy."""
        g = _dims(_need(g, torch.float32, self.device, "g", 2), "g", self.n_out, None)
        G = torch.empty((self.n_out, t_count, self.P), dtype=torch.complex64, device=self.device)
        self._call("tvolap_adjoint_output", _ptr(g), g.shape[1], g.shape[1], int(t_first),
                   int(t_count), _ptr(G))
        return G

    def _adjoint_operands(self, G, Pspec, dP):
        G = _dims(_need(G, torch.complex64, self.device, "G", 3), "G", self.n_out, None, self.P)
        Pspec = _dims(_need(Pspec, torch.complex64, self.device, "Pspec", 4), "Pspec", self.n_out,
                      None, self.M, self.P)
        dP = _dims(_need(dP, torch.complex64, self.device, "dP", 4), "dP", *Pspec.shape)
        return G, Pspec, dP

    def adjoint_mac(self, G, g_first, X, x_first, Pspec, q_first, q_count, dP, dX=None,
                    dx_row=0):
        """dP (written in place for t - 2m in the q range) and the input-block
        gradients, written to rows dx_row .. of dX [n_out, rows, P] (default: a
        new [n_out, q_count, P])."""
        G, Pspec, dP = self._adjoint_operands(G, Pspec, dP)
        X = _dims(_need(X, torch.complex64, self.device, "X", 3), "X", self.n_in, None, self.P)
        if dX is None:
            dX = torch.empty((self.n_out, q_count, self.P), dtype=torch.complex64,
                             device=self.device)
        _dims(_need(dX, torch.complex64, self.device, "dX", 3), "dX", self.n_out, None, self.P)
        if dx_row < 0 or dx_row + q_count > dX.shape[1]:
            raise ValueError("dX rows out of range")
        ptr = ctypes.c_void_p(dX.data_ptr() + dx_row * self.P * 8)
        self._call("tvolap_adjoint_mac", _ptr(G), int(g_first), G.shape[1], _ptr(X), int(x_first),
                   X.shape[1], _ptr(Pspec), Pspec.shape[1], int(q_first), int(q_count), _ptr(dP),
                   ptr, dX.shape[1])
        return dX

    def adjoint_mac_x(self, G, g_first, x, Pspec, q_first, q_count, dP, dX=None, dx_row=0):
        """adjoint_mac with the input spectra recomputed inside the kernel from
        x [n_in, N] (nothing stored between forward and backward)."""
        G, Pspec, dP = self._adjoint_operands(G, Pspec, dP)
        x = _dims(_need(x.contiguous(), torch.float32, self.device, "x", 2), "x", self.n_in, None)
        if dX is None:
            dX = torch.empty((self.n_out, q_count, self.P), dtype=torch.complex64,
                             device=self.device)
        _dims(_need(dX, torch.complex64, self.device, "dX", 3), "dX", self.n_out, None, self.P)
        if dx_row < 0 or dx_row + q_count > dX.shape[1]:
            raise ValueError("dX rows out of range")
        ptr = ctypes.c_void_p(dX.data_ptr() + dx_row * self.P * 8)
        self._call("tvolap_adjoint_mac_x", _ptr(G), int(g_first), G.shape[1], _ptr(x), x.shape[1],
                   x.shape[1], _ptr(Pspec), Pspec.shape[1], int(q_first), int(q_count), _ptr(dP),
                   ptr, dX.shape[1])
        return dX

    def adjoint_input(self, dX: torch.Tensor, q_first: int, dx: torch.Tensor):
        """dx [n_in, N] += the input gradient of blocks q_first .. + dX.shape[1] - 1."""
        _dims(_need(dX, torch.complex64, self.device, "dX", 3), "dX", self.n_out, None, self.P)
        _dims(_need(dx, torch.float32, self.device, "dx", 2), "dx", self.n_in, None)
        self._call("tvolap_adjoint_input", _ptr(dX), int(q_first), dX.shape[1], _ptr(dx),
                   dx.shape[1], dx.shape[1])
        return dx
