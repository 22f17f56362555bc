"""Python binding of two-level non-uniform partitions (tvolap_nu_*): argument
marshalling only. A head level (hop La, Ma partitions) covers taps [0, D),
D = 2 La Ma, at the small hop's latency; a tail level (hop ratio * La, Mb
partitions) covers the rest at a lower cost per sample, its output added D
samples later."""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from .tvolap import _dims, _need, _ptr, n_blocks_for


class NonUniform:
    def __init__(self, La: int, Ma: int, ratio: int, Mb: int, n_in: int = 1,
                 n_out: int | None = None, out_to_in=None, n_slots: int = 1, device=None,
                 stream=None):
        self.lib = _lib.load()
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        n_out = n_in if n_out is None else n_out
        self.La, self.Ma, self.ratio, self.Mb = int(La), int(Ma), int(ratio), int(Mb)
        self.Lb = self.La * self.ratio
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
            _lib.check(self.lib.tvolap_nu_create(ctypes.byref(h), self.La, self.Ma, self.ratio,
                                                 self.Mb, self.n_in, self.n_out, o2i,
                                                 self.n_slots,
                                                 ctypes.c_void_p(self.stream.cuda_stream)),
                       "tvolap_nu_create")
        self.h = h
        D, mx = ctypes.c_int64(), ctypes.c_int64()
        self._call("tvolap_nu_dims", None, None, ctypes.byref(D), ctypes.byref(mx))
        self.head_taps, self.max_taps = D.value, mx.value

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.tvolap_nu_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        return _lib.check(getattr(self.lib, name)(self.h, *args), name)

    def reset(self):
        self._call("tvolap_nu_reset")

    def check(self):
        self._call("tvolap_nu_check")

    def set_option(self, option: int, value: int, level: int = -1):
        """tvolap_set_option for the head (0), the tail (1) or both (-1)."""
        self._call("tvolap_nu_set_option", int(level), int(option), int(value))

    def load_bank(self, first_slot: int, irs: torch.Tensor):
        """irs: device float32 [count, ir_len], ir_len <= head_taps + 2 Lb Mb."""
        irs = _need(irs, torch.float32, self.device, "irs", 2)
        self._call("tvolap_nu_load_bank", int(first_slot), irs.shape[0], _ptr(irs), irs.shape[1],
                   irs.shape[1])

    def process_signal(self, x: torch.Tensor, sched_a, sched_b=None, sched_alpha=None,
                       out_len: int | None = None, out: torch.Tensor | None = None) -> torch.Tensor:
        """Offline: x [n_in, N] -> y [n_out, out_len] (into out [n_out, >= out_len]
        when given); schedules per head block."""
        x = _dims(_need(x, torch.float32, self.device, "x", 2), "x", self.n_in, None)
        N = x.shape[1]
        out_len = N if out_len is None else int(out_len)
        nb = n_blocks_for(out_len, self.La)
        sa = _need(sched_a, torch.int32, self.device, "sched_a", 2)
        if sa.shape[0] != self.n_out or sa.shape[1] < nb:
            raise ValueError(f"sched_a must be [{self.n_out}, >= {nb}]")
        for t, nm in ((sched_b, "sched_b"), (sched_alpha, "sched_alpha")):
            if t is not None and tuple(t.shape) != tuple(sa.shape):
                raise ValueError(f"{nm} must match sched_a's shape")
        sb = None if sched_b is None else _need(sched_b, torch.int32, self.device, "sched_b", 2)
        sal = None if sched_alpha is None else _need(sched_alpha, torch.float32, self.device,
                                                     "sched_alpha", 2)
        if out is None:
            out = torch.empty((self.n_out, out_len), dtype=torch.float32, device=self.device)
        _dims(_need(out, torch.float32, self.device, "out", 2), "out", self.n_out, None)
        if out.shape[1] < out_len:
            raise ValueError(f"out must have >= {out_len} columns")
        self._call("tvolap_nu_process_signal", _ptr(x), N, N, _ptr(sa), _ptr(sb), _ptr(sal),
                   sa.shape[1], _ptr(out), out_len, out.shape[1])
        return out

    def process_block(self, x: torch.Tensor, out: torch.Tensor | None = None, sel_a=None,
                      sel_b=None, sel_alpha=None) -> torch.Tensor:
        """One head hop: x [n_in, La] -> [n_out, La] (delayed by La)."""
        x = _need(x, torch.float32, self.device, "x", 2)
        if tuple(x.shape) != (self.n_in, self.La):
            raise ValueError(f"x must be [{self.n_in}, {self.La}]")
        if out is None:
            out = torch.empty((self.n_out, self.La), dtype=torch.float32, device=self.device)
        _dims(_need(out, torch.float32, self.device, "out", 2), "out", self.n_out, self.La)
        for t, nm, dt in ((sel_a, "sel_a", torch.int32), (sel_b, "sel_b", torch.int32),
                          (sel_alpha, "sel_alpha", torch.float32)):
            if t is not None:
                _dims(_need(t, dt, self.device, nm, 1), nm, self.n_out)
        self._call("tvolap_nu_process_block", _ptr(x), _ptr(out), _ptr(sel_a), _ptr(sel_b),
                   _ptr(sel_alpha))
        return out
