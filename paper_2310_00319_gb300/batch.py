"""Python binding of batched sources (tvolap_batch_*): argument marshalling only.

Many independent sources with different hops, impulse-response lengths and
signal lengths run together: the library groups them by hop (one plan per
group, channels = sources, tvolap_process_ragged), runs every group on one
stream, can capture the whole batch as one CUDA graph, and picks the
multiply-accumulate staging per group by timing the variants on the batch.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .tvolap import _ptr


class _Source(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("M", ctypes.c_int), ("n_filters", ctypes.c_int),
                ("N", ctypes.c_int64), ("out_len", ctypes.c_int64)]


def _partitions(ir_len: int, L: int) -> int:
    return max(1, -(-ir_len // (2 * L)))


class BatchedTvolap:
    """sources: objects with L, x [N] (float32), irs [n_filters, ir_len]
    (float32), sched [n_blocks] (int32 index into irs per block, t = l + 1) and
    out_len. All calls are ordered on ``stream`` (default: a new stream)."""

    def __init__(self, sources, device=None, stream=None):
        self.lib = _lib.load()
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.sources = sources
        n = len(sources)
        arr = (_Source * n)(*[_Source(int(s.L), _partitions(s.irs.shape[1], int(s.L)),
                                      s.irs.shape[0], s.x.shape[0], int(s.out_len))
                              for s in sources])
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self.lib.tvolap_batch_create(ctypes.byref(h), arr, n,
                                                    ctypes.c_void_p(self.stream.cuda_stream)),
                       "tvolap_batch_create")
        self.h = h
        keep = []                       # device copies alive until the stream has read them
        with torch.cuda.device(self.device):
            for i, s in enumerate(sources):
                nb = 0 if s.out_len <= 0 else (int(s.out_len) - 1) // int(s.L) + 2
                x = torch.from_numpy(np.ascontiguousarray(s.x, np.float32)).to(self.device)
                sc = torch.from_numpy(np.ascontiguousarray(s.sched[:nb], np.int32)).to(self.device)
                irs = torch.from_numpy(np.ascontiguousarray(s.irs, np.float32)).to(self.device)
                self.stream.wait_stream(torch.cuda.current_stream(self.device))
                self._call("tvolap_batch_set_source", i,
                           _ptr(x) if x.numel() else None, _ptr(sc) if sc.numel() else None)
                self._call("tvolap_batch_load_filters", i, _ptr(irs), irs.shape[1], irs.shape[1])
                keep += [x, sc, irs]
            self.stream.synchronize()
        del keep
        self.graph = False

    def set_source(self, i: int, x: torch.Tensor, sched: torch.Tensor):
        """Replace source i's input (device float32 [N]) and schedule (device
        int32 [n_blocks], indices into its filters); later runs and graph
        replays read them."""
        x = x.contiguous()
        sched = sched.to(torch.int32).contiguous()
        if not 0 <= int(i) < len(self.sources):
            raise IndexError(f"source {i} out of range")
        src = self.sources[i]
        N, out_len, L = src.x.shape[0], int(src.out_len), int(src.L)
        nb = 0 if out_len <= 0 else (out_len - 1) // L + 2
        for t, nm in ((x, "x"), (sched, "sched")):
            if t.device.type != "cuda" or (self.device.index is not None
                                           and t.device.index != self.device.index):
                raise ValueError(f"{nm} must be on {self.device}")
        if x.dtype != torch.float32 or x.dim() != 1 or x.numel() != N:
            raise ValueError(f"x must be float32 [{N}] (source {i}'s length)")
        if sched.dim() != 1 or sched.numel() < nb:
            raise ValueError(f"sched must be int32 [>= {nb}] (source {i}'s blocks)")
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self._call("tvolap_batch_set_source", int(i), _ptr(x) if x.numel() else None,
                   _ptr(sched) if sched.numel() else None)
        x.record_stream(self.stream)
        sched.record_stream(self.stream)

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.tvolap_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        return _lib.check(getattr(self.lib, name)(self.h, *args), name)

    # ------------------------------------------------------------------ runs
    def run(self):
        """Enqueue one run of every source (a graph replay once captured)."""
        self._call("tvolap_batch_run")

    def capture(self):
        """Record one run of the whole batch as a CUDA graph."""
        self._call("tvolap_batch_capture")
        self.graph = True

    def replay(self):
        if not self.graph:
            self.capture()
        self.run()

    def autotune(self, reps: int = 3) -> dict:
        """Per hop group, keep the fastest multiply-accumulate staging, then
        the fastest transform CTA size. Returns {L: staging};
        group_tiling(g) gives both choices."""
        ng = self.n_groups
        chosen = (ctypes.c_int * ng)()
        self._call("tvolap_batch_autotune", int(reps), chosen)
        self.graph = False
        return {self.group_info(g)[0]: int(chosen[g]) for g in range(ng)}

    def set_staging(self, staging: int, group: int = -1):
        """Multiply-accumulate staging of one hop group (-1: all)."""
        self._call("tvolap_batch_set_staging", int(group), int(staging))
        self.graph = False

    def check(self):
        """Synchronise and raise on deferred device errors of any group."""
        self._call("tvolap_batch_check")

    # ------------------------------------------------------------------ results
    def output(self, i: int) -> torch.Tensor:
        """Output of source i (a copy, ordered after the batch's work)."""
        n = int(self.sources[i].out_len)
        y = torch.empty(n, dtype=torch.float32, device=self.device)
        if n:
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
            self._call("tvolap_batch_get_output", int(i), _ptr(y))
            torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return y

    @property
    def n_groups(self) -> int:
        n = ctypes.c_int()
        self._call("tvolap_batch_groups", ctypes.byref(n))
        return n.value

    def group_info(self, g: int):
        """(hop L, sources, staging) of hop group g (increasing hop order)."""
        L, n, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._call("tvolap_batch_group_info", int(g), ctypes.byref(L), ctypes.byref(n),
                   ctypes.byref(st))
        return L.value, n.value, st.value

    def group_tiling(self, g: int):
        """(multiply-accumulate staging, transform CTA size; 0 = default) of
        hop group g."""
        st, th = ctypes.c_int(), ctypes.c_int()
        self._call("tvolap_batch_group_tiling", int(g), ctypes.byref(st), ctypes.byref(th))
        return st.value, th.value
