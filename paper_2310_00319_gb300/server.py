"""Python binding of the streaming server (tvolap_server_*) and of its host
scheduler (tvolap_sched_*): argument marshalling only.

The staging arrays are numpy views of the server's pinned host memory, in two
sets used by alternate ticks. ``due`` picks the next tick's set (``buf``) after
waiting for the tick that used it before; then write, for each id it returns,
the stream's L new samples to ``inp[id, :L]`` and the filter index of the
block to ``sel[id]``. Once that tick has finished (``wait``, or the ``due`` call
two ticks later) its output block of output o is ``out[id, o, :L]`` of the same
set (``outs(buf)``).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

STATE_FREE, STATE_PENDING, STATE_LIVE = 0, 1, 2
OPT_GRAPH, OPT_WAIT_US, OPT_TIMING, OPT_FAIL_ADMITS = 1, 2, 3, 4


class _Stats(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_int64), ("stream_blocks", ctypes.c_int64),
                ("channel_samples", ctypes.c_int64), ("mac_bytes", ctypes.c_int64),
                ("live", ctypes.c_int32), ("pending", ctypes.c_int32),
                ("last_due", ctypes.c_int32), ("last_items", ctypes.c_int32),
                ("arena_bytes", ctypes.c_int64), ("arena_used", ctypes.c_int64),
                ("stage_ms", ctypes.c_double * 3), ("timed_ticks", ctypes.c_int64)]


def _np_view(ptr, shape, dtype):
    n = int(np.prod(shape))
    ctype = np.ctypeslib.as_ctypes_type(dtype)
    buf = (ctype * n).from_address(ptr)
    return np.ctypeslib.as_array(buf).reshape(shape)


def partitions(ir_len: int, L: int) -> int:
    return max(1, -(-ir_len // (2 * L)))


class Server:
    """Streams of hops base_hop .. max_hop (powers of two, at most 8x apart),
    up to ``capacity`` at once, 1 or 2 outputs each, in an arena of
    ``arena_bytes`` device bytes."""

    def __init__(self, base_hop: int, max_hop: int, capacity: int, max_out: int = 2,
                 arena_bytes: int = 1 << 30, device=None, stream=None):
        import torch
        self.lib = _lib.load()
        self.device = torch.device(device if device is not None else "cuda")
        self.base_hop, self.max_hop, self.capacity, self.max_out = base_hop, max_hop, capacity, max_out
        h = ctypes.c_void_p()
        sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        with torch.cuda.device(self.device):
            _lib.check(self.lib.tvolap_server_create(ctypes.byref(h), base_hop, max_hop, capacity,
                                                     max_out, int(arena_bytes), sp),
                       "tvolap_server_create")
        self.h = h
        self._in, self._out = [], []
        for b in (0, 1):
            pin, pst, psel, pout, post = (ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_void_p(),
                                          ctypes.c_void_p(), ctypes.c_int64())
            _lib.check(self.lib.tvolap_server_staging(h, b, ctypes.byref(pin), ctypes.byref(pst),
                                                      ctypes.byref(psel), ctypes.byref(pout),
                                                      ctypes.byref(post)), "tvolap_server_staging")
            self._in.append(_np_view(pin.value, (capacity, pst.value), np.float32))
            self._out.append(_np_view(pout.value, (capacity, max_out, post.value), np.float32))
        self.sel = _np_view(psel.value, (capacity,), np.int32)
        self.buf = 0             # staging set of the next tick (set by due)
        self._ids = np.zeros(capacity, np.int32)
        self._keep = {}          # response buffers held until their stream is live
        self._queued = {}        # response buffers of requests waiting in the queue
        self._admitted = []      # (ticket, id, wait_ticks) not yet taken by admitted()
        self._adm_t = np.zeros(capacity, np.int64)
        self._adm_i = np.zeros(capacity, np.int32)
        self._adm_w = np.zeros(capacity, np.int64)

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.tvolap_server_destroy(self.h)
            self.h = ctypes.c_void_p()
            self._in = self._out = self.sel = None
            self._keep.clear()
            self._queued.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        return _lib.check(getattr(self.lib, name)(self.h, *args), name)

    # ------------------------------------------------------------------ queue
    @staticmethod
    def _irs(irs):
        import torch
        if irs.dtype != torch.float32 or irs.device.type != "cuda" or irs.dim() != 3:
            raise ValueError("irs must be a CUDA float32 tensor [n_filters, n_out, ir_len]")
        return irs.contiguous()

    def submit(self, L: int, irs, M: int | None = None) -> int:
        """Queue a stream (admission queue): admitted at once when it fits,
        otherwise, in arrival order, at a later due() as streams retire.
        Returns the request's ticket; admitted() maps tickets to stream ids."""
        import torch
        irs = self._irs(irs)
        F, n_out, ir_len = irs.shape
        M = partitions(ir_len, L) if M is None else M
        t = ctypes.c_int64()
        with torch.cuda.device(self.device):
            self._call("tvolap_server_submit", L, M, n_out, F, ctypes.c_void_p(irs.data_ptr()),
                       ir_len, ir_len, ctypes.byref(t))
        self._queued[t.value] = irs
        self._drain()
        return t.value

    def _drain(self):
        n = ctypes.c_int()
        while True:
            self._call("tvolap_server_admitted", self._adm_t.ctypes.data_as(_lib.P_int64),
                       self._adm_i.ctypes.data_as(_lib.P_int32),
                       self._adm_w.ctypes.data_as(_lib.P_int64), self.capacity, ctypes.byref(n))
            for k in range(n.value):
                t, i, w = int(self._adm_t[k]), int(self._adm_i[k]), int(self._adm_w[k])
                self._keep[i] = self._queued.pop(t)
                self._admitted.append((t, i, w))
            if n.value < self.capacity:
                return

    def admitted(self) -> list:
        """(ticket, stream id, base ticks waited) of the requests admitted from
        the queue since the last call, oldest first."""
        out, self._admitted = self._admitted, []
        return out

    def cancel(self, ticket: int):
        self._call("tvolap_server_cancel", ctypes.c_int64(ticket))
        self._queued.pop(ticket, None)

    def queue(self) -> dict:
        w, o, a, m = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._call("tvolap_server_queue", ctypes.byref(w), ctypes.byref(o), ctypes.byref(a),
                   ctypes.byref(m))
        return {"waiting": w.value, "oldest_wait_ticks": o.value, "admitted_total": a.value,
                "max_wait_ticks": m.value}

    # ------------------------------------------------------------------ streams
    def footprint(self, L: int, M: int, n_out: int, n_filters: int) -> int:
        b = ctypes.c_int64()
        self._call("tvolap_server_footprint", L, M, n_out, n_filters, ctypes.byref(b))
        return b.value

    def admit(self, L: int, irs, M: int | None = None) -> int:
        """irs: device float32 tensor [n_filters, n_out, ir_len] (filter f,
        output o). Returns the stream id; raises TvolapError (status
        TVOLAP_ERR_CAPACITY) when it does not fit."""
        import torch
        irs = self._irs(irs)
        F, n_out, ir_len = irs.shape
        M = partitions(ir_len, L) if M is None else M
        i = ctypes.c_int()
        with torch.cuda.device(self.device):
            self._call("tvolap_server_admit", L, M, n_out, F, ctypes.c_void_p(irs.data_ptr()),
                       ir_len, ir_len, ctypes.byref(i))
        self._keep[i.value] = irs
        return i.value

    def retire(self, i: int):
        self._call("tvolap_server_retire", int(i))

    def snapshot(self, i: int, out=None):
        """Stream i's transformed filters and streaming state (after the ticks
        in flight) as a uint8 tensor (device by default, or into out)."""
        import torch
        n = ctypes.c_int64()
        self._call("tvolap_server_stream_bytes", int(i), ctypes.byref(n))
        if out is None:
            out = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        if out.dtype != torch.uint8 or not out.is_contiguous() or out.numel() < n.value:
            raise ValueError(f"out must be a contiguous uint8 tensor of >= {n.value} bytes")
        self._call("tvolap_server_snapshot", int(i), ctypes.c_void_p(out.data_ptr()), out.numel())
        return out

    def restore(self, snap) -> int:
        """Admit a stream from a snapshot (this or another server with the
        same hops); it continues where the snapshot was taken. Returns its id."""
        import torch
        if not isinstance(snap, torch.Tensor) or snap.dtype != torch.uint8 or \
                not snap.is_contiguous():
            raise ValueError("snap must be a contiguous uint8 tensor (from snapshot())")
        i = ctypes.c_int()
        self._call("tvolap_server_restore", ctypes.c_void_p(snap.data_ptr()), snap.numel(),
                   ctypes.byref(i))
        self._keep[i.value] = snap           # read by the admission copy until the stream is live
        return i.value

    def state(self, i: int):
        st, bl, ph = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        self._call("tvolap_server_state", int(i), ctypes.byref(st), ctypes.byref(bl),
                   ctypes.byref(ph))
        return st.value, bl.value, ph.value

    # ------------------------------------------------------------------ ticks
    @property
    def inp(self) -> np.ndarray:
        """Input staging of the next tick's set [capacity, max_hop]."""
        return self._in[self.buf]

    @property
    def out(self) -> np.ndarray:
        """Output staging of the set ``buf`` [capacity, max_out, max_hop]."""
        return self._out[self.buf]

    def outs(self, b: int) -> np.ndarray:
        return self._out[b]

    def due(self) -> np.ndarray:
        n, b = ctypes.c_int(), ctypes.c_int()
        self._call("tvolap_server_due", self._ids.ctypes.data_as(_lib.P_int32), self.capacity,
                   ctypes.byref(n), ctypes.byref(b))
        self.buf = b.value
        ids = self._ids[:n.value].copy()
        self._drain()
        for i in [k for k in self._keep if self.state(k)[0] != STATE_PENDING]:
            del self._keep[i]
        return ids

    def tick(self):
        self._call("tvolap_server_tick")

    def wait(self):
        """Returns None, or raises TvolapError (e.g. TVOLAP_ERR_TIMEOUT)."""
        self._call("tvolap_server_wait")
        self._keep.clear()

    def post(self, seq: int):
        self._call("tvolap_server_post", ctypes.c_uint64(seq))

    def set_option(self, option: int, value: int):
        self._call("tvolap_server_set_option", int(option), int(value))

    def stats(self) -> dict:
        s = _Stats()
        self._call("tvolap_server_stats_get", ctypes.byref(s))
        d = {k: getattr(s, k) for k, _ in _Stats._fields_ if k != "stage_ms"}
        d["stage_ms"] = list(s.stage_ms)
        return d


class Scheduler:
    """The server's host scheduler alone (no GPU needed)."""

    def __init__(self, base_hop: int, max_hop: int, capacity: int, max_out: int = 2,
                 arena_bytes: int = 1 << 30):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(self.lib.tvolap_sched_create(ctypes.byref(h), base_hop, max_hop, capacity,
                                                max_out, int(arena_bytes)), "tvolap_sched_create")
        self.h, self.capacity = h, capacity
        self._ids = np.zeros(capacity, np.int32)

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.tvolap_sched_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        return _lib.check(getattr(self.lib, name)(self.h, *args), name)

    @staticmethod
    def footprint(L, M, n_out, n_filters) -> int:
        b = ctypes.c_int64()
        _lib.check(_lib.load().tvolap_sched_footprint(L, M, n_out, n_filters, ctypes.byref(b)),
                   "tvolap_sched_footprint")
        return b.value

    def submit(self, L, M, n_out, n_filters) -> int:
        t = ctypes.c_int64()
        self._call("tvolap_sched_submit", L, M, n_out, n_filters, ctypes.byref(t))
        return t.value

    def pump(self) -> int:
        n = ctypes.c_int()
        self._call("tvolap_sched_pump", ctypes.byref(n))
        return n.value

    def cancel(self, ticket: int):
        self._call("tvolap_sched_cancel", ctypes.c_int64(ticket))

    def admitted(self) -> list:
        cap = 64
        t, i, w = np.zeros(cap, np.int64), np.zeros(cap, np.int32), np.zeros(cap, np.int64)
        n, out = ctypes.c_int(), []
        while True:
            self._call("tvolap_sched_admitted", t.ctypes.data_as(_lib.P_int64),
                       i.ctypes.data_as(_lib.P_int32), w.ctypes.data_as(_lib.P_int64), cap,
                       ctypes.byref(n))
            out += [(int(t[k]), int(i[k]), int(w[k])) for k in range(n.value)]
            if n.value < cap:
                return out

    def queue(self):
        w, o = ctypes.c_int(), ctypes.c_int64()
        self._call("tvolap_sched_queue", ctypes.byref(w), ctypes.byref(o))
        return w.value, o.value

    def admit(self, L, M, n_out, n_filters):
        i, off, ph = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        self._call("tvolap_sched_admit", L, M, n_out, n_filters, ctypes.byref(i),
                   ctypes.byref(off), ctypes.byref(ph))
        return i.value, off.value, ph.value

    def fail_admits(self, n: int):
        """Fault injection: the next n admissions with valid arguments are
        refused (TVOLAP_ERR_CAPACITY) and change nothing."""
        self._call("tvolap_sched_fail_admits", int(n))

    def activate(self, i):
        self._call("tvolap_sched_activate", int(i))

    def retire(self, i):
        self._call("tvolap_sched_retire", int(i))

    def due(self) -> np.ndarray:
        n = ctypes.c_int()
        self._call("tvolap_sched_due", self._ids.ctypes.data_as(_lib.P_int32), self.capacity,
                   ctypes.byref(n))
        return self._ids[:n.value].copy()

    def advance(self):
        self._call("tvolap_sched_advance")

    def phase_loads(self) -> np.ndarray:
        loads = np.zeros(8, np.int64)
        n = ctypes.c_int()
        self._call("tvolap_sched_phase_loads", loads.ctypes.data_as(_lib.P_int64), 8,
                   ctypes.byref(n))
        return loads[:n.value].copy()

    def arena(self):
        u, f = ctypes.c_int64(), ctypes.c_int64()
        self._call("tvolap_sched_arena", ctypes.byref(u), ctypes.byref(f))
        return u.value, f.value
