"""Many independent sources with different hops, impulse-response lengths and
signal lengths in a few launches.

Sources are grouped by hop L (the transform size); each group is one plan
whose channels are the group's sources, processed with
tvolap_process_ragged (per-channel lengths and partition counts). All plans
share one CUDA stream, so the whole batch can be captured once as a CUDA graph
and replayed. ``autotune`` picks the multiply-accumulate staging per group by
timing the variants on the batch itself.
"""
from __future__ import annotations

import numpy as np
import torch

from .tvolap import Plan, n_blocks_for


class HopGroup:
    def __init__(self, L, sources, index, device, stream):
        self.L, self.index = L, index
        n = len(sources)
        self.M = max(s.M for s in sources)
        n_slots = sum(s.irs.shape[0] for s in sources)
        self.plan = Plan(L, self.M, n_in=n, n_out=n, n_slots=n_slots, device=device, stream=stream)
        self.N = [s.x.shape[0] for s in sources]
        self.out_len = [s.out_len for s in sources]
        self.max_out = max(self.out_len)
        nb = n_blocks_for(self.max_out, L)
        xs = max(self.N)
        x = np.zeros((n, xs), np.float32)
        sched = np.zeros((n, nb), np.int32)
        slot0 = 0
        dev = device
        with torch.cuda.stream(stream):
            for c, s in enumerate(sources):
                x[c, :s.x.shape[0]] = s.x
                k = min(nb, s.sched.shape[0])
                sched[c, :k] = s.sched[:k] + slot0
                self.plan.load_bank(slot0, torch.from_numpy(s.irs).to(dev))
                slot0 += s.irs.shape[0]
            self.x = torch.from_numpy(x).to(dev)
            self.sched = torch.from_numpy(sched).to(dev)
            self.n = torch.tensor(self.N, dtype=torch.int64, device=dev)
            self.ol = torch.tensor(self.out_len, dtype=torch.int64, device=dev)
            self.parts = torch.tensor([s.M for s in sources], dtype=torch.int32, device=dev)
            self.y = torch.zeros((n, self.max_out), dtype=torch.float32, device=dev)

    def run(self):
        self.plan.process_ragged(self.x, self.n, self.ol, self.parts, self.max_out, self.sched,
                                 out=self.y)


class BatchedTvolap:
    """sources: objects with L, x [N], irs [n_ir, ir_len], sched [n_blocks]
    (index into irs per block, t = l + 1), out_len."""

    def __init__(self, sources, device=None):
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = torch.cuda.Stream(self.device)
        by_L = {}
        for i, s in enumerate(sources):
            by_L.setdefault(int(s.L), []).append(i)
        self.groups = []
        for L in sorted(by_L):
            idx = by_L[L]
            self.groups.append(HopGroup(L, [sources[i] for i in idx], idx, self.device,
                                        self.stream))
        self.n_sources = len(sources)
        self.graph = None
        torch.cuda.synchronize(self.device)

    def run(self):
        """Enqueue every group on the batch's stream."""
        for g in self.groups:
            g.run()

    def capture(self):
        """Record the whole batch as one CUDA graph (after one eager run, so
        every workspace already has its size)."""
        self.run()
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self.run()
        torch.cuda.synchronize(self.device)
        return self.graph

    def replay(self):
        """Replay the captured batch on the batch's stream."""
        if self.graph is None:
            self.capture()
        with torch.cuda.stream(self.stream):
            self.graph.replay()

    def output(self, i):
        """Output of source i (a view into its group's buffer)."""
        for g in self.groups:
            if i in g.index:
                c = g.index.index(i)
                return g.y[c, :g.out_len[c]]
        raise IndexError(i)

    def autotune(self, reps=3):
        """Per group, time the multiply-accumulate stagings on this batch (TMA
        groups of up to 3 or 4 filters, cp.async) and keep the fastest.
        Returns {L: (chosen option, ms per option)}."""
        chosen = {}
        for g in self.groups:
            times = []
            for opt in (0, 1, 2):
                g.plan.set_option(1, opt)
                g.run()
                torch.cuda.synchronize(self.device)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                for _ in range(reps):
                    g.run()
                e1.record(self.stream)
                torch.cuda.synchronize(self.device)
                times.append(e0.elapsed_time(e1) / reps)
            best = int(np.argmin(times))
            g.plan.set_option(1, best)
            chosen[g.L] = (best, times)
        self.graph = None                               # recapture with the chosen kernels
        return chosen
