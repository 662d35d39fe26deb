"""Continuous-batching server for SpKAdd requests.

Each request is one independent problem B = A_1 + ... + A_k (its own k,
shape and dtype) whose inputs are already on the device.  The server admits
queued requests into a batch while the batch's device memory fits the budget,
runs the batch through the batched C ABI (one set of kernel launches for all
its problems), and starts the next batch while earlier ones still run:
batches rotate over a few CUDA streams, so a batch's symbolic phase -- the
one host synchronisation -- overlaps the other streams' work.  A batch stops
taking requests once it holds enough work (input nonzeros) to amortise its
launches, so small requests share launches and large ones run alone.

Admission is by device memory, in two steps.  A request joins a batch when
its bound fits the budget: workspace plus an output no larger than its
input (nnz(B) <= sum_i nnz(A_i), Sec. II-A).  After the batch's symbolic
phase (Sec. II-D: the exact nnz(B) of every request) the charge drops to the
outputs' exact size before they are allocated, so the memory a request does
not need goes back to admission at once.  Outputs are one flat buffer per
array and dtype for the whole batch.

Latency is arrival to outputs complete: the completion time of a request is
its batch's completion event, placed on a common time line with the arrival
clock.  With ``batching=False`` every request runs alone (one batch of one),
the one-launch-set-per-request baseline.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (default_options, spkadd_batch_numeric_raw, spkadd_batch_plan_raw, spkadd_batch_symbolic,
               spkadd_destroy, spkadd_get_info)

__all__ = ["Request", "Server", "ServeStats", "output_digest"]


@dataclass
class Request:
    """One SpKAdd problem: inputs (col_ptr, row_idx, val) on the device, m rows."""

    rid: int
    A: list
    m: int
    arrival: float = 0.0          # seconds after the start of the trace
    tag: int = -1                 # caller's label (e.g. the input pool entry)
    done: float = float("nan")    # completion time on the same clock
    out: tuple | None = None      # (col_ptr int64, row_idx int32, val) views
    nnz_out: int = -1
    batch_id: int = -1
    _desc: dict = field(default_factory=dict, repr=False)

    def __post_init__(self):
        k = len(self.A)
        cp, ri, va = self.A[0]
        self.n = cp.numel() - 1
        self.dtype = va.dtype
        self.k = k
        nnz = np.asarray([a[1].numel() for a in self.A], dtype=np.int64)
        self.nnz_in = int(nnz.sum())
        self._desc = dict(
            nnz=nnz,
            cp=np.asarray([a[0].data_ptr() for a in self.A], dtype=np.uint64),
            ri=np.asarray([a[1].data_ptr() if a[1].numel() else 0 for a in self.A], dtype=np.uint64),
            va=np.asarray([a[2].data_ptr() if a[2].numel() else 0 for a in self.A], dtype=np.uint64))

    def bytes_bound(self) -> int:
        """An upper bound of the device bytes the request may need while in flight: B <= inputs
        (nnz(B) <= sum_i nnz(A_i), Sec. II-A), plus workspace."""
        sv = self.A[0][2].element_size()
        return self.nnz_in * (4 + sv) + (self.n + 1) * 8 + self.workspace_bytes()

    def workspace_bytes(self) -> int:
        """An estimate of the planner's workspace for the request: per-column and per-input tables, and the
        thread-block item records, bounded as the library bounds them for the default class limits (512 /
        4096 / 4096), at 52 bytes each (record, search row and the copy grouped by problem kind).  After the
        symbolic phase the server charges the batch's actual workspace instead."""
        slabs = max(1, -(-self.m // (1 << 20)))
        heavy = min(self.n, self.nnz_in // 4097)
        cta = min(self.n, self.nnz_in // 513)
        items = self.nnz_in // 4032 + heavy * (slabs + 1) + cta + 16
        return 48 * self.n + 64 * self.k + 52 * items + 4096

    def output_bytes(self, nnz_out: int) -> int:
        """B's exact size once the symbolic phase has given nnz(B)."""
        return (self.n + 1) * 8 + nnz_out * (4 + self.A[0][2].element_size())


@dataclass
class ServeStats:
    requests: int
    batches: int
    seconds: float
    nnz_in: int
    latencies: list

    def pct(self, p: float) -> float:
        lat = sorted(self.latencies)
        if not lat:
            return float("nan")
        return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]

    def summary(self) -> dict:
        return {"requests": self.requests, "batches": self.batches, "seconds": self.seconds,
                "nnz_per_s": self.nnz_in / self.seconds if self.seconds > 0 else None,
                "requests_per_s": self.requests / self.seconds if self.seconds > 0 else None,
                "p50_ms": self.pct(50) * 1e3, "p99_ms": self.pct(99) * 1e3, "max_ms": max(self.latencies) * 1e3,
                "mean_batch": self.requests / max(self.batches, 1)}


class _Batch:
    def __init__(self, reqs, handle, bufs, event, stream, charged):
        self.reqs = reqs
        self.handle = handle
        self.bufs = bufs
        self.event = event
        self.stream = stream
        self.charged = charged


class Server:
    """Continuous batching over the batched C ABI.

    mem_budget   device bytes the in-flight batches may hold (outputs and
                 workspace; the inputs are the caller's)
    max_batch    most requests in one batch
    max_batch_nnz  most input nonzeros in a batch (its first request is
                 always taken): small requests share launches, large ones run
                 alone and pipeline across streams
    batching     False: every request is its own batch (baseline)
    on_done      optional callback(request) run when a request's batch has
                 completed, with request.out set to its output views (they
                 are released after the callback); it runs on the serving
                 thread, so it delays the loop
    """

    def __init__(self, device, mem_budget: int, max_batch: int = 4096, batching: bool = True, options=None,
                 on_done=None, streams: int = 3, max_batch_nnz: int = 1 << 25):
        self.device = torch.device(device)
        self.mem_budget = int(mem_budget)
        self.max_batch = max_batch if batching else 1
        self.max_batch_nnz = max_batch_nnz
        self.options = options if options is not None else default_options()
        self.on_done = on_done
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(max(1, streams))]

    # -- one batch -----------------------------------------------------------
    def _start(self, reqs, stream, charged):
        desc = [r._desc for r in reqs]
        k = np.asarray([r.k for r in reqs], dtype=np.int32)
        h = spkadd_batch_plan_raw(k, [r.m for r in reqs], [r.n for r in reqs],
                                  np.concatenate([d["nnz"] for d in desc]), np.concatenate([d["cp"] for d in desc]),
                                  np.concatenate([d["ri"] for d in desc]), np.concatenate([d["va"] for d in desc]),
                                  [r.dtype for r in reqs], stream=stream, options=self.options, device=self.device)
        nnz = np.asarray(spkadd_batch_symbolic(h), dtype=np.int64)
        # The outputs' exact size and the batch's actual workspace (with the per-input offsets of split
        # windows, sized by the symbolic phase) replace their bounds in the charge before the outputs are
        # allocated.
        ws = int(spkadd_get_info(h)["workspace_bytes"])
        slack = sum(r.bytes_bound() - r.output_bytes(int(z)) for r, z in zip(reqs, nnz)) - ws
        self._used -= slack
        charged -= slack
        n1 = np.asarray([r.n + 1 for r in reqs], dtype=np.int64)
        is64 = np.asarray([r.dtype == torch.float64 for r in reqs])
        with torch.cuda.stream(stream):
            cp = torch.empty(int(n1.sum()), dtype=torch.int64, device=self.device)
            ri = torch.empty(max(int(nnz.sum()), 1), dtype=torch.int32, device=self.device)
            v64 = torch.empty(max(int(nnz[is64].sum()), 1), dtype=torch.float64, device=self.device)
            v32 = torch.empty(max(int(nnz[~is64].sum()), 1), dtype=torch.float32, device=self.device)

        def offs(sizes):
            o = np.zeros(sizes.size, dtype=np.int64)
            o[1:] = np.cumsum(sizes[:-1])
            return o

        o_cp, o_ri = offs(n1), offs(nnz)
        o_va = np.zeros(len(reqs), dtype=np.int64)
        o_va[is64] = offs(nnz[is64])
        o_va[~is64] = offs(nnz[~is64])
        a_cp = np.uint64(cp.data_ptr()) + o_cp.astype(np.uint64) * np.uint64(8)
        a_ri = np.uint64(ri.data_ptr()) + o_ri.astype(np.uint64) * np.uint64(4)
        a_va = np.where(is64, np.uint64(v64.data_ptr()) + o_va.astype(np.uint64) * np.uint64(8),
                        np.uint64(v32.data_ptr()) + o_va.astype(np.uint64) * np.uint64(4)).astype(np.uint64)
        spkadd_batch_numeric_raw(h, a_cp, a_ri, a_va)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        for q, r in enumerate(reqs):
            r.nnz_out = int(nnz[q])
            if self.on_done is not None:
                vb = v64 if is64[q] else v32
                r.out = (cp[o_cp[q]:o_cp[q] + n1[q]], ri[o_ri[q]:o_ri[q] + nnz[q]], vb[o_va[q]:o_va[q] + nnz[q]])
        return _Batch(reqs, h, (cp, ri, v64, v32), ev, stream, charged)

    def _finish(self, b, t0_event, t0_host):
        t = t0_host + t0_event.elapsed_time(b.event) / 1e3
        for r in b.reqs:
            r.done = t
        spkadd_destroy(b.handle)
        if self.on_done is not None:
            for r in b.reqs:
                self.on_done(r)
                r.out = None
        b.bufs = None

    # -- a trace ---------------------------------------------------------------
    def run(self, requests) -> ServeStats:
        """Serve `requests` (sorted by arrival, seconds from now) in real time."""
        with torch.cuda.device(self.device):  # the C library launches on the current device
            return self._run(requests)

    def _run(self, requests) -> ServeStats:
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue = collections.deque()
        self._inflight = collections.deque()
        self._used = 0
        self.peak_charged = 0
        nb = 0
        torch.cuda.synchronize(self.device)
        t0_event = torch.cuda.Event(enable_timing=True)
        t0_event.record(torch.cuda.current_stream(self.device))
        t0_event.synchronize()
        self._t0_event = t0_event
        t0 = time.perf_counter()
        inflight = self._inflight
        while pending or queue or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            while inflight and inflight[0].event.query():
                b = inflight.popleft()
                self._finish(b, t0_event, 0.0)
                self._used -= b.charged
            if queue and len(inflight) < len(self.streams):
                take, charge, work = [], 0, 0
                while queue and len(take) < self.max_batch:
                    if take and work + queue[0].nnz_in > self.max_batch_nnz:
                        break  # a large request runs in a batch of its own
                    c = queue[0].bytes_bound()
                    if take and self._used + charge + c > self.mem_budget:
                        break
                    if not take and inflight and self._used + c > self.mem_budget:
                        break  # wait for memory to come back
                    take.append(queue.popleft())
                    charge += c
                    work += take[-1].nnz_in
                if take:
                    stream = self.streams[nb % len(self.streams)]
                    for r in take:
                        r.batch_id = nb
                    self._used += charge
                    self.peak_charged = max(self.peak_charged, self._used)
                    inflight.append(self._start(take, stream, charge))
                    nb += 1
                    continue
            # nothing to start: wait for the next arrival or the oldest batch
            if inflight:
                if pending and not queue:
                    dt = pending[0].arrival - (time.perf_counter() - t0)
                    if dt > 0 and not inflight[0].event.query():
                        time.sleep(min(dt, 2e-4))
                else:
                    inflight[0].event.synchronize()
            elif pending:
                dt = pending[0].arrival - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
        total = max(r.done for r in requests) if requests else 0.0
        lat = [r.done - r.arrival for r in requests]
        return ServeStats(len(requests), nb, total, sum(r.nnz_in for r in requests), lat)


def output_digest(out) -> tuple:
    """(col_ptr hash, row_idx hash, sum of values, sum of |values|) of one output; indices hash exactly."""
    cp, ri, va = out
    w_cp = torch.arange(1, cp.numel() + 1, device=cp.device, dtype=torch.int64)
    w_ri = torch.arange(1, ri.numel() + 1, device=ri.device, dtype=torch.int64)
    h_cp = int((cp * w_cp).sum())
    h_ri = int((ri.to(torch.int64) * w_ri).sum()) if ri.numel() else 0
    v = va.to(torch.float64)
    return h_cp, h_ri, float(v.sum()), float(v.abs().sum())
