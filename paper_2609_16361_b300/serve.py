"""Continuous-batching serving loop for simulation requests (Sod / Becker tubes, Taylor-Green
boxes, FP32 or FP16 storage, different step counts).

Requests arrive over time.  A request is admitted as soon as its populations fit in the HBM
budget (FIFO, head of line waits) and a slot is free; its domain is created and initialised
on the device and stays resident until it finishes.  Resident domains advance together,
`chunk` steps at a time, so a request that arrives while others run joins at the next chunk
boundary.  Per chunk every small resident domain advances (one batch call: under the default
schedule each domain replays its own single-domain sweeps from a CUDA graph, the domains spread
over concurrent streams; the table schedules share one launch per step and storage/collision
group), and of the large ones (each fills the GPU on its own) only the one with the least
remaining work (cells x steps) — shortest-remaining-work-first, so short large requests are not
held behind long ones.  A finished request's conserved fields are read back and its memory is
released, which may admit waiting requests.

With one_buffer_large, large requests keep one population buffer (AA pattern: half their
memory, the same traffic and collisions); small ones stay two-buffer for the batched kernel.
With moments, FP32 requests of the regularized collision keep their state as the 20 moments of
each cell's outgoing set (160 instead of 280 bytes per cell update, bitwise the same run); they
advance by their own sweeps in every schedule.

A domain's result does not depend on which other domains share its launches, so every
request's result is bitwise the same alone and in the mix.

Failure detection: after every chunk each advanced request's state is scanned for non-finite
populations (grlb_check_finite, a read-only pass of about half a sweep's traffic, into a
page-locked flag the host reads once the chunk has run).  A request whose state went non-finite
is evicted at once -- its memory is released and it is reported with status "nonfinite" --
while the others continue unchanged (their launches never read another domain's memory).  A
request that finishes in the chunk where it blew up is caught by its readback instead.  `serial_plain` is the baseline:
the same trace first-in first-out, one domain at a time, one single-domain launch per step.
"""
from __future__ import annotations

import collections
import hashlib
import time
from dataclasses import dataclass, field

import numpy as np

from . import autotune, capi
from . import inputs as _inputs


@dataclass
class Result:
    rid: int
    kind: str
    steps: int
    cells: int
    arrival: float
    admitted: float = 0.0
    finished: float = 0.0
    digest: str = ""
    status: str = "ok"        # "ok", or "nonfinite" (evicted or read back with NaN / inf)
    totals: np.ndarray = field(default_factory=lambda: np.zeros(5))
    fields: np.ndarray | None = None  # conserved fields, kept only when asked for

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def _finish(res: Result, dom: capi.Domain, t0: float, keep: bool):
    Q = dom.conserved()
    res.finished = time.perf_counter() - t0
    res.digest = hashlib.sha256(Q.tobytes()).hexdigest()
    res.totals = Q.sum(axis=1)
    if not np.isfinite(Q).all():
        res.status = "nonfinite"
    if keep:
        res.fields = Q


class Server:
    def __init__(self, hbm_budget: float = 150e9, max_resident: int = 512, chunk: int = 200,
                 use_graph: bool = True, tile_table: dict | None = None, stream=None,
                 keep_fields: bool = False, large_cells: int = 262144, srpt: bool = True,
                 one_buffer_large: bool = False, check_finite: bool = True, moments: bool = False):
        import torch
        self.budget = float(hbm_budget)
        self.max_resident = max_resident
        self.chunk = chunk
        self.use_graph = use_graph
        self.tile_table = tile_table or {}
        self.stream = stream or torch.cuda.Stream()
        self.peak_bytes = 0
        self.peak_resident = 0
        self.launch_steps = 0
        self.keep_fields = keep_fields
        self.large_cells = large_cells  # same threshold as the batch's solo_min_cells
        self.srpt = srpt
        # large requests with one population buffer (AA pattern): half their memory, same
        # traffic; small ones run in the batched kernel, which needs two buffers
        self.one_buffer_large = one_buffer_large
        self.check_finite = check_finite  # scan every advanced request after each chunk
        self.moments = moments  # FP32 regularized requests keep their state as moments
        self.evicted = 0

    def run(self, trace, realtime: bool = True, lookahead: int = 12):
        """Serve `trace` (list of inputs.Request sorted by arrival).  Returns Results in
        request order.  realtime=False admits every request at t = 0 (closed-loop).

        The host never waits for the chunk it just enqueued: up to `lookahead` chunks are in
        flight; new requests are created and their fields uploaded (copy stream) behind them;
        finished requests are read back by a worker thread on a readback stream that waits only
        for the event of the chunk they finished in."""
        import queue
        import threading

        import torch
        st = self.stream.cuda_stream
        rstream = torch.cuda.Stream()
        pending = collections.deque(sorted(trace, key=lambda r: r.arrival))
        waiting = collections.deque()
        resident = []   # [req, dom, remaining, bytes, Result]
        results = {}
        lock = threading.Lock()
        state = {"used": 0.0, "draining": 0, "error": None}
        inflight = collections.deque()
        checks = collections.deque()  # (event, page-locked flags, [(slot, resident entry)])
        batch = None
        mask = None
        dirty = True
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        host = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        todo = queue.Queue()

        def reader():
            while True:
                item = todo.get()
                if item is None:
                    return
                entries, ev, failed = item
                try:
                    rstream.wait_event(ev)
                    for r, dom, _, need, res in entries:
                        capi.grlb_set_stream(dom.h, rstream.cuda_stream)
                        if not failed:   # evicted requests are not read back
                            _finish(res, dom, t0, self.keep_fields)
                        dom.close()
                        with lock:
                            results[r.rid] = res
                            state["used"] -= need
                            state["draining"] -= 1
                except Exception as e:  # surfaced by the main loop
                    with lock:
                        state["error"] = e
                        state["draining"] -= len(entries)

        def failed_entries(block: bool):
            """Resident entries whose finiteness flag is set, from the checks that have run."""
            bad = []
            while checks and (block or checks[0][0].query()):
                cev, flags, entries = checks.popleft()
                cev.synchronize()
                f = flags.numpy()
                for slot, x in entries:
                    if f[slot] and any(y is x for y in resident) and not any(y is x for y in bad):
                        bad.append(x)
            return bad

        worker = threading.Thread(target=reader, daemon=True)
        worker.start()
        try:
            while True:
                bad = failed_entries(block=False)
                if bad:
                    # the batch lists the failed domains: destroy it before they are released;
                    # their memory is freed after everything already enqueued that touches them
                    if batch is not None:
                        capi.grlb_batch_destroy(batch)
                        batch = None
                    fev = torch.cuda.Event()
                    fev.record(self.stream)
                    for x in bad:
                        x[4].status = "nonfinite"
                        x[4].finished = now()
                    resident = [x for x in resident if not any(x is y for y in bad)]
                    self.evicted += len(bad)
                    with lock:
                        state["draining"] += len(bad)
                    todo.put((bad, fev, True))
                    dirty = True
                with lock:
                    if state["error"] is not None:
                        raise state["error"]
                    used, draining = state["used"], state["draining"]
                if not (pending or waiting or resident or draining):
                    break
                t = now()
                while pending and (not realtime or pending[0].arrival <= t):
                    waiting.append(pending.popleft())
                # admission: FIFO while the head fits in the budget and a slot is free
                while waiting and len(resident) < self.max_resident:
                    r = waiting[0]
                    prm = request_params(r, self.large_cells, self.one_buffer_large, self.moments)
                    need = capi.grlb_bytes_for(prm)
                    if need == 0:
                        raise capi.GrlbError(-1, f"request {r.rid}: invalid parameters")
                    with lock:
                        used = state["used"]
                        draining = state["draining"]
                    if used + need > self.budget:
                        if not resident and not draining:
                            raise capi.GrlbError(-2, f"request {r.rid} needs {need} B > budget")
                        break
                    waiting.popleft()
                    dom = capi.Domain(prm, stream=st)
                    capi.grlb_stage_primitive(dom.h, host(r.case.rho), host(r.case.u), host(r.case.p))
                    capi.grlb_init_from_stage(dom.h)
                    res = Result(r.rid, r.kind, r.steps, r.case.params.ncells,
                                 r.arrival if realtime else 0.0, admitted=now())
                    resident.append([r, dom, r.steps, need, res])
                    with lock:
                        state["used"] += need
                        self.peak_bytes = max(self.peak_bytes, state["used"])
                    dirty = True
                self.peak_resident = max(self.peak_resident, len(resident))
                if not resident:
                    if waiting or draining:
                        time.sleep(0.0005)   # memory comes back as the reader finishes
                    elif pending:
                        time.sleep(max(0.0, pending[0].arrival - now()))
                    continue
                if dirty:
                    if batch is not None:
                        capi.grlb_batch_destroy(batch)
                    batch = capi.grlb_batch_create([x[1].h for x in resident],
                                                   use_graph=int(self.use_graph),
                                                   solo_min_cells=self.large_cells)
                    capi.grlb_batch_set_stream(batch, st)
                    if self.tile_table:
                        capi.grlb_batch_set_tile_x(
                            batch, autotune.plan([x[0].case for x in resident], self.tile_table))
                    mask = None
                    dirty = False
                # every small domain; of the large ones the least remaining work first
                large = [i for i, x in enumerate(resident) if x[1].N >= self.large_cells]
                pick = set(range(len(resident)))
                if self.srpt and len(large) > 1:
                    keep = min(large, key=lambda i: resident[i][1].N * resident[i][2])
                    pick -= set(large) - {keep}
                new_mask = [1 if i in pick else 0 for i in range(len(resident))]
                if new_mask != mask:
                    capi.grlb_batch_set_active(batch, new_mask)
                    mask = new_mask
                k = min(self.chunk, min(resident[i][2] for i in pick))
                capi.grlb_batch_step(batch, k)
                self.launch_steps += k
                flags = None
                if self.check_finite:
                    flags = torch.zeros(len(resident), dtype=torch.int32, pin_memory=True)
                    for i in pick:
                        capi.grlb_check_finite(resident[i][1].h, flags.data_ptr() + 4 * i)
                ev = torch.cuda.Event()
                ev.record(self.stream)
                inflight.append(ev)
                if flags is not None:
                    checks.append((ev, flags, [(i, resident[i]) for i in pick]))
                for i in pick:
                    resident[i][2] -= k
                done = [x for x in resident if x[2] == 0]
                if done:
                    # the batch lists these domains and reads their state when destroyed, so it
                    # goes first; the reader thread closes the domains afterwards
                    capi.grlb_batch_destroy(batch)
                    batch = None
                    with lock:
                        state["draining"] += len(done)
                    todo.put((done, ev, False))
                    resident = [x for x in resident if x[2] > 0]
                    dirty = True
                while len(inflight) > lookahead:
                    inflight.popleft().synchronize()
        finally:
            todo.put(None)
            worker.join()
            torch.cuda.synchronize()
            if batch is not None:
                capi.grlb_batch_destroy(batch)
            for x in resident:
                x[1].close()
        return [results[r.rid] for r in sorted(trace, key=lambda r: r.rid)]


def request_params(r, large_cells: int, one_buffer_large: bool, moments: bool = False):
    """Domain parameters of a request: with `moments`, FP32 requests of the regularized
    collision keep their state as moments (streaming 2: 20 values per cell, bitwise the same
    run); otherwise one population buffer for large requests if asked."""
    prm = r.case.params
    if moments and prm.storage == _inputs.STORE_F32 and prm.collision == _inputs.COLL_RLB_SENSOR:
        return prm.replace(streaming=2)
    if one_buffer_large and prm.ncells >= large_cells:
        return prm.replace(streaming=1)
    return prm


def serial_plain(trace, realtime: bool = True, stream=None, keep_fields: bool = False,
                 one_buffer_large: bool = False, large_cells: int = 262144, moments: bool = False):
    """Baseline: first-in first-out, one domain at a time through grlb_step on `stream` (no
    batching; grlb_step replays a small domain's sweeps from a CUDA graph of 8 launches); the
    same buffer choice per request as the server's."""
    import torch
    stream = stream or torch.cuda.Stream()
    st = stream.cuda_stream
    out = []
    t0 = time.perf_counter()
    for r in sorted(trace, key=lambda r: r.arrival):
        if realtime:
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        res = Result(r.rid, r.kind, r.steps, r.case.params.ncells, r.arrival if realtime else 0.0,
                     admitted=time.perf_counter() - t0)
        dom = capi.Domain(request_params(r, large_cells, one_buffer_large, moments), stream=st)
        dom.init(r.case.rho, r.case.u, r.case.p)
        dom.step(r.steps)
        _finish(res, dom, t0, keep_fields)
        dom.close()
        out.append(res)
    return sorted(out, key=lambda x: x.rid)


def summarize(results, t_span: float | None = None) -> dict:
    """Throughput and latency over all requests (a failed request counts with the time it was
    reported); `failed` counts the requests with a non-finite state."""
    lat = np.array([r.latency for r in results])
    span = t_span if t_span is not None else max(r.finished for r in results) - min(
        r.arrival for r in results)
    cells = sum(r.cells * r.steps for r in results)
    return {"solves": len(results), "solves_per_s": len(results) / span,
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "span_s": span,
            "mlups": cells / span / 1e6, "failed": sum(r.status != "ok" for r in results)}
