"""Continuous-batching server for solve requests.

A request is a polynomial system (square; optionally with the constants of
its embedding for a top dimension D).  Requests are admitted as they arrive
and their work overlaps on the device:

* plain requests that arrived while earlier work runs are gathered into the
  next batch, and a batch is launched as soon as fewer than `max_inflight`
  batches are on the GPU: one phc_track_many call (one launch per number of
  unknowns, every warp on one request's system at a time), so small
  requests share launches that fill the GPU;
* an embedded request is cut into chunks of its top-stage paths;
  every chunk runs the top stage of E_D, then one phc_cascade_from per
  cascade stage, each fed directly by the previous stage's device outputs
  (Section 3.1: regular endpoints with a nonzero slack start the next
  stage), so a chunk's paths flow through every stage while later chunks
  are still waiting; with pipelined=True the top stage and the first
  cascade stage share one launch (phc_track_pipeline).

Small requests come first.  Batches run on high-priority streams, chunks on
low-priority ones (big_streams of them, each with handles of its own, since
calls on one handle must not overlap), and the server launches a chunk only
when a chunk stream is free: while small requests wait or run (or did within
idle_after seconds) one chunk at a time of big_chunk paths under a grid cap
of big_share_busy of the SMs, otherwise up to one chunk per chunk stream of
big_chunk_idle paths under big_share.  A
persistent launch keeps its SMs until its paths are done and the FP64 pipe
of an SM is shared by every warp resident on it, so it is this cap -- not
the stream priority alone -- that keeps most SMs for the small requests
while the large one advances on the rest; every chunk ends within about the
time of its longest path, so the cap follows the load.  Every path gives the
same result in any chunk and under any grid (a path's arithmetic does not
depend on the launch), so no result depends on the schedule.

Every unit of work ends with an event; the loop polls the events, copies the
classes and endpoints of finished work to the host, retires it (freeing its
memory budget) and launches waiting work.  Nothing waits on the host
between stages.  Latency is the time from a request's arrival to the moment
the server sees its results on the host.

All tracking runs in libphc.so; this module only schedules.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import _lib
from ._lib import (STATS_DTYPE, phc_cascade_from, phc_default_opts, phc_embed, phc_make_homotopy, phc_num_paths,
                   phc_track_many, phc_track_paths, phc_track_pipeline)


@dataclass
class Request:
    rid: int
    system: object            # n_eq, n_var, terms_per_eq, exps, coefs
    gamma: complex
    arrival: float = 0.0      # seconds after the start of the run
    top_dim: int = 0          # > 0: embedded request solved through the cascade to dimension 0
    gammas: np.ndarray | None = None   # [n_eq, top_dim]
    hyper: np.ndarray | None = None    # [top_dim, n_var + 1]


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    n_paths: int
    stages: list = field(default_factory=list)  # per stage: (x [n_var, P] complex, cls [P] int8)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def _bezout(system) -> int:
    """Product of the equations' total degrees (the number of start paths)."""
    e = np.asarray(system.exps, dtype=np.int64)
    tpe = np.asarray(system.terms_per_eq)
    off, P = 0, 1
    for m in tpe:
        P *= int(e[off:off + int(m)].sum(axis=1).max())
        off += int(m)
    return P


def _bytes_for(n_var: int, n_paths: int) -> int:
    return n_paths * (16 * n_var + 1 + 1 + STATS_DTYPE.itemsize)


class _Embedded:
    """An admitted embedded request: its systems E_D, ..., E_1 (host
    lists), per chunk stream its handles, and its chunks so far."""

    def __init__(self, req, systems, handles, n_paths, admitted, nbytes):
        self.req = req
        self.systems = systems
        self.handles = handles        # [stream][stage] phc_homotopy handles
        self.n_paths = n_paths
        self.admitted = admitted
        self.nbytes = nbytes
        self.next_first = 0
        self.chunks = []              # (first, per stage (x, cls) device outputs, event)
        self.pending = 0              # chunks launched and not yet finished

    @property
    def launched_all(self) -> bool:
        return self.next_first >= self.n_paths


class Server:
    def __init__(self, slots: int = 4, mem_bytes: int = 16 << 30, big_share: float = 1.0, opts=None,
                 device="cuda", max_inflight: int = 4, batch_paths: int = 60_000, pipelined: bool = False,
                 big_chunk: int = 2048, big_streams: int = 3, big_share_busy: float = 0.3,
                 big_chunk_idle: int = 16384, idle_after: float = 0.5):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.slots = slots                  # embedded requests admitted at once
        self.max_inflight = max_inflight    # batches of plain requests on the GPU at once
        self.batch_paths = batch_paths      # paths per batch (bounds a batch's duration)
        self.mem_bytes = mem_bytes
        self.big_share = big_share          # grid cap of a chunk when no small request waits or runs
        self.big_share_busy = big_share_busy  # ... and while small requests wait or run
        self.big_chunk = big_chunk          # top-stage paths per chunk while small requests wait or run
        self.big_chunk_idle = big_chunk_idle  # ... and when none do
        self.idle_after = idle_after        # seconds without small requests before chunks grow
        # embedded requests: the top stage and the first cascade stage in one
        # pipelined launch, or (default) one launch each, which lets both use
        # the tail hand-off
        self.pipelined = pipelined
        self.opts = opts if opts is not None else phc_default_opts()
        # lower number = higher priority: small requests first, chunks of large ones after
        self.batch_streams = [torch.cuda.Stream(device=self.device, priority=-100) for _ in range(max_inflight)]
        self.chunk_streams = [torch.cuda.Stream(device=self.device, priority=0) for _ in range(big_streams)]
        self.n_sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        self._keep = []  # handles of finished work, destroyed after the run

    def _opts(self):
        opts = phc_default_opts()
        for name, _ in _lib.phc_opts._fields_:
            setattr(opts, name, getattr(self.opts, name))
        return opts

    def plan_paths(self, req: Request) -> tuple[int, int]:
        """(paths of the top stage, bytes of device memory the plan needs)."""
        n = req.system.n_var + req.top_dim
        P = _bezout(req.system)
        return P, _bytes_for(n, P) * (1 + req.top_dim)

    @staticmethod
    def _download(stages):
        """Host copies of finished stages (called once the work's event fired)."""
        return [(x.cpu().numpy(), c.cpu().numpy()) for x, c in stages]

    def _launch_batch(self, reqs, stream):
        """Plain requests as one phc_track_many call on `stream`."""
        torch = self.torch
        with torch.cuda.stream(stream):
            hs = [phc_make_homotopy(r.system, r.gamma) for r in reqs]
            outs = []
            for h in hs:
                P = phc_num_paths(h)
                outs.append((torch.empty((h.n, P), dtype=torch.complex128, device=self.device),
                             torch.empty(P, dtype=torch.int8, device=self.device),
                             torch.empty((P, STATS_DTYPE.itemsize), dtype=torch.uint8, device=self.device)))
            phc_track_many(hs, self._opts(), [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs],
                           stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        return hs, [[(o[0], o[1])] for o in outs], ev, [phc_num_paths(h) for h in hs]

    def _admit_embedded(self, req: Request, admitted: float, nbytes: int) -> _Embedded:
        """The systems E_D, ..., E_1 of the request and, per chunk stream,
        handles of its own."""
        D = req.top_dim
        systems = [phc_embed(req.system, D, req.gammas, req.hyper)]
        for k in range(D - 1, 0, -1):
            systems.append(phc_embed(req.system, k, req.gammas[:, :k], req.hyper[:k]))
        handles = [[phc_make_homotopy(E, req.gamma) for E in systems] for _ in self.chunk_streams]
        return _Embedded(req, systems, handles, phc_num_paths(handles[0][0]), admitted, nbytes)

    def _launch_chunk(self, e: _Embedded, si: int, cap: float, chunk: int):
        """The next chunk of e on chunk stream si: the top stage, then every
        cascade stage from the device outputs of the stage above."""
        torch = self.torch
        opts = self._opts()
        if cap < 1.0:
            opts.max_blocks = max(1, int(cap * self.n_sms))
        D = e.req.top_dim
        first = e.next_first
        n = min(chunk, e.n_paths - first)
        e.next_first += n
        stream, hs = self.chunk_streams[si], e.handles[si]
        N = hs[0].n
        with torch.cuda.stream(stream):
            def buf(n_var):
                return (torch.empty((n_var, n), dtype=torch.complex128, device=self.device),
                        torch.empty(n, dtype=torch.int8, device=self.device),
                        torch.empty((n, STATS_DTYPE.itemsize), dtype=torch.uint8, device=self.device),
                        torch.empty(n, dtype=torch.uint8, device=self.device))

            xt, ct, stt, _ = buf(N)
            xn, cn, stn, szn = buf(N - 1)
            if self.pipelined:
                phc_track_pipeline(hs[0], D, first, n, opts, xt, ct, stt, xn, cn, szn, stn, stream)
            else:
                # top stage, then the first cascade stage from its device outputs
                # (each launch with its tail hand-off)
                phc_track_paths(hs[0], first, n, opts, xt, ct, stt, stream)
                phc_cascade_from(hs[0], D, xt, ct, None, n, opts, xn, cn, szn, stn, stream)
            stages = [(xt, ct), (xn, cn)]
            prev = (xn, cn, szn)
            for j, k in enumerate(range(D - 1, 0, -1)):
                hk = hs[j + 1]
                xo, co, sto, szo = buf(hk.n - 1)
                phc_cascade_from(hk, k, prev[0], prev[1], prev[2], n, opts, xo, co, szo, sto, stream)
                stages.append((xo, co))
                prev = (xo, co, szo)
            ev = torch.cuda.Event()
            ev.record(stream)
        e.chunks.append((first, stages, ev))
        e.pending += 1
        return ev

    @staticmethod
    def _download_chunks(e: _Embedded):
        """Host copies of a finished embedded request: per stage the chunks
        concatenated in path order."""
        chunks = sorted(e.chunks, key=lambda c: c[0])
        n_stages = len(chunks[0][1])
        return [(np.concatenate([c[1][s][0].cpu().numpy() for c in chunks], axis=1),
                 np.concatenate([c[1][s][1].cpu().numpy() for c in chunks])) for s in range(n_stages)]

    def run(self, requests, realtime: bool = True, poll: float = 2e-4):
        """Serve `requests` (arrival times relative to the start); returns
        the results in request order."""
        torch = self.torch
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        waiting = []                                   # arrived plain requests
        free_batch = list(range(self.max_inflight))
        free_chunk = list(range(len(self.chunk_streams)))
        chunk_busy = {}                                # chunk stream -> (embedded request, event)
        bigs = []                                      # admitted embedded requests
        mem_used = 0
        active = []   # batches: (slot, reqs, bytes, admitted, handles, host, event, n_paths)
        results = {}
        # last time a small request waited or ran; the session starts as if one
        # just had, so a large request arriving first begins with capped chunks
        # (small requests may follow it within idle_after seconds)
        last_small = 0.0
        t0 = time.perf_counter()
        while pending or waiting or active or bigs:
            now = time.perf_counter() - t0
            progressed = False
            for a in list(active):
                slot, reqs, nbytes, admitted, handles, host, ev, npaths = a
                if not ev.query():
                    continue
                fin = time.perf_counter() - t0
                for r, dev_stages, P in zip(reqs, host, npaths):
                    results[r.rid] = Result(r.rid, r.arrival, admitted, fin, P, self._download(dev_stages))
                free_batch.append(slot)
                self._keep.extend(handles)
                active.remove(a)
                mem_used -= nbytes
                progressed = True
            for si, (e, ev) in list(chunk_busy.items()):
                if not ev.query():
                    continue
                del chunk_busy[si]
                free_chunk.append(si)
                e.pending -= 1
                progressed = True
                if e.launched_all and e.pending == 0:
                    fin = time.perf_counter() - t0
                    r = e.req
                    results[r.rid] = Result(r.rid, r.arrival, e.admitted, fin, e.n_paths, self._download_chunks(e))
                    self._keep.extend(h for hs in e.handles for h in hs)
                    bigs.remove(e)
                    mem_used -= e.nbytes
            while pending and (pending[0].arrival <= now or not realtime):
                req = pending[0]
                if req.top_dim > 0:
                    _, nbytes = self.plan_paths(req)
                    if len(bigs) >= self.slots or ((active or bigs) and mem_used + nbytes > self.mem_bytes):
                        break
                    pending.pop(0)
                    bigs.append(self._admit_embedded(req, time.perf_counter() - t0, nbytes))
                    mem_used += nbytes
                else:
                    waiting.append(pending.pop(0))
                progressed = True
            if waiting and free_batch:
                batch, nbytes, npath = [], 0, 0
                while waiting:
                    P, b = self.plan_paths(waiting[0])
                    if batch and (mem_used + nbytes + b > self.mem_bytes or npath + P > self.batch_paths):
                        break
                    npath += P
                    nbytes += b
                    batch.append(waiting.pop(0))
                slot = free_batch.pop(0)
                admitted = time.perf_counter() - t0
                hs, host, ev, npaths = self._launch_batch(batch, self.batch_streams[slot])
                active.append((slot, batch, nbytes, admitted, hs, host, ev, npaths))
                mem_used += nbytes
                progressed = True
            # chunks of embedded requests (first admitted first) on free chunk streams
            if waiting or active:
                last_small = now
            busy = now - last_small < self.idle_after
            for e in bigs:
                # while small requests are served one chunk at a time runs (the cap
                # bounds the SMs of all chunks together), otherwise one per chunk stream
                while free_chunk and not e.launched_all and not (busy and chunk_busy):
                    si = free_chunk.pop(0)
                    chunk_busy[si] = (e, self._launch_chunk(e, si, self.big_share_busy if busy else self.big_share,
                                                            self.big_chunk if busy else self.big_chunk_idle))
                    progressed = True
            if not progressed:
                time.sleep(poll)
        torch.cuda.synchronize(self.device)
        self._keep.clear()
        return [results[r.rid] for r in requests]


def solve_alone(req: Request, opts=None, device="cuda") -> Result:
    """The same plan for one request on an otherwise idle device."""
    srv = Server(slots=1, opts=opts, device=device, max_inflight=1)
    r = Request(req.rid, req.system, req.gamma, 0.0, req.top_dim, req.gammas, req.hyper)
    return srv.run([r], realtime=False)[0]


def latency_summary(results, rids=None) -> dict:
    lat = np.array([r.latency for r in results if rids is None or r.rid in rids])
    if lat.size == 0:
        return {"count": 0}
    return {"count": int(lat.size), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "max_s": float(lat.max())}
