"""Continuous-batching server for solve requests.

A request is a polynomial system (square; optionally with the constants of
its embedding for a top dimension D).  Requests are admitted as they arrive
and their work overlaps on the device:

* plain requests that arrived while earlier work runs are gathered into the
  next batch, and a batch is launched as soon as fewer than `max_inflight`
  batches are on the GPU: one phc_track_many call (one launch per number of
  unknowns, every warp on one request's system at a time), so small
  requests share launches that fill the GPU;
* an embedded request runs on a stream of its own as soon as it arrives:
  the top stage of E_D, then one phc_cascade_from per cascade stage, each
  fed directly by the previous stage's device outputs (Section 3.1: regular
  endpoints with a nonzero slack start the next stage); with pipelined=True
  the top stage and the first cascade stage share one launch
  (phc_track_pipeline).  It gets a grid cap (big_share of the SMs) so that
  batches of small requests keep SMs.

Every unit of work ends with an event; the loop polls the events, copies the
classes and endpoints of finished work to the host, retires it (freeing its
memory budget) and launches waiting work.  Nothing waits on the
host between stages.  Latency is the time from a request's arrival to the
moment the server sees its results on the host.

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


class Server:
    def __init__(self, slots: int = 4, mem_bytes: int = 16 << 30, big_share: float = 0.6, opts=None,
                 device="cuda", max_inflight: int = 4, batch_paths: int = 60_000, pipelined: bool = False):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.slots = slots                  # streams for embedded requests
        self.max_inflight = max_inflight    # batches of plain requests on the GPU at once
        self.batch_paths = batch_paths      # paths per batch (bounds a batch's duration)
        self.mem_bytes = mem_bytes
        self.big_share = big_share
        # embedded requests: the top stage and the first cascade stage in one
        # pipelined launch, or (default) one launch each, which lets both use
        # the tail hand-off
        self.pipelined = pipelined
        self.opts = opts if opts is not None else phc_default_opts()
        self.batch_streams = [torch.cuda.Stream(device=self.device) for _ in range(max_inflight)]
        self.big_streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
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

    def _launch_embedded(self, req: Request, stream):
        torch = self.torch
        opts = self._opts()
        handles, stages = [], []
        with torch.cuda.stream(stream):
            D = req.top_dim
            E = phc_embed(req.system, D, req.gammas, req.hyper)
            h = phc_make_homotopy(E, req.gamma)
            handles.append(h)
            P = phc_num_paths(h)
            opts.max_blocks = max(1, int(self.big_share * self.n_sms))
            N = h.n

            def buf(n_var):
                return (torch.empty((n_var, P), dtype=torch.complex128, device=self.device),
                        torch.empty(P, dtype=torch.int8, device=self.device),
                        torch.empty((P, STATS_DTYPE.itemsize), dtype=torch.uint8, device=self.device),
                        torch.empty(P, dtype=torch.uint8, device=self.device))

            xt, ct, stt, _ = buf(N)
            xn, cn, stn, szn = buf(N - 1)
            if self.pipelined:
                phc_track_pipeline(h, D, 0, P, opts, xt, ct, stt, xn, cn, szn, stn, stream)
            else:
                # top stage, then the first cascade stage from its device outputs
                # (each launch with its tail hand-off)
                phc_track_paths(h, 0, P, opts, xt, ct, stt, stream)
                phc_cascade_from(h, D, xt, ct, None, P, opts, xn, cn, szn, stn, stream)
            stages += [(xt, ct), (xn, cn)]
            prev = (xn, cn, szn)
            for k in range(D - 1, 0, -1):
                Ek = phc_embed(req.system, k, req.gammas[:, :k], req.hyper[:k])
                hk = phc_make_homotopy(Ek, req.gamma)
                handles.append(hk)
                xo, co, sto, szo = buf(hk.n - 1)
                phc_cascade_from(hk, k, prev[0], prev[1], prev[2], P, opts, xo, co, szo, sto, stream)
                stages.append((xo, co))
                prev = (xo, co, szo)
            ev = torch.cuda.Event()
            ev.record(stream)
        return handles, stages, ev, P

    def run(self, requests, realtime: bool = True, poll: float = 2e-4):
        """Serve `requests` (arrival times relative to the start); returns
        the results in request order."""
        torch = self.torch
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        waiting = []                                   # arrived plain requests
        free_batch = list(range(self.max_inflight))
        free_big = list(range(self.slots))
        mem_used = 0
        active = []   # (kind, slot, reqs, bytes, admitted, handles, host, event, n_paths)
        results = {}
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            progressed = False
            for a in list(active):
                kind, slot, reqs, nbytes, admitted, handles, host, ev, npaths = a
                if not ev.query():
                    continue
                if kind == "batch":
                    for r, dev_stages, P in zip(reqs, host, npaths):
                        results[r.rid] = Result(r.rid, r.arrival, admitted, 0.0, P, self._download(dev_stages))
                    free_batch.append(slot)
                else:
                    r = reqs[0]
                    results[r.rid] = Result(r.rid, r.arrival, admitted, 0.0, npaths, self._download(host))
                    free_big.append(slot)
                fin = time.perf_counter() - t0
                for r in reqs:
                    results[r.rid].finished = fin
                self._keep.extend(handles)
                active.remove(a)
                mem_used -= nbytes
                progressed = True
            while pending and (pending[0].arrival <= now or not realtime):
                req = pending[0]
                if req.top_dim > 0:
                    _, nbytes = self.plan_paths(req)
                    if not free_big or (active and mem_used + nbytes > self.mem_bytes):
                        break
                    pending.pop(0)
                    slot = free_big.pop(0)
                    admitted = time.perf_counter() - t0
                    handles, host, ev, P = self._launch_embedded(req, self.big_streams[slot])
                    active.append(("big", slot, [req], nbytes, admitted, handles, host, ev, P))
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
                active.append(("batch", slot, batch, nbytes, admitted, hs, host, ev, npaths))
                mem_used += nbytes
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
