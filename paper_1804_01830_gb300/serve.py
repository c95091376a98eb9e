"""Continuous-batching stress server on one GPU.

Requests (grid geometry, dislocation families, densities) arrive at any time from
any thread.  A scheduler thread

  * keeps one built context per (geometry, family set) in a cache, so the kernel
    spectra of a geometry stay resident in HBM and are built once (Sec. 2.3: the
    coefficients are computed once per geometry).  A request may carry densities for
    a subset of the context's families only (``fam``): Eq. 3b sums over the families
    present and the coefficients are linear in b, so one context per geometry serves
    every subset (dds_stress_subset).  Idle contexts are evicted, least recently used
    first, when the HBM budget needs room;
  * admits a request when its device footprint fits the budget: the context (computed
    from its plan before it is built, dds_footprint) if not yet resident, plus the
    request's density and stress buffers;
  * evaluates the waiting requests of one context and family subset together (one
    call, the spectra read once), and runs different contexts on different CUDA
    streams, so work admitted while other work is on the GPU overlaps with it;
  * returns results through futures and records, per request, the latency (submission
    to result on the host) and its parts: queueing before launch, host-to-device copy,
    device evaluation and device-to-host copy (CUDA events on the request's stream).

A context has one set of work buffers, so at most one evaluation per context is in
flight; requests for a busy context wait while other contexts proceed.
"""
from __future__ import annotations

import queue
import threading
import time
from collections import OrderedDict
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import StressContext


@dataclass(eq=False)
class StressRequest:
    grid: tuple            # (nx, ny, nz)
    cells: tuple           # (dx, dy, dz) in m
    mu: float
    nu: float
    t: np.ndarray          # (F, 3): the family set of the context
    b: np.ndarray          # (F, 3)
    rho: object            # (n, nz, ny, nx) float32: torch tensor (pinned host or device) or numpy
    fam: tuple = None      # indices into (t, b) of rho's n families; None: all F, in order
    submitted: float = field(default=0.0)

    def key(self):
        """Identity of the geometry and family set (one cached context per key)."""
        k = self.__dict__.get("_key")
        if k is None:
            k = (tuple(int(v) for v in self.grid), tuple(float(v) for v in self.cells), float(self.mu),
                 float(self.nu), np.asarray(self.t, np.float64).tobytes(), np.asarray(self.b, np.float64).tobytes())
            self.__dict__["_key"] = k
        return k

    def batch_key(self):
        """Requests evaluated in one call: same context and same family subset."""
        return (self.key(), None if self.fam is None else tuple(int(f) for f in self.fam))

    def n_rho(self) -> int:
        return len(self.t) if self.fam is None else len(self.fam)


class _Entry:
    def __init__(self, ctx, nbytes: int):
        self.ctx = ctx
        self.nbytes = nbytes
        self.busy = False


def io_buffer_bytes(grid, n_rho: int, nb: int = 1) -> int:
    """Device bytes of one launch's density and stress buffers for nb requests."""
    nx, ny, nz = grid
    return 4 * nx * ny * nz * (n_rho + 6) * nb


class CudaBackend:
    """The device side of the server: contexts, streams, launches and their results.

    The scheduler (StressServer) only calls these methods, so its admission, batching
    and eviction logic can run against another backend (the CPU tests use a fake)."""

    def __init__(self, device: int, n_streams: int, max_batch: int):
        import torch
        self.torch = torch
        self.device = device
        self.max_batch = max_batch
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_streams)]

    def _context(self, req: StressRequest):
        ctx = StressContext(self.device)
        nx, ny, nz = req.grid
        dx, dy, dz = req.cells
        ctx.set_geometry(nx, ny, nz, dx, dy, dz, req.mu, req.nu).set_families(req.t, req.b)
        return ctx

    def footprint(self, req: StressRequest) -> int:
        """Device bytes the request's context will hold once built (spectra, work buffers
        for a full batch, and the per-stream density and stress buffers that build()
        leaves cached), computed before building."""
        ctx = self._context(req)
        try:
            lib = ctx.footprint(self.max_batch)
        finally:
            ctx.close()
        return lib + len(self.streams) * io_buffer_bytes(req.grid, req.n_rho(), self.max_batch) + (2 << 20)

    def build(self, req: StressRequest):
        """A built context for the request's geometry and families, and its device bytes."""
        torch = self.torch
        ctx = self._context(req)
        ctx.build_kernels(self.streams[0])
        nx, ny, nz = req.grid
        n = req.n_rho()
        if self.max_batch > 1:
            # size the work buffers for a full batch now (growing them later synchronises the device)
            with torch.cuda.stream(self.streams[0]):
                z = torch.zeros((self.max_batch, 1, nz, ny, nx), device=f"cuda:{self.device}")
                ctx.stress_subset([0], z, stream=self.streams[0])
            self.streams[0].synchronize()
            del z
        # buffers for as many batches as there are streams -- pinned host results, and on
        # each stream the device densities and stresses -- allocated and released here so
        # that the allocators keep them cached, instead of allocating on the scheduler
        # thread while requests wait
        dev = f"cuda:{self.device}"
        keep = [torch.empty((self.max_batch, 6, nz, ny, nx), dtype=torch.float32, pin_memory=True)
                for _ in range(len(self.streams))]
        for st in self.streams:
            with torch.cuda.stream(st):
                keep.append(torch.empty((self.max_batch, n, nz, ny, nx), dtype=torch.float32, device=dev))
                keep.append(torch.empty((self.max_batch, 6, nz, ny, nx), dtype=torch.float32, device=dev))
        del keep
        return ctx, self.footprint(req)

    def launch(self, ctx, reqs, stream):
        """Enqueue one batch on `stream`: densities in, evaluation, results to pinned host
        memory, with CUDA events between the steps.  Returns a job handle for ready() /
        results() / timings()."""
        torch = self.torch
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            rho = torch.empty((len(reqs),) + tuple(reqs[0].rho.shape), dtype=torch.float32,
                              device=f"cuda:{self.device}")
            for i, r in enumerate(reqs):
                rho[i].copy_(r.rho, non_blocking=True)
            ev[1].record(stream)
            if reqs[0].fam is None:
                sigma = ctx.stress_multi(rho, stream=stream)
            else:
                sigma = ctx.stress_subset(reqs[0].fam, rho, stream=stream)
            ev[2].record(stream)
            out = torch.empty(sigma.shape, dtype=sigma.dtype, pin_memory=True)
            out.copy_(sigma, non_blocking=True)
            ev[3].record(stream)
        return {"events": ev, "keep": (rho, sigma), "out": out}

    @staticmethod
    def ready(job) -> bool:
        return job["events"][3].query()

    @staticmethod
    def results(job):
        """Per request of the batch, sigma (6, nz, ny, nx) as a view of the pinned buffer."""
        out = job["out"].numpy()
        return [out[i] for i in range(out.shape[0])]

    @staticmethod
    def timings(job):
        """(h2d, device, d2h) milliseconds of a finished job."""
        e = job["events"]
        return e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])

    @staticmethod
    def interval(job, ref):
        """(start, end) of the job's evaluation kernels in ms after event `ref`."""
        e = job["events"]
        return ref.elapsed_time(e[1]), ref.elapsed_time(e[2])

    def pin(self, rho: np.ndarray):
        return self.torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32)).pin_memory()

    @staticmethod
    def close_context(ctx):
        ctx.close()


class StressServer:
    def __init__(self, device: int = 0, hbm_budget: float = 150e9, n_streams: int = 4, max_batch: int = 8,
                 backend=None):
        self.backend = backend if backend is not None else CudaBackend(device, n_streams, max_batch)
        self.device = device
        self.budget = float(hbm_budget)
        self.max_batch = max_batch
        self.streams = list(self.backend.streams)
        self.free_streams = list(self.streams)
        self.cache: "OrderedDict[tuple, _Entry]" = OrderedDict()
        self.resident = 0
        self.pending: list = []            # (request, future)
        self.inflight: list = []           # dicts: job, stream, entry, items, io
        self.inbox: "queue.Queue" = queue.Queue()
        self.latencies: list = []
        self.records: list = []            # per request: latency and its parts, seconds / ms
        self.keep_jobs = False             # keep finished jobs (tests read their event intervals)
        self.finished_jobs: list = []
        self.stop_flag = False
        self.error = None
        self.thread = threading.Thread(target=self._run, name="stress-scheduler", daemon=True)
        self.thread.start()

    # ---------------------------------------------------------------- public --
    def submit(self, req: StressRequest) -> Future:
        """Queue a request; the future yields sigma (6, nz, ny, nx) as a numpy array."""
        fut: Future = Future()
        if isinstance(req.rho, np.ndarray):
            req.rho = self.backend.pin(req.rho)
        req.submitted = time.perf_counter()
        self.inbox.put((req, fut))
        return fut

    def close(self):
        self.stop_flag = True
        self.thread.join()
        for e in self.cache.values():
            self.backend.close_context(e.ctx)
        self.cache.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def warm(self, req: StressRequest):
        """Build (and cache) the context of a request ahead of time (synchronous)."""
        done, err = threading.Event(), []
        self.inbox.put(("warm", req, done, err))
        done.wait()
        if err:
            raise err[0]

    # ------------------------------------------------------------- scheduler --
    def _get_entry(self, req: StressRequest):
        k = req.key()
        e = self.cache.get(k)
        if e is not None:
            self.cache.move_to_end(k)
            return e
        return None

    def _build_entry(self, req: StressRequest):
        ctx, nbytes = self.backend.build(req)
        e = _Entry(ctx, nbytes)
        self.cache[req.key()] = e
        self.resident += e.nbytes
        return e

    def _footprint(self, req: StressRequest) -> int:
        fp = getattr(self.backend, "footprint", None)
        return int(fp(req)) if fp is not None else 0

    def _make_room(self, need: float, keep=None) -> bool:
        """Evict idle contexts other than `keep`, least recently used first, until `need`
        more bytes fit."""
        while self.resident + need > self.budget:
            victim = next((k for k, e in self.cache.items() if not e.busy and k != keep), None)
            if victim is None:
                return False
            e = self.cache.pop(victim)
            self.resident -= e.nbytes
            self.backend.close_context(e.ctx)
        return True

    def _fit(self, group, keep, extra: float = 0.0):
        """The longest prefix of `group` whose buffers (plus `extra` bytes) fit the budget
        once idle contexts other than `keep` are evicted."""
        n = len(group)
        while n > 0 and not self._make_room(extra + self._io_bytes([r for r, _ in group[:n]]), keep):
            n -= 1
        return group[:n]

    def _reject(self, key, ex):
        """Fail every waiting request of `key` and drop its (idle) context."""
        for r, fut in self.pending:
            if r.key() == key and not fut.done():
                fut.set_exception(ex)
        self.pending = [x for x in self.pending if x[0].key() != key]
        e = self.cache.get(key)
        if e is not None and not e.busy:
            del self.cache[key]
            self.resident -= e.nbytes
            self.backend.close_context(e.ctx)

    @staticmethod
    def _io_bytes(reqs):
        return sum(io_buffer_bytes(r.grid, r.n_rho()) for r in reqs)

    def _launch(self, entry: _Entry, items):
        stream = self.free_streams.pop()
        reqs = [r for r, _ in items]
        t_launch = time.perf_counter()
        job = self.backend.launch(entry.ctx, reqs, stream)
        entry.busy = True
        io = self._io_bytes(reqs)
        self.inflight.append({"job": job, "stream": stream, "entry": entry, "items": items, "io": io,
                              "launched": t_launch})
        self.resident += io

    def _complete(self):
        still = []
        for job in self.inflight:
            if self.backend.ready(job["job"]):
                res = self.backend.results(job["job"])
                now = time.perf_counter()
                # release the context, stream and buffers before waking the waiters, so a
                # caller that resubmits at once finds them free
                job["entry"].busy = False
                self.free_streams.append(job["stream"])
                self.resident -= job["io"]
                tm = getattr(self.backend, "timings", None)
                parts = tm(job["job"]) if tm is not None else (0.0, 0.0, 0.0)
                for (r, fut), sig in zip(job["items"], res):
                    self.latencies.append(now - r.submitted)
                    self.records.append({"latency_s": now - r.submitted, "queue_s": job["launched"] - r.submitted,
                                         "h2d_ms": parts[0], "device_ms": parts[1], "d2h_ms": parts[2],
                                         "batch": len(job["items"]), "cells": int(np.prod(r.grid))})
                    fut.set_result(sig)
                if self.keep_jobs:
                    self.finished_jobs.append(job)
            else:
                still.append(job)
        self.inflight = still

    def _schedule(self):
        progressed = True
        while progressed and self.pending and self.free_streams:
            progressed = False
            for req, fut in self.pending:
                entry = self._get_entry(req)
                if entry is not None and entry.busy:
                    continue                       # its context is on the GPU; try others
                k = req.key()
                bk = req.batch_key()
                group = [(r, f) for r, f in self.pending if r.batch_key() == bk][: self.max_batch]
                if entry is None:
                    # room for the new context (its footprint comes from its plan) and the
                    # buffers of at least the first request, then build
                    try:
                        need = self._footprint(req)
                    except Exception as ex:        # a geometry the library refuses fails its requests only
                        self._reject(k, ex)
                        progressed = True
                        break
                    if self._fit(group, None, extra=need):
                        try:
                            entry = self._build_entry(req)
                        except Exception as ex:    # a context that cannot be built fails its requests only
                            self._reject(k, ex)
                            progressed = True
                            break
                if entry is not None:
                    group = self._fit(group, k)
                if entry is None or not group:
                    if not self.inflight:
                        # nothing else holds device memory: this request can never fit
                        self._reject(k, MemoryError(
                            f"stress request needs more than the {self.budget:.3g}-byte HBM budget"))
                        progressed = True
                        break
                    continue                       # wait for work in flight to release memory
                taken = {id(item[1]) for item in group}
                self.pending = [x for x in self.pending if id(x[1]) not in taken]
                self._launch(entry, group)
                progressed = True
                break

    def _run(self):
        try:
            while True:
                while True:
                    try:
                        msg = self.inbox.get_nowait()
                    except queue.Empty:
                        break
                    if msg[0] == "warm":
                        _, req, done, err = msg
                        try:
                            if self._get_entry(req) is None:
                                if not self._make_room(self._footprint(req)):
                                    raise MemoryError(f"context does not fit the {self.budget:.3g}-byte HBM budget")
                                self._build_entry(req)
                        except Exception as ex:
                            err.append(ex)
                        done.set()
                    else:
                        self.pending.append(msg)
                self._complete()
                self._schedule()
                if self.stop_flag and not self.pending and not self.inflight and self.inbox.empty():
                    return
                time.sleep(0.0002 if (self.inflight or self.pending) else 0.001)
        except BaseException as ex:          # surface scheduler failures to every waiter
            self.error = ex
            for _, fut in self.pending:
                if not fut.done():
                    fut.set_exception(ex)
            for job in self.inflight:
                for _, fut in job["items"]:
                    if not fut.done():
                        fut.set_exception(ex)
            raise

    # ------------------------------------------------------------- metrics --
    def latency_ms(self):
        lat = np.array(self.latencies) * 1e3
        if lat.size == 0:
            return {"n": 0}
        return {"n": int(lat.size), "p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                "mean": float(lat.mean()), "max": float(lat.max())}

    def breakdown_ms(self):
        """p50 / p99 of each latency part over the recorded requests (queue: submission to
        launch on the host; h2d, device, d2h: CUDA events on the request's stream; rest:
        latency minus those, i.e. the host noticing completion and returning the result)."""
        if not self.records:
            return {}
        q = np.array([r["queue_s"] for r in self.records]) * 1e3
        h = np.array([r["h2d_ms"] for r in self.records])
        d = np.array([r["device_ms"] for r in self.records])
        o = np.array([r["d2h_ms"] for r in self.records])
        lat = np.array([r["latency_s"] for r in self.records]) * 1e3
        rest = lat - q - h - d - o
        out = {}
        for name, a in (("queue", q), ("h2d", h), ("device", d), ("d2h", o), ("rest", rest)):
            out[name] = {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99))}
        return out
