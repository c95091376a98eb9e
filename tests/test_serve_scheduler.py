"""Host logic of the stress server, on the CPU: the scheduler runs against a fake
device backend whose launches finish when the test says so.  Checked: batching of
same-geometry requests up to max_batch, results routed to the right futures in
order, busy contexts skipped while other contexts run, least-recently-used eviction
under the HBM budget (never of the context about to run), requests that can never
fit failed with MemoryError (a context's footprint counted before it is built), build
failures failing only their own requests, family subsets batched only with the same
subset, and the latency breakdown."""
import threading
import time

import numpy as np
import pytest

from paper_1804_01830_gb300.serve import StressRequest, StressServer

CTX_BYTES = 1000


class FakeCtx:
    def __init__(self, key):
        self.key = key
        self.closed = False


class FakeBackend:
    """Streams are names; a context costs CTX_BYTES; a launch's result for request i is
    rho_i summed, times (1..6); jobs finish when `release()` is called (or at once when
    auto is set)."""

    def __init__(self, n_streams=2, auto=True, fail_grid=None):
        self.streams = [f"s{i}" for i in range(n_streams)]
        self.auto = auto
        self.fail_grid = fail_grid
        self.lock = threading.Lock()
        self.builds, self.closes, self.launches = [], [], []
        self.jobs = []

    def footprint(self, req):
        return CTX_BYTES

    def build(self, req):
        if self.fail_grid is not None and tuple(req.grid) == self.fail_grid:
            raise RuntimeError("build failed")
        with self.lock:
            self.builds.append(req.grid)
        return FakeCtx(req.grid), CTX_BYTES

    def launch(self, ctx, reqs, stream):
        assert not ctx.closed, "launch on a closed context"
        job = {"ctx": ctx, "stream": stream, "out": [float(np.sum(r.rho)) * np.arange(1, 7) for r in reqs],
               "done": threading.Event()}
        if self.auto:
            job["done"].set()
        with self.lock:
            self.launches.append((ctx.key, len(reqs), stream))
            self.jobs.append(job)
        return job

    def release(self):
        with self.lock:
            for j in self.jobs:
                j["done"].set()

    @staticmethod
    def ready(job):
        return job["done"].is_set()

    @staticmethod
    def results(job):
        return job["out"]

    @staticmethod
    def timings(job):
        return 0.5, 2.0, 1.0

    @staticmethod
    def pin(rho):
        return rho

    def close_context(self, ctx):
        ctx.closed = True
        with self.lock:
            self.closes.append(ctx.key)


def request(grid, value, n_fam=1):
    nx, ny, nz = grid
    t = np.tile([[1.0, 0.0, 0.0]], (n_fam, 1))
    return StressRequest(grid, (1e-6, 1e-6, 1e-6), 1e10, 0.3, t, t.copy(),
                         np.full((n_fam, nz, ny, nx), value, np.float32))


def io(grid, n_fam=1):
    return StressServer._io_bytes([request(grid, 0.0, n_fam)])


def wait_until(cond, timeout=5.0):
    t0 = time.time()
    while not cond():
        assert time.time() - t0 < timeout, "condition not reached"
        time.sleep(0.001)


def expect(fut, rho_sum):
    np.testing.assert_allclose(fut.result(timeout=5), rho_sum * np.arange(1, 7))


def test_same_geometry_requests_batch_up_to_max_batch():
    be = FakeBackend(n_streams=2, auto=False)
    g = (4, 2, 1)
    with StressServer(hbm_budget=1e9, max_batch=4, backend=be) as srv:
        first = srv.submit(request(g, 1.0))
        wait_until(lambda: len(be.launches) == 1)
        # the context is busy: these wait, then go out as one batch of 4 and one of 2
        rest = [srv.submit(request(g, float(i + 2))) for i in range(6)]
        time.sleep(0.02)
        assert len(be.launches) == 1
        be.auto = True
        be.release()
        for i, f in enumerate(rest):
            expect(f, 8.0 * (i + 2))
        expect(first, 8.0)
    assert [n for _, n, _ in be.launches] == [1, 4, 2]
    assert be.builds == [g]                       # built once, cached
    assert srv.latency_ms()["n"] == 7


def test_busy_context_does_not_block_other_geometries():
    be = FakeBackend(n_streams=3, auto=False)
    a, b = (4, 2, 1), (8, 2, 1)
    with StressServer(hbm_budget=1e9, max_batch=2, backend=be) as srv:
        fa = srv.submit(request(a, 1.0))
        wait_until(lambda: len(be.launches) == 1)
        fa2 = srv.submit(request(a, 2.0))           # waits for a's context
        fb = srv.submit(request(b, 3.0))            # runs meanwhile, on another stream
        wait_until(lambda: len(be.launches) == 2)
        assert be.launches[1][0] == b and be.launches[1][2] != be.launches[0][2]
        be.auto = True
        be.release()
        expect(fa, 8.0)
        expect(fa2, 16.0)
        expect(fb, 48.0)


def test_streams_bound_the_work_in_flight():
    be = FakeBackend(n_streams=2, auto=False)
    grids = [(4, 2, 1), (8, 2, 1), (4, 4, 1)]
    with StressServer(hbm_budget=1e9, max_batch=2, backend=be) as srv:
        futs = [srv.submit(request(g, 1.0)) for g in grids]
        wait_until(lambda: len(be.launches) == 2)
        time.sleep(0.02)
        assert len(be.launches) == 2                # both streams taken
        be.auto = True
        be.release()
        for f, g in zip(futs, grids):
            expect(f, float(np.prod(g)))


def test_least_recently_used_context_is_evicted():
    be = FakeBackend()
    A, B, C, D = (4, 2, 1), (8, 2, 1), (4, 4, 1), (8, 4, 1)
    budget = 2 * CTX_BYTES + io(D) + 1            # two contexts and one request's buffers
    with StressServer(hbm_budget=budget, max_batch=2, backend=be) as srv:
        for g in (A, B, C):
            expect(srv.submit(request(g, 1.0)), float(np.prod(g)))
        assert be.closes == [A]                   # C evicted the oldest
        expect(srv.submit(request(B, 1.0)), 16.0)  # B is now the most recent
        expect(srv.submit(request(D, 1.0)), 32.0)
        assert be.closes == [A, C]
        assert srv.resident == 2 * CTX_BYTES
    assert sorted(be.closes) == sorted([A, C, B, D])   # close() releases the rest


def test_context_footprint_is_counted_before_building():
    # room for the buffers but not for the context too: nothing is built, the request fails
    be = FakeBackend()
    g = (4, 2, 1)
    budget = CTX_BYTES + io(g) - 1
    with StressServer(hbm_budget=budget, backend=be) as srv:
        with pytest.raises(MemoryError):
            srv.submit(request(g, 1.0)).result(timeout=5)
        assert be.launches == [] and be.builds == []
        assert srv.resident == 0 and not srv.cache
    assert be.closes == []
    with StressServer(hbm_budget=CTX_BYTES - 1, backend=be) as srv:   # warm: the context alone
        with pytest.raises(MemoryError):
            srv.warm(request(g, 0.0))
    assert be.builds == []


def test_context_about_to_run_is_never_evicted():
    # a backend that learns a context's size only by building it: room for the buffers
    # but not for the context too; the only idle context is the one just built, and it
    # must not be closed under the launch (the fake asserts that)
    class LateSize(FakeBackend):
        footprint = None
    be = LateSize()
    g = (4, 2, 1)
    budget = CTX_BYTES + io(g) - 1
    with StressServer(hbm_budget=budget, backend=be) as srv:
        with pytest.raises(MemoryError):
            srv.submit(request(g, 1.0)).result(timeout=5)
        assert be.launches == []
        assert srv.resident == 0 and not srv.cache
    assert be.closes == [g]


def test_family_subsets_batch_only_with_the_same_subset():
    be = FakeBackend(n_streams=1, auto=False)
    g = (4, 2, 1)
    t = np.tile([[1.0, 0.0, 0.0]], (4, 1))

    def sub(fam, value):
        nx, ny, nz = g
        return StressRequest(g, (1e-6, 1e-6, 1e-6), 1e10, 0.3, t, t.copy(),
                             np.full((len(fam), nz, ny, nx), value, np.float32), fam=tuple(fam))
    with StressServer(hbm_budget=1e9, max_batch=4, backend=be) as srv:
        first = srv.submit(sub([0], 1.0))
        wait_until(lambda: len(be.launches) == 1)
        futs = [srv.submit(sub(f, 1.0)) for f in ([1, 2], [0], [1, 2], [3], [0])]
        time.sleep(0.02)
        be.auto = True
        be.release()
        for f, fam in zip(futs, ([1, 2], [0], [1, 2], [3], [0])):
            expect(f, 8.0 * len(fam))
        expect(first, 8.0)
        br = srv.breakdown_ms()
    assert be.builds == [g]                        # one context serves every subset
    assert sorted(n for _, n, _ in be.launches[1:]) == [1, 2, 2]
    assert br["device"]["p50"] == 2.0 and br["h2d"]["p99"] == 0.5 and br["queue"]["p50"] >= 0.0


def test_requests_that_fit_only_alone_are_split():
    be = FakeBackend()
    g = (4, 2, 1)
    budget = CTX_BYTES + io(g) + 1                # one request's buffers at a time
    with StressServer(hbm_budget=budget, max_batch=4, backend=be) as srv:
        srv.warm(request(g, 0.0))
        futs = [srv.submit(request(g, float(i))) for i in range(3)]
        for i, f in enumerate(futs):
            expect(f, 8.0 * i)
    assert all(n == 1 for _, n, _ in be.launches)


def test_waits_for_memory_held_by_work_in_flight():
    be = FakeBackend(n_streams=2, auto=False)
    A, B = (4, 2, 1), (8, 2, 1)
    budget = CTX_BYTES + io(B) + io(A) + 1        # a second context fits only after A is idle
    with StressServer(hbm_budget=budget, backend=be) as srv:
        fa = srv.submit(request(A, 1.0))
        wait_until(lambda: len(be.launches) == 1)
        fb = srv.submit(request(B, 1.0))
        time.sleep(0.02)
        assert len(be.launches) == 1 and not fb.done()   # not rejected: A will release memory
        be.auto = True
        be.release()
        expect(fa, 8.0)
        expect(fb, 16.0)
    assert be.closes[0] == A


def test_build_failure_fails_only_its_requests():
    bad, good = (4, 2, 1), (8, 2, 1)
    be = FakeBackend(fail_grid=bad)
    with StressServer(hbm_budget=1e9, backend=be) as srv:
        fb = srv.submit(request(bad, 1.0))
        fg = srv.submit(request(good, 1.0))
        with pytest.raises(RuntimeError, match="build failed"):
            fb.result(timeout=5)
        expect(fg, 16.0)
        with pytest.raises(RuntimeError, match="build failed"):
            srv.warm(request(bad, 0.0))
        assert srv.error is None


def test_keys_separate_geometry_and_families():
    g = (4, 2, 1)
    r1, r2, r3 = request(g, 0.0), request(g, 1.0), request(g, 0.0, n_fam=2)
    r4 = request(g, 0.0)
    r4.cells = (1e-6, 1e-6, 2e-6)
    assert r1.key() == r2.key()
    assert len({r1.key(), r3.key(), r4.key()}) == 3
