"""Serving: a continuous-batching request loop over the C ABI.

A request asks for window statistics (sum, mean, std) of one image for a
list of windows.  The server

- admits requests as they arrive, as long as a request slot and the device
  memory budget allow (tables, build scratch, the staged image and the
  outputs are all counted against the budget); a request that fits may go
  ahead of an older one that does not, a bounded number of times;
- keeps built summed-area tables resident, keyed by image id, evicting
  first the tables no in-flight request uses that were asked for least
  often (least recently among equals), so a
  repeated query on the same image skips the upload and the rebuild (a
  request that arrives while its image is still being built waits for that
  build on the device instead of building again);
- runs admitted requests on a small set of CUDA streams, so the builds and
  queries of different requests overlap on the device;
- records, per request, the time from arrival to completion;
- checks every build's device status when its first request completes: a
  build whose bounded look-back wait expired (``SWA_ETIMEOUT``) is dropped
  from the cache, and every request served from it is reported failed
  (``Request.error``) instead of completed;
- rejects, by itself, a request that could never fit the budget.

``plain_path`` runs the same requests the plain way for comparison: one at a
time on one stream, uploading, building, querying and freeing the tables of
every request.

Results stay in device memory (tensors in ``Request.result``); a client copies
them out when it needs them.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

import paper_2410_16291_gb300 as swa


@dataclass
class Request:
    rid: int
    image_id: object
    host_image: object          # pinned host tensor (uint8 or int16 bit patterns)
    windows: list               # [(wh, ww, sy, sx), ...]
    arrival: float = 0.0        # seconds from the start of the run
    result: list = None         # per window: {"sum", "mean", "std"} device tensors
    admitted: float = None
    done: float = None
    hit: bool = False
    bypassed: int = 0            # younger requests admitted while this one waited
    error: str = None            # set when the request failed (results not valid)

    @property
    def failed(self):
        return self.error is not None

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


@dataclass
class _Entry:
    sat: object                  # swa.SAT (anything with .free())
    nbytes: int
    ready: object = None         # torch.cuda.Event recorded after the build
    refs: int = 0
    status: int = None           # the build's status once read (swa.SWA_OK, ...)
    dropped: bool = False        # out of the cache; freed when refs reaches 0


class TableCache:
    """Resident tables keyed by image id under a byte budget.

    ``used`` counts the cached tables plus whatever transient bytes callers
    reserve; ``reserve`` evicts unreferenced tables until the request fits:
    with policy "lfu" (the default) those asked for least often first (the
    counts, kept by ``count``, outlive an eviction), least recently used
    among equals; with "lru" least recently used first.  Under a budget far
    below the tables of a skewed request stream, keeping the often-asked
    tables rebuilds fewer bytes: replaying the served workload's trace
    (46 images, 424 GB of tables) under 100 GB, 81 misses and 796 GB of
    tables rebuilt against 99 misses and 938 GB with LRU.
    """

    def __init__(self, budget_bytes: int, policy: str = "lfu"):
        if policy not in ("lfu", "lru"):
            raise ValueError("policy must be 'lfu' or 'lru'")
        self.budget = int(budget_bytes)
        self.policy = policy
        self.entries: "collections.OrderedDict[object, _Entry]" = collections.OrderedDict()
        self.freq = collections.Counter()
        self.used = 0
        self.evictions = 0

    def count(self, key):
        """One more request for ``key`` (once per admitted request)."""
        self.freq[key] += 1

    def get(self, key):
        e = self.entries.get(key)
        if e is not None:
            self.entries.move_to_end(key)
        return e

    def reserve(self, need: int) -> bool:
        """Reserve ``need`` bytes, evicting only if that makes them fit: a
        reservation that fails evicts nothing."""
        if self.used + need <= self.budget:
            self.used += need
            return True
        freeable = sum(e.nbytes for e in self.entries.values() if not e.refs)
        if self.used - freeable + need > self.budget:
            return False
        order = list(self.entries.keys())             # least recently used first
        if self.policy == "lfu":
            rank = {k: i for i, k in enumerate(order)}
            order.sort(key=lambda k: (self.freq[k], rank[k]))
        for key in order:
            e = self.entries[key]
            if e.refs:
                continue
            del self.entries[key]
            e.sat.free()
            self.used -= e.nbytes
            self.evictions += 1
            if self.used + need <= self.budget:
                self.used += need
                return True
        return False

    def insert(self, key, entry: _Entry):
        """Cache a built table whose bytes were already reserved."""
        self.entries[key] = entry

    def drop(self, key, entry: _Entry):
        """Take a table out of the cache (a failed build): no later request
        finds it; its memory goes back once no in-flight request uses it."""
        if self.entries.get(key) is entry:
            del self.entries[key]
        entry.dropped = True
        self.release_dropped(entry)

    def release_dropped(self, entry: _Entry):
        if entry.dropped and not entry.refs and entry.sat is not None:
            entry.sat.free()
            entry.sat = None
            self.used -= entry.nbytes

    def release(self, nbytes: int):
        self.used -= nbytes

    def clear(self):
        for e in self.entries.values():
            e.sat.free()
        self.entries.clear()
        self.used = 0


def table_bytes(rows, cols, dtype_code):
    """(resident table bytes, transient build scratch bytes) of one image."""
    import ctypes
    t, s = ctypes.c_int64(), ctypes.c_int64()
    swa.check(swa.lib().swa_sat_bytes(rows, cols, dtype_code, swa.SWA_WITH_SQ, ctypes.byref(t),
                                      ctypes.byref(s)), "swa_sat_bytes")
    return t.value, s.value


def output_bytes(rows, cols, windows):
    n = 0
    for wh, ww, sy, sx in windows:
        R, C = swa.window_shape(rows, cols, wh, ww, sy, sx)
        n += R * C
    return 24 * n


class Server:
    """Continuous-batching server with a resident-table cache (least often
    requested tables evicted first).

    budget_bytes: device memory the server may hold at once.
    streams: number of CUDA streams requests are spread over, or a list of
    existing torch.cuda.Stream objects to use (a long-lived server reuses
    its streams, and with them the device blocks PyTorch's caching allocator
    keeps per stream).
    slots: maximum number of requests on the device at once.
    lookahead, max_bypass: admission may skip over a request that does not
    fit yet (see ``_admit``).
    keep_results: keep each request's output tensors in ``Request.result``
    after it completes (they are outside the budget from then on).
    on_complete: optional ``f(request)`` called on the host as each request
    finishes (failed ones included), before its results are dropped: the
    place for a client to copy or reduce them.  Work it enqueues on the
    device must run on the current stream; the output tensors are released
    to PyTorch's allocator right after the call, so the callback marks them
    (``Tensor.record_stream``) if it uses them on another stream.
    """

    def __init__(self, budget_bytes: int, streams: int = 4, slots: int = 8,
                 keep_results: bool = True, lookahead: int = 8, max_bypass: int = 16,
                 on_complete=None):
        import torch
        self.keep_results = keep_results
        self.on_complete = on_complete
        self.torch = torch
        self.budget = int(budget_bytes)
        if isinstance(streams, int):
            self.streams = [torch.cuda.Stream() for _ in range(streams)]
        else:
            self.streams = list(streams)
        self.slots = slots
        self.lookahead = lookahead
        self.max_bypass = max_bypass
        self.cache = TableCache(budget_bytes)
        self.inflight = []           # (request, event, transient_bytes, entry, image_tensor)
        self.waiting = collections.deque()
        self.completed = []          # every finished request, failed ones included
        self.failed = []             # the failed ones (Request.error says why)
        self.hits = 0
        self.misses = 0
        self._rr = 0

    @property
    def evictions(self):
        return self.cache.evictions

    # ----------------------------------------------------------- dispatch --
    def _try_admit(self, req: Request, now: float):
        """True if admitted, False if it does not fit yet, None if it can
        never fit the budget."""
        torch = self.torch
        rows, cols = req.host_image.shape
        code = swa._dtype_code(req.host_image)
        out_b = output_bytes(rows, cols, req.windows)
        entry = self.cache.get(req.image_id)
        if entry is not None:
            transient = out_b
            if not self.cache.reserve(transient):
                return False
        else:
            tab_b, scr_b = table_bytes(rows, cols, code)
            img_b = rows * cols * req.host_image.element_size()
            transient = out_b + scr_b + img_b
            if tab_b + transient > self.budget:
                req.error = "needs %d bytes, budget %d" % (tab_b + transient, self.budget)
                return None
            if not self.cache.reserve(tab_b + transient):
                return False
        s = self.streams[self._rr % len(self.streams)]
        self._rr += 1
        img_dev = None
        with torch.cuda.stream(s):
            if entry is None:
                img_dev = req.host_image.to("cuda", non_blocking=True)
                sat = swa.build_sat(img_dev, with_sq=True, stream=s)
                ready = torch.cuda.Event()
                ready.record(s)
                entry = _Entry(sat, tab_b, ready)
                self.cache.insert(req.image_id, entry)
                self.misses += 1
            else:
                s.wait_event(entry.ready)       # a build still in flight, or done
                req.hit = True
                self.hits += 1
            entry.refs += 1
            req.result = entry.sat.window_stats(req.windows, stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
        req.admitted = now
        self.cache.count(req.image_id)
        self.inflight.append((req, ev, transient, entry, img_dev))
        return True

    def _finish(self, req: Request, now: float):
        req.done = now
        if self.on_complete is not None:
            self.on_complete(req)
        if req.failed:
            req.result = None
            self.failed.append(req)
        elif not self.keep_results:
            req.result = None
        self.completed.append(req)

    def _poll(self, now: float):
        still = []
        for req, ev, transient, entry, img_dev in self.inflight:
            if ev.query():
                # The build finished before this request's queries did: read
                # its device status once (no stream is drained).
                if entry.status is None:
                    entry.status = entry.sat.status()
                    if entry.status != swa.SWA_OK:
                        self.cache.drop(req.image_id, entry)
                if entry.status != swa.SWA_OK:
                    req.error = "table build failed: %s" % (
                        swa.lib().swa_status_str(entry.status).decode())
                entry.refs -= 1
                self.cache.release(transient)
                self.cache.release_dropped(entry)
                self._finish(req, now)
            else:
                still.append((req, ev, transient, entry, img_dev))
        self.inflight = still

    def _admit(self, now: float) -> bool:
        """Admit waiting requests in arrival order while slots and memory
        allow.  When the oldest request does not fit, up to ``lookahead``
        younger ones that do fit (typically cache hits, which need only
        output memory) go ahead of it; each bypass is counted on the oldest
        request, and after ``max_bypass`` of them nothing may overtake it,
        so a large miss is delayed but never starved."""
        progressed = False
        while self.waiting and len(self.inflight) < self.slots:
            head = self.waiting[0]
            ok = self._try_admit(head, now)
            if ok is None:                      # can never fit: fail it alone
                self.waiting.popleft()
                self._finish(head, now)
                progressed = True
                continue
            if ok:
                self.waiting.popleft()
                progressed = True
                continue
            if head.bypassed >= self.max_bypass:
                break
            admitted = None
            for i in range(1, min(len(self.waiting), 1 + self.lookahead)):
                ok = self._try_admit(self.waiting[i], now)
                if ok is None:
                    self._finish(self.waiting[i], now)
                    admitted = i
                    break
                if ok:
                    admitted = i
                    head.bypassed += 1
                    break
            if admitted is None:
                break
            del self.waiting[admitted]
            progressed = True
        return progressed

    # -------------------------------------------------------------- run ---
    def run(self, requests, realtime: bool = True, poll_s: float = 50e-6):
        """Serve `requests` (sorted by arrival).  With realtime, a request
        becomes visible at its arrival time; otherwise all arrive at once."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        t0 = time.perf_counter()
        while pending or self.waiting or self.inflight:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                if not realtime:
                    r.arrival = now
                self.waiting.append(r)
            self._poll(now)
            progressed = self._admit(now)
            if not progressed:
                nxt = pending[0].arrival - now if pending else poll_s
                time.sleep(max(0.0, min(poll_s, nxt)))
        self.torch.cuda.synchronize()
        return time.perf_counter() - t0

    def close(self):
        self.cache.clear()


def plain_path(requests, realtime: bool = True, stream=None, keep_results: bool = True):
    """The plain per-request path: in arrival order, one request at a time on
    one stream, upload + build + query + free, waiting for each to finish."""
    import torch
    s = stream or torch.cuda.Stream()
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    for r in reqs:
        if realtime:
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        else:
            r.arrival = time.perf_counter() - t0
        with torch.cuda.stream(s):
            img = r.host_image.to("cuda", non_blocking=True)
            sat = swa.build_sat(img, with_sq=True, stream=s)
            r.result = sat.window_stats(r.windows, stream=s)
        s.synchronize()
        st = sat.status()
        sat.free()
        r.done = time.perf_counter() - t0
        if st != swa.SWA_OK:
            r.error = "table build failed: %s" % swa.lib().swa_status_str(st).decode()
        if not keep_results or r.failed:
            r.result = None
    return time.perf_counter() - t0


def latency_summary(requests):
    """Latency percentiles over the requests that completed without error;
    failed requests are counted separately."""
    failed = sum(1 for r in requests if r.failed)
    lat = np.array([r.latency for r in requests if r.latency is not None and not r.failed])
    if not len(lat):
        return {"failed": failed} if failed else {}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3),
            "requests": int(len(lat)), "failed": failed}
