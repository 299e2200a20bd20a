"""Continuous-batching potential server on one GPU.

Requests (one nested mesh each: levels, N, dx0, host density) arrive over
time.  Every call to ``Server.step()``:

1. retires the batches whose completion event has fired (each request's
   resident set -- plan, device buffers and page-locked staging -- goes back
   to a pool keyed by shape, its bytes back to the budget);
2. admits waiting requests, oldest first, while a stream slot is free and the
   request's device footprint fits the HBM budget (``nm_footprint_bytes`` plus
   its density and potential buffers; idle resident sets are evicted, least
   recently used first, when the budget needs their memory);
3. launches the admitted requests as one ``nm_batch_potential`` call on the
   free stream: upload of the densities, the batched solve and the download of
   the potentials, all ordered on that stream.

Batches on different streams overlap on the device, and requests that arrive
while earlier batches run join the next batch: continuous batching.  Plans,
their Green spectra and the request buffers stay resident between requests of
the same shape (``Server.prewarm`` makes them ahead of the stream), so a
request of a seen shape allocates neither device nor page-locked memory.  The
arithmetic all runs in the CUDA library; this module only schedules.
"""
import collections
import time

import numpy as np

from . import nm

_ES = {"fp32": 4, "fp64": 8, "fp64x": 8}


class Request:
    def __init__(self, rid, levels, N, dx0, rho, arrival=0.0, G=1.0, keep_result=True, method="original"):
        self.rid = rid
        self.levels, self.N, self.dx0, self.G = int(levels), int(N), float(dx0), float(G)
        self.method = method            # "original", "dipole", "dipole3" or "dipole3_ds"
        self.rho = rho                  # host (levels, N, N, N): numpy array or (pinned) CPU tensor
        self.arrival = float(arrival)   # wall-clock seconds (perf_counter) of arrival
        self.keep_result = keep_result
        self.admitted = None
        self.done = None
        self.result = None              # host float64 potentials when keep_result
        self.error = None
        self.bytes = 0

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


class _Resident:
    """What one request shape keeps on the device between requests: a plan
    (its workspace and Green spectrum) and the density and potential buffers,
    with page-locked host staging for both, so that serving a request of a
    seen shape allocates nothing."""

    def __init__(self, torch, key, precision, interp, device):
        L, N, dx0, G, method = key
        self.key = key
        self.plan = nm.Plan(L, N, dx0, G, precision=precision, method=method, interp=interp)
        shape = (L, N, N, N)
        dt = torch.float32 if precision == "fp32" else torch.float64
        try:
            self.rho_dev = torch.empty(shape, dtype=dt, device=device)
            self.phi_dev = torch.empty(shape, dtype=torch.float64, device=device)
            self.rho_pin = torch.empty(shape, dtype=dt, pin_memory=True)
            self.phi_pin = torch.empty(shape, dtype=torch.float64, pin_memory=True)
        except Exception:
            self.plan.close()
            raise
        self.bytes = self.plan.workspace_bytes() + self.rho_dev.nbytes + self.phi_dev.nbytes

    def close(self):
        if self.plan is not None:
            self.plan.close()
        self.plan = self.rho_dev = self.phi_dev = self.rho_pin = self.phi_pin = None


class Server:
    def __init__(self, hbm_budget_bytes, slots=4, precision="fp32", max_batch=64, device=None, interp="diagonal",
                 per_shape_cap=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.peak_used = 0
        self.precision = precision
        self.interp = interp
        self.max_batch = int(max_batch)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.free = list(range(slots))
        self.pool = collections.OrderedDict()   # key -> [_Resident], least recently used first
        self.pool_bytes = 0
        self.queue = collections.deque()
        self.inflight = []
        self.completed = []
        self.failed = []
        self.batches = 0
        self.residents_made = 0
        self.res_count = {}                     # key -> resident sets in existence
        self.per_shape_cap = int(per_shape_cap if per_shape_cap is not None else slots)
        self.scan_limit = 4 * self.max_batch

    # ------------------------------------------------------------------ memory
    def _dtype(self):
        return self.torch.float32 if self.precision == "fp32" else self.torch.float64

    @staticmethod
    def _key(r):
        return (r.levels, r.N, r.dx0, r.G, r.method)

    def request_bytes(self, r, with_plan=True):
        """Device bytes a request of this shape occupies: its density and
        potential buffers, and (with_plan) the plan's workspace."""
        cells = r.levels * r.N ** 3
        b = cells * (_ES[self.precision] + 8)
        if with_plan:
            b += nm.footprint_bytes(r.levels, r.N, r.dx0, r.G, self.precision, r.method, self.interp)
        return b

    def _pool_put(self, res):
        self.pool.setdefault(res.key, []).append(res)
        self.pool.move_to_end(res.key)
        self.pool_bytes += res.bytes

    def _pool_take(self, key):
        lst = self.pool.get(key)
        if not lst:
            return None
        res = lst.pop()
        self.pool_bytes -= res.bytes
        if not lst:
            del self.pool[key]
        return res

    def _evict_until(self, need):
        while self.used + self.pool_bytes + need > self.budget and self.pool:
            key, lst = next(iter(self.pool.items()))
            res = lst.pop()
            self.pool_bytes -= res.bytes
            self._close(res)
            if not lst:
                del self.pool[key]
        return self.used + self.pool_bytes + need <= self.budget

    def _make(self, key):
        res = _Resident(self.torch, key, self.precision, self.interp, self.device)
        self.residents_made += 1
        self.res_count[key] = self.res_count.get(key, 0) + 1
        return res

    def _close(self, res):
        self.res_count[res.key] = self.res_count.get(res.key, 1) - 1
        res.close()

    def prewarm(self, shapes, per_shape=1, method="original", G=1.0):
        """Make plans, Green spectra and buffers for request shapes ahead of
        time: ``shapes`` = iterable of (levels, N) (dx0 = 1/N) or (levels, N,
        dx0); ``per_shape`` residents each, while the HBM budget allows (the
        smallest shapes first).  Returns the number made."""
        made = 0
        keys = []
        for sh in shapes:
            L, N = int(sh[0]), int(sh[1])
            dx0 = float(sh[2]) if len(sh) > 2 else 1.0 / N
            keys.append((L, N, dx0, float(G), method))
        keys.sort(key=lambda k: k[0] * k[1] ** 3)
        for key in keys:
            for _ in range(per_shape - len(self.pool.get(key, []))):
                need = nm.footprint_bytes(key[0], key[1], key[2], key[3], self.precision, key[4], self.interp) \
                    + key[0] * key[1] ** 3 * (_ES[self.precision] + 8)
                if self.used + self.pool_bytes + need > self.budget:
                    return made
                res = self._make(key)
                res.plan.green()
                self._pool_put(res)
                made += 1
        self.torch.cuda.synchronize(self.device)
        return made

    # ------------------------------------------------------------------ loop
    def submit(self, r):
        self.queue.append(r)

    def _retire(self):
        keep = []
        for (si, ev, batch) in self.inflight:
            if ev.query():
                now = time.perf_counter()
                for r in batch:
                    r.done = now
                    if r.keep_result:
                        r.result = r._res.phi_pin.numpy().copy()
                    self.used -= r.bytes
                    self._pool_put(r._res)
                    r._res = None
                    self.completed.append(r)
                self.free.append(si)
            else:
                keep.append((si, ev, batch))
        self.inflight = keep

    def _admit(self):
        """Requests for the next batch, oldest first.  A request whose shape
        has no idle resident set is admitted with a new one only while that
        shape has fewer than `per_shape_cap` sets; otherwise it waits in the
        queue (later requests of other shapes may pass it), so a warm server
        allocates nothing however many requests of one shape are queued."""
        batch = []
        keep = collections.deque()
        scanned = 0
        while self.queue and len(batch) < self.max_batch and scanned < self.scan_limit:
            r = self.queue.popleft()
            scanned += 1
            key = self._key(r)
            res = self._pool_take(key)
            if res is None and self.res_count.get(key, 0) >= self.per_shape_cap:
                keep.append(r)                  # all of this shape's sets are in flight
                continue
            try:
                need = res.bytes if res is not None else self.request_bytes(r)
            except Exception as e:              # invalid shape: rejected by the library
                r.error = str(e)
                self.failed.append(r)
                continue
            if need > self.budget:
                r.error = "footprint %d bytes exceeds the HBM budget %d" % (need, self.budget)
                if res is not None:
                    self._pool_put(res)
                self.failed.append(r)
                continue
            if not self._evict_until(need):
                if res is not None:
                    self._pool_put(res)
                keep.append(r)
                break
            if res is None:
                try:
                    res = self._make(key)
                except Exception as e:          # invalid shape or allocation failure
                    r.error = str(e)
                    self.failed.append(r)
                    continue
                need = res.bytes
            r._res = res
            r.bytes = need
            self.used += need
            self.peak_used = max(self.peak_used, self.used + self.pool_bytes)
            r.admitted = time.perf_counter()
            batch.append(r)
        # the passed-over requests keep their places at the head of the queue
        keep.extend(self.queue)
        self.queue = keep
        return batch

    def step(self):
        """Retire finished batches, then admit and launch one new batch."""
        torch = self.torch
        self._retire()
        if not self.free or not self.queue:
            return 0
        batch = self._admit()
        if not batch:
            return 0
        si = self.free.pop()
        s = self.streams[si]
        with torch.cuda.stream(s):
            for r in batch:
                res = r._res
                rho = r.rho
                if isinstance(rho, torch.Tensor) and rho.is_pinned() and rho.dtype == self._dtype() \
                        and rho.is_contiguous():
                    src = rho                       # caller-pinned: straight from there
                else:
                    arr = rho.numpy() if isinstance(rho, torch.Tensor) else np.asarray(rho)
                    np.copyto(res.rho_pin.numpy(), arr, casting="same_kind")
                    src = res.rho_pin
                res.rho_dev.copy_(src, non_blocking=True)
            nm.batch_potential([r._res.plan for r in batch], [r._res.rho_dev for r in batch],
                               [r._res.phi_dev for r in batch], stream=s)
            for r in batch:
                r._res.phi_pin.copy_(r._res.phi_dev, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        self.inflight.append((si, ev, batch))
        self.batches += 1
        return len(batch)

    def busy(self):
        return bool(self.queue or self.inflight)

    def drain(self, poll_s=20e-6):
        while self.busy():
            if self.step() == 0:
                time.sleep(poll_s)

    def close(self):
        self.drain()
        for lst in self.pool.values():
            for res in lst:
                self._close(res)
        self.pool.clear()
        self.pool_bytes = 0


def run_stream(server, requests, poll_s=20e-6):
    """Feed ``requests`` (``arrival`` = offset in seconds from now) as they fall
    due and serve them all; returns (elapsed seconds, completed requests)."""
    t0 = time.perf_counter()
    pending = sorted(requests, key=lambda r: r.arrival)
    for r in pending:
        r.arrival += t0
    i = 0
    while i < len(pending) or server.busy():
        now = time.perf_counter()
        while i < len(pending) and pending[i].arrival <= now:
            server.submit(pending[i])
            i += 1
        if server.step() == 0:
            time.sleep(poll_s)
    return time.perf_counter() - t0, server.completed


def latency_stats(requests):
    lat = np.array([r.latency for r in requests if r.latency is not None])
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
