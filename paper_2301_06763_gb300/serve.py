"""Continuous-batching potential server on one GPU.

Requests (one nested mesh each: levels, N, dx0, host density) arrive over
time.  Every call to ``Server.step()``:

1. retires the batches whose completion event has fired (their plans go back
   to a pool of resident plans keyed by shape, their bytes back to the budget);
2. admits waiting requests, oldest first, while a stream slot is free and the
   request's device footprint fits the HBM budget (``nm_footprint_bytes`` plus
   its density and potential buffers; idle pooled plans are evicted, least
   recently used first, when the budget needs their memory);
3. launches the admitted requests as one ``nm_batch_potential`` call on the
   free stream: upload of the densities, the batched solve and the download of
   the potentials, all ordered on that stream.

Batches on different streams overlap on the device, and requests that arrive
while earlier batches run join the next batch: continuous batching.  Plans and
their Green spectra stay resident between requests of the same shape.  The
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


class Server:
    def __init__(self, hbm_budget_bytes, slots=4, precision="fp32", max_batch=64, device=None, interp="diagonal"):
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
        self.pool = collections.OrderedDict()   # (L, N, dx0, G, method) -> [Plan], LRU order
        self.pool_bytes = 0
        self.queue = collections.deque()
        self.inflight = []
        self.completed = []
        self.failed = []
        self.batches = 0

    # ------------------------------------------------------------------ memory
    def _dtype(self):
        return self.torch.float32 if self.precision == "fp32" else self.torch.float64

    def request_bytes(self, r, with_plan=True):
        cells = r.levels * r.N ** 3
        b = cells * (_ES[self.precision] + 8)
        if with_plan:
            b += nm.footprint_bytes(r.levels, r.N, r.dx0, r.G, self.precision, r.method, self.interp)
        return b

    def _take_plan(self, r):
        key = (r.levels, r.N, r.dx0, r.G, r.method)
        plans = self.pool.get(key)
        if plans:
            p = plans.pop()
            self.pool_bytes -= p.workspace_bytes()
            if not plans:
                del self.pool[key]
            return p, False
        return None, True

    def _evict_until(self, need):
        while self.used + self.pool_bytes + need > self.budget and self.pool:
            key, plans = next(iter(self.pool.items()))
            p = plans.pop()
            self.pool_bytes -= p.workspace_bytes()
            p.close()
            if not plans:
                del self.pool[key]
        return self.used + self.pool_bytes + need <= self.budget

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
                        r.result = r._phi_host.numpy()
                    self.used -= r.bytes
                    key = (r.levels, r.N, r.dx0, r.G, r.method)
                    self.pool.setdefault(key, []).append(r._plan)
                    self.pool.move_to_end(key)
                    self.pool_bytes += r._plan.workspace_bytes()
                    r._plan = r._rho_dev = r._phi_dev = r._rho_pin = r._phi_host = None
                    self.completed.append(r)
                self.free.append(si)
            else:
                keep.append((si, ev, batch))
        self.inflight = keep

    def _admit(self):
        batch = []
        while self.queue and len(batch) < self.max_batch:
            r = self.queue[0]
            plan, need_plan = self._take_plan(r)
            try:
                need = self.request_bytes(r, with_plan=need_plan)
                if plan is not None:        # a pooled plan's workspace moves from the pool to `used`
                    need += plan.workspace_bytes()
            except Exception as e:          # invalid shape: rejected by the library
                self.queue.popleft()
                r.error = str(e)
                self.failed.append(r)
                continue
            if need > self.budget:
                self.queue.popleft()
                r.error = "footprint %d bytes exceeds the HBM budget %d" % (need, self.budget)
                if plan is not None:
                    self.pool.setdefault((r.levels, r.N, r.dx0, r.G, r.method), []).append(plan)
                    self.pool_bytes += plan.workspace_bytes()
                self.failed.append(r)
                continue
            if not self._evict_until(need):
                if plan is not None:
                    self.pool.setdefault((r.levels, r.N, r.dx0, r.G, r.method), []).append(plan)
                    self.pool_bytes += plan.workspace_bytes()
                break
            self.queue.popleft()
            try:
                if plan is None:
                    plan = nm.Plan(r.levels, r.N, r.dx0, r.G, precision=self.precision, method=r.method,
                                   interp=self.interp)
                    need = self.request_bytes(r, with_plan=False) + plan.workspace_bytes()
            except Exception as e:          # invalid shape or allocation failure
                r.error = str(e)
                self.failed.append(r)
                continue
            r._plan = plan
            r.bytes = need
            self.used += need
            self.peak_used = max(self.peak_used, self.used + self.pool_bytes)
            r.admitted = time.perf_counter()
            batch.append(r)
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
                shape = (r.levels, r.N, r.N, r.N)
                if isinstance(r.rho, torch.Tensor) and r.rho.is_pinned() and r.rho.dtype == self._dtype():
                    r._rho_pin = r.rho                  # caller-pinned: no host copy
                else:
                    arr = r.rho.numpy() if isinstance(r.rho, torch.Tensor) else r.rho
                    r._rho_pin = torch.from_numpy(np.ascontiguousarray(
                        arr, dtype=np.float32 if self.precision == "fp32" else np.float64)).pin_memory()
                r._rho_dev = torch.empty(shape, dtype=self._dtype(), device=self.device)
                r._phi_dev = torch.empty(shape, dtype=torch.float64, device=self.device)
                r._rho_dev.copy_(r._rho_pin, non_blocking=True)
            nm.batch_potential([r._plan for r in batch], [r._rho_dev for r in batch],
                               [r._phi_dev for r in batch], stream=s)
            for r in batch:
                r._phi_host = torch.empty(r._phi_dev.shape, dtype=torch.float64, pin_memory=True)
                r._phi_host.copy_(r._phi_dev, non_blocking=True)
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
        for plans in self.pool.values():
            for p in plans:
                p.close()
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
