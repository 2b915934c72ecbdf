"""Continuous-batching request loop over the lookup library.

Requests (a batch of query coordinates against one device-resident texture, a
filter, stochastic or deterministic) arrive over time.  The server keeps a fixed
set of slots, each a CUDA stream.  A waiting request is admitted when a slot is
free and its device footprint (coordinates, levels of detail, results) fits in the
memory budget next to the requests already admitted; requests that arrive while
others run are admitted as slots and memory free up, and the work of all admitted
requests overlaps on the GPU.  Each request runs as a sequence of chunks (host to
device copy, one library call, device to host copy) on its slot's stream; chunks
pass query_offset so the random variates stay keyed on the request-local query
index: a request's result is the same whether it runs alone or in any mix.

Memory accounting: the budget covers what is resident on the device for serving,
the textures' bytes (``resident_bytes``) plus every slot's buffers.  A slot keeps
its buffers between requests (so that admitting a request usually allocates
nothing), so the scheduler charges each slot the bytes it holds, idle or not, and a
request is admitted only if the slot's buffers after growing for it, plus every
other slot's holdings and the resident bytes, fit in the budget; idle slots'
buffers are released when that makes room.

The loop itself (admission, budget, chunking, completion) lives in ``Scheduler``,
which talks to the device through a small backend interface so that it can be
tested without a GPU; ``TorchBackend`` is the real one.  A backend provides
``channels(texture)``, ``hold_after(slot, request)`` (bytes the slot holds once it
has begun the request), ``release(slot)`` (free an idle slot's buffers), ``begin``,
``launch_chunk``, ``chunk_done`` and ``finish``.
"""
import collections
import math
import time

import paper_2305_05810_gb300 as stf


class BudgetError(RuntimeError):
    """A request can never fit in the memory budget (STF_ERR_BUDGET)."""
    status = 7


class Request:
    """One lookup request.  ``coords`` is a host tensor (pinned for overlap),
    n x 2 for 2D textures and n x 3 for 3D grids; ``lod`` is optional (2D)."""

    def __init__(self, rid, texture, coords, lod=None, *, filter="bspline3", stochastic=True,
                 seed=0, level_mode=stf.LEVEL_STOCHASTIC, arrival=0.0):
        self.rid = rid
        self.texture = texture
        self.coords = coords
        self.lod = lod
        self.filter = filter
        self.stochastic = stochastic
        self.seed = seed
        self.level_mode = level_mode
        self.arrival = arrival
        self.n = int(coords.shape[0])
        self.result = None
        self.t_admit = None
        self.t_done = None

    def device_bytes(self, channels):
        per = self.coords.shape[1] * 4 + channels * 4 + (4 if self.lod is not None else 0)
        return self.n * per

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.arrival


class Scheduler:
    """Admission, chunking and completion; the device side is the backend."""

    def __init__(self, backend, n_slots=8, budget_bytes=16 << 30, chunk_queries=1 << 20,
                 max_chunks_in_flight=2, clock=time.perf_counter, resident_bytes=0):
        self.backend = backend
        self.n_slots = n_slots
        self.budget = int(budget_bytes)
        self.resident = int(resident_bytes)
        if self.resident > self.budget:
            raise BudgetError("resident textures (%d bytes) exceed the budget (%d)" % (self.resident, self.budget))
        self.chunk = int(chunk_queries)
        self.depth = max_chunks_in_flight
        self.clock = clock
        self.waiting = collections.deque()
        self.free_slots = collections.deque(range(n_slots))
        self.active = {}            # slot -> job
        self.hold = [0] * n_slots   # device bytes each slot holds (idle slots keep buffers)
        self.done = []
        self.rejected = []
        self.peak_in_use = self.resident
        self.peak_active = 0

    @property
    def in_use(self):
        """Device bytes charged against the budget: resident textures plus every
        slot's buffers."""
        return self.resident + sum(self.hold)

    def submit(self, req):
        need = self.backend.hold_after(None, req)
        if self.resident + need > self.budget:
            self.rejected.append(req)
            raise BudgetError("request %r needs %d bytes next to %d resident, budget is %d" %
                              (req.rid, need, self.resident, self.budget))
        self.waiting.append(req)

    def _fit(self, req):
        """A free slot the request fits in, releasing idle slots' buffers if that
        makes room; None if it must wait."""
        best = None
        for slot in self.free_slots:
            after = self.in_use - self.hold[slot] + self.backend.hold_after(slot, req)
            if best is None or after < best[1]:
                best = (slot, after)
        slot, after = best
        if after <= self.budget:
            return slot
        for other in list(self.free_slots):
            if other != slot and self.hold[other] > 0:
                self.backend.release(other)
                after -= self.hold[other]
                self.hold[other] = 0
                if after <= self.budget:
                    return slot
        if after - self.hold[slot] + self.backend.hold_after(None, req) <= self.budget:
            self.backend.release(slot)                  # regrow this slot from nothing
            self.hold[slot] = 0
            return slot
        return None

    def _admit(self):
        while self.waiting and self.free_slots:
            req = self.waiting[0]
            slot = self._fit(req)
            if slot is None:
                return                                  # FIFO: wait for memory
            self.waiting.popleft()
            self.free_slots.remove(slot)
            self.hold[slot] = self.backend.hold_after(slot, req)
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            assert self.in_use <= self.budget
            req.t_admit = self.clock()
            job = {"req": req, "slot": slot, "next": 0, "inflight": collections.deque(),
                   "state": self.backend.begin(req, slot)}
            self.active[slot] = job
            self.peak_active = max(self.peak_active, len(self.active))

    def _issue(self):
        for slot, job in self.active.items():
            req = job["req"]
            while job["next"] < req.n and len(job["inflight"]) < self.depth:
                a = job["next"]
                b = min(req.n, a + self.chunk)
                job["inflight"].append(self.backend.launch_chunk(job["state"], req, slot, a, b))
                job["next"] = b

    def _retire(self):
        finished = []
        for slot, job in self.active.items():
            q = job["inflight"]
            while q and self.backend.chunk_done(q[0]):
                q.popleft()
            if not q and job["next"] >= job["req"].n:
                finished.append(slot)
        for slot in finished:
            job = self.active.pop(slot)
            req = job["req"]
            req.result = self.backend.finish(job["state"], req)
            req.t_done = self.clock()
            self.free_slots.append(slot)
            self.done.append(req)

    def step(self):
        self._retire()
        self._admit()
        self._issue()

    def idle(self):
        return not self.waiting and not self.active

    def run(self, requests, realtime=True):
        """Serve requests (sorted by arrival).  With realtime, arrivals are released
        at their arrival times relative to the start; latencies are measured from
        those times."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        t0 = self.clock()
        for r in pending:
            r.arrival = t0 + r.arrival if realtime else t0
        while pending or not self.idle():
            now = self.clock()
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                try:
                    self.submit(r)
                except BudgetError:
                    pass
            self.step()
            if self.idle() and pending:
                wait = pending[0].arrival - self.clock()
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        return self.done


class TorchBackend:
    """Device side of the scheduler: torch streams, pinned host buffers, the C ABI.

    Each slot owns device buffers (coordinates, levels of detail, results) and a
    pinned host buffer for results; all grow to the largest request the slot has
    served and are then reused, so admitting a request usually allocates nothing
    (device and pinned-host allocations synchronise and would stall the other
    slots).  ``hold_after`` reports the device bytes a slot's buffers take once they
    have grown for a request, which the scheduler charges against its budget;
    ``release`` drops an idle slot's device buffers (their blocks return to torch's
    caching allocator, which reuses them for the next growth).  With
    keep_results the result of each request is copied out of the slot's pinned buffer
    into its own host tensor; otherwise ``on_result(request, view)`` (if given) sees
    the pinned view before the slot is reused."""

    def __init__(self, textures, n_slots=8, device=None, keep_results=True, on_result=None):
        import torch
        self.torch = torch
        self.textures = textures                       # key -> stf.Texture
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_slots)]
        self.slot_bufs = [{} for _ in range(n_slots)]
        self.keep_results = keep_results
        self.on_result = on_result

    def channels(self, key):
        return self.textures[key].channels

    @staticmethod
    def _alloc_numel(numel):
        return max(numel, 1 << 16)

    def _needs(self, req):
        C = self.textures[req.texture].channels
        d = {"coords": req.n * req.coords.shape[1], "out": req.n * C}
        if req.lod is not None:
            d["lod"] = req.n
        return d

    def hold_after(self, slot, req):
        """Device bytes slot holds after begin(req) (slot None: an empty slot)."""
        have = {} if slot is None else {k: b.numel() for k, b in self.slot_bufs[slot].items()
                                        if k != "h_out"}
        for k, numel in self._needs(req).items():
            if have.get(k, 0) < numel:
                have[k] = self._alloc_numel(numel)
        return 4 * sum(have.values())

    def release(self, slot):
        for k in [k for k in self.slot_bufs[slot] if k != "h_out"]:
            del self.slot_bufs[slot][k]

    def _buf(self, slot, name, numel, host=False):
        b = self.slot_bufs[slot].get(name)
        if b is None or b.numel() < numel:
            if host:
                b = self.torch.empty(self._alloc_numel(numel), dtype=self.torch.float32, pin_memory=True)
            else:
                with self.torch.cuda.stream(self.streams[slot]):
                    b = self.torch.empty(self._alloc_numel(numel), dtype=self.torch.float32, device=self.device)
            self.slot_bufs[slot][name] = b
        return b

    def begin(self, req, slot):
        torch = self.torch
        T = self.textures[req.texture]
        d = req.coords.shape[1]
        d_coords = self._buf(slot, "coords", req.n * d)[: req.n * d].view(req.n, d)
        d_lod = None if req.lod is None else self._buf(slot, "lod", req.n)[: req.n]
        d_out = self._buf(slot, "out", req.n * T.channels)[: req.n * T.channels].view(req.n, T.channels)
        h_out = self._buf(slot, "h_out", req.n * T.channels, host=True)[: req.n * T.channels].view(req.n, T.channels)
        params = stf.make_params(req.filter, seed=req.seed, level_mode=req.level_mode)
        return {"T": T, "d_coords": d_coords, "d_lod": d_lod, "d_out": d_out, "h_out": h_out,
                "params": params}

    def launch_chunk(self, st, req, slot, a, b):
        torch = self.torch
        s = self.streams[slot]
        with torch.cuda.stream(s):
            st["d_coords"][a:b].copy_(req.coords[a:b], non_blocking=True)
            lod = None
            if req.lod is not None:
                st["d_lod"][a:b].copy_(req.lod[a:b], non_blocking=True)
                lod = st["d_lod"][a:b]
            p = st["params"]
            p.query_offset = a
            if req.stochastic:
                stf.stf_lookup_batch(st["T"].handle, p, st["d_coords"][a:b], lod, b - a,
                                     st["d_out"][a:b], None, s)
            else:
                stf.stf_lookup_batch_deterministic(st["T"].handle, p, st["d_coords"][a:b], lod,
                                                   b - a, st["d_out"][a:b], s)
            st["h_out"][a:b].copy_(st["d_out"][a:b], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return ev

    def chunk_done(self, ev):
        return ev.query()

    def finish(self, st, req):
        if self.on_result is not None:
            self.on_result(req, st["h_out"])
        return st["h_out"].clone() if self.keep_results else None


def poisson_requests(n, rate_per_s, sizes, make, seed=6):
    """n requests with exponential inter-arrival times (Poisson process of the given
    rate) and log-uniform sizes in [sizes[0], sizes[1]]; make(i, size, rng) builds
    each Request (its arrival is filled in here)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    lo, hi = math.log(sizes[0]), math.log(sizes[1])
    for i in range(n):
        t += rng.exponential(1.0 / rate_per_s)
        size = int(round(math.exp(rng.uniform(lo, hi))))
        r = make(i, size, rng)
        r.arrival = t
        out.append(r)
    return out


def latency_summary(done):
    lat = sorted(r.latency for r in done)
    if not lat:
        return {}
    pick = lambda p: lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]
    return {"p50_ms": 1e3 * pick(50), "p99_ms": 1e3 * pick(99), "mean_ms": 1e3 * sum(lat) / len(lat),
            "requests": len(lat)}
