"""Scheduler logic of the serving loop with a fake device backend (CPU only):
admission by free slots and memory budget, chunking with query offsets,
completion, overlap of admitted requests, rejection of oversize requests."""
import numpy as np
import pytest

from paper_2305_05810_gb300 import serving


class FakeBackend:
    """Chunks complete `latency` ticks after launch; results record the offsets.  Each
    slot's buffers grow to the largest request it has begun and stay until released,
    like the real backend's; `held` is the device bytes they take."""

    def __init__(self, latency=3, channels=1):
        self.t = 0
        self.latency = latency
        self.ch = channels
        self.launched = []
        self.bufs = {}               # slot -> bytes held
        self.max_held = 0

    def channels(self, key):
        return self.ch

    def hold_after(self, slot, req):
        return max(self.bufs.get(slot, 0) if slot is not None else 0, req.device_bytes(self.ch))

    def release(self, slot):
        self.bufs.pop(slot, None)

    @property
    def held(self):
        return sum(self.bufs.values())

    def begin(self, req, slot):
        self.bufs[slot] = self.hold_after(slot, req)
        self.max_held = max(self.max_held, self.held)
        return {"out": np.full(req.n, -1, dtype=np.int64), "slot": slot}

    def launch_chunk(self, st, req, slot, a, b):
        self.launched.append((req.rid, slot, a, b))
        st["out"][a:b] = np.arange(a, b)          # query_offset keyed: request-local index
        return self.t + self.latency

    def chunk_done(self, due):
        return self.t >= due

    def finish(self, st, req):
        return st["out"]


class Coords:
    def __init__(self, n, d=3):
        self.shape = (n, d)


def make_req(rid, n, arrival=0.0):
    return serving.Request(rid, "tex", Coords(n), arrival=arrival)


def drive(sched, be, reqs, max_ticks=10000):
    for r in reqs:
        sched.submit(r)
    for _ in range(max_ticks):
        sched.step()
        be.t += 1
        if sched.idle():
            return
    raise AssertionError("scheduler did not drain")


def test_all_requests_complete_with_full_coverage_and_budget_respected():
    be = FakeBackend()
    budget = 16 * 1000 * 10          # bytes; 16 bytes per query (12 in + 4 out)
    sched = serving.Scheduler(be, n_slots=3, budget_bytes=budget, chunk_queries=700,
                              max_chunks_in_flight=2, clock=lambda: be.t)
    sizes = [100, 5000, 2500, 10000, 1, 3000, 4999, 64]
    reqs = [make_req(i, n) for i, n in enumerate(sizes)]
    drive(sched, be, reqs)
    assert sorted(r.rid for r in sched.done) == list(range(len(sizes)))
    for r in reqs:
        assert np.array_equal(r.result, np.arange(r.n))         # every query covered once
        assert r.t_admit >= 0 and r.t_done >= r.t_admit
    assert sched.peak_in_use <= budget
    assert sched.peak_active <= 3
    assert sched.peak_active >= 2                                # admitted requests overlap
    for rid in range(len(sizes)):
        offs = [(a, b) for (q, _, a, b) in be.launched if q == rid]
        assert offs[0][0] == 0 and offs[-1][1] == sizes[rid]
        assert all(b - a <= 700 for a, b in offs)
        assert all(offs[k][1] == offs[k + 1][0] for k in range(len(offs) - 1))


def test_held_buffers_of_idle_slots_count_against_the_budget():
    """Slots keep their buffers between requests; the device bytes actually held
    (every slot's buffers plus the resident textures) never exceed the budget, and
    idle slots' buffers are released when a request needs the room."""
    be = FakeBackend(latency=2)
    resident = 20000
    budget = resident + 16 * 6000
    sched = serving.Scheduler(be, n_slots=4, budget_bytes=budget, chunk_queries=500,
                              clock=lambda: be.t, resident_bytes=resident)
    rng = np.random.default_rng(1)
    sizes = [int(x) for x in rng.integers(1, 6000, 60)] + [6000, 5999, 1]
    reqs = [make_req(i, n) for i, n in enumerate(sizes)]
    for r in reqs:
        sched.submit(r)
    for _ in range(100000):
        sched.step()
        assert be.held + resident <= budget
        assert sched.in_use == be.held + resident          # the charge is what is held
        be.t += 1
        if sched.idle():
            break
    assert len(sched.done) == len(sizes)
    assert be.max_held + resident <= budget and sched.peak_in_use <= budget
    assert sched.peak_active >= 2


def test_resident_textures_larger_than_budget_are_rejected():
    with pytest.raises(serving.BudgetError):
        serving.Scheduler(FakeBackend(), budget_bytes=1000, resident_bytes=1001)


def test_fifo_admission_waits_for_memory():
    be = FakeBackend(latency=5)
    sched = serving.Scheduler(be, n_slots=4, budget_bytes=16 * 1000, chunk_queries=1000,
                              clock=lambda: be.t)
    big, small = make_req(0, 900), make_req(1, 900)
    sched.submit(big)
    sched.submit(small)
    sched.step()
    assert len(sched.active) == 1 and len(sched.waiting) == 1     # second does not fit yet
    drive(sched, be, [])
    assert [r.rid for r in sched.done] == [0, 1]
    assert small.t_admit >= big.t_done


def test_oversize_request_is_rejected():
    be = FakeBackend()
    sched = serving.Scheduler(be, n_slots=2, budget_bytes=1000, clock=lambda: be.t)
    with pytest.raises(serving.BudgetError) as e:
        sched.submit(make_req(0, 1000))
    assert e.value.status == 7 and sched.rejected


def test_poisson_arrivals_and_sizes():
    reqs = serving.poisson_requests(2000, 100.0, (1000, 4 << 20), lambda i, s, rng: make_req(i, s))
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) > 0)
    assert abs(np.mean(np.diff(arr)) - 0.01) < 0.002
    sizes = np.array([r.n for r in reqs])
    assert sizes.min() >= 1000 and sizes.max() <= 4 << 20
    assert abs(np.median(np.log(sizes)) - (np.log(1000) + np.log(4 << 20)) / 2) < 0.5


def test_latency_summary():
    reqs = [make_req(i, 1) for i in range(100)]
    for i, r in enumerate(reqs):
        r.arrival, r.t_done = 0.0, (i + 1) * 1e-3
    s = serving.latency_summary(reqs)
    assert abs(s["p50_ms"] - 50.5) < 1.0 and abs(s["p99_ms"] - 99.0) < 1.01
