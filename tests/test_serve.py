"""The continuous-batching loop's admission logic without a GPU (FakeExecutor on
a virtual clock): every request completes, the memory budget is never
exceeded, admission follows arrival order, concurrency stays within the
slots, plans are reused per size class, and a request too large for the
budget is rejected instead of blocking the queue."""
import pytest

from paper_2103_01874_gb300 import serve


class VClock:
    def __init__(self, tick=1e-4):
        self.t = 0.0
        self.tick = tick

    def __call__(self):
        self.t += self.tick
        return self.t

    def sleep(self, dt):
        self.t += dt


class Watch(serve.Server):
    """Server that asserts the budget after every admission."""

    def _evict_for(self, need):
        ok = super()._evict_for(need)
        if ok:
            assert self._in_use() + need <= self.budget
        return ok


def _run(reqs, budget, slots=4, dur=lambda r: 0.002 * (r.shape[0] / 32) ** 3):
    clk = VClock()
    ex = serve.FakeExecutor(dur, clk)
    srv = Watch(ex, budget, slots)
    stats, res = srv.run(reqs, clock=clk, sleep=clk.sleep, keep={r.rid for r in reqs})
    return srv, ex, stats, res


SHAPES = [(32, 32, 32), (48, 32, 64), (64, 64, 64), (96, 64, 96)]


def test_all_complete_in_order_within_budget():
    reqs = serve.poisson_requests(200, rate=2000.0, shapes=SHAPES, seed=1)
    budget = 12 * 8 * 11 * 96 * 64 * 96
    srv, ex, st, res = _run(reqs, budget)
    assert st.completed == 200 and st.rejected == 0 and len(res) == 200
    assert st.peak_bytes <= budget
    assert 1 <= st.max_active <= 4
    order = sorted(reqs, key=lambda r: r.arrival)
    adm = [r.admitted for r in order]
    assert adm == sorted(adm), "admission follows arrival order"
    assert all(r.done >= r.admitted >= r.arrival for r in reqs)
    assert st.latency_ms_p99 >= st.latency_ms_p50 > 0
    # plans are reused: far fewer creations than requests
    assert st.plans_created <= 4 * len(SHAPES) * 2
    assert not ex.live


def test_tight_budget_serialises_and_evicts():
    # two size classes of equal footprint and a budget for one request at a time:
    # requests run one by one and the other class's idle plan is evicted
    shapes = [(96, 64, 96), (64, 96, 96)]
    reqs = serve.poisson_requests(60, rate=5000.0, shapes=shapes, seed=2)
    one = 8 * 11 * 96 * 64 * 96 + 4 * 96 * 64 * 96
    srv, ex, st, _ = _run(reqs, budget=one, slots=8)
    assert st.completed == 60
    assert st.max_active == 1
    assert st.evictions > 0
    assert st.peak_bytes <= one


def test_small_requests_share_a_budget_sized_for_a_large_one():
    reqs = serve.poisson_requests(80, rate=5000.0, shapes=SHAPES, seed=4)
    one = 8 * 11 * 96 * 64 * 96 + 4 * 96 * 64 * 96
    srv, ex, st, _ = _run(reqs, budget=one, slots=8)
    assert st.completed == 80 and st.peak_bytes <= one
    assert st.max_active > 1  # several small requests fit together


def test_oversized_request_is_rejected_not_blocking():
    reqs = serve.poisson_requests(20, rate=1000.0, shapes=[(32, 32, 32)], seed=3)
    reqs.insert(5, serve.Request(999, (512, 512, 512), 1, 0, reqs[4].arrival))
    srv, ex, st, _ = _run(reqs, budget=50_000_000)
    assert st.rejected == 1 and st.completed == 20


def test_reserve_builds_a_resident_pool_within_budget():
    clk = VClock()
    ex = serve.FakeExecutor(lambda r: 0.002, clk)
    classes = [(s, p) for s in SHAPES for p in (0, 1)]
    srv = Watch(ex, 10 ** 12, slots=4)
    assert srv.reserve(classes, per_class=2) == 2 * len(classes)
    assert srv.reserve(classes, per_class=2) == 0          # already resident
    reqs = serve.poisson_requests(100, rate=2000.0, shapes=SHAPES, seed=3)
    before = srv.plans_created
    st, _ = srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert st.completed == 100
    assert srv.plans_created - before <= 2 * len(classes)  # the pool absorbs most of the traffic
    # a tight budget stops the reservation
    tight = Watch(serve.FakeExecutor(lambda r: 0.002, VClock()), ex.plan_bytes_for(SHAPES[0], 0) + 1, slots=4)
    assert tight.reserve(classes, per_class=2) == 1
