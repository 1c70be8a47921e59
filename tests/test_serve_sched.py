"""Host-side scheduling of the streaming server, on the CPU with a fake executor
and a virtual clock: continuous admission as slots and compute free up,
earliest-deadline-first dispatch, in-order chunks per stream, and the stall
timeout that releases a stream whose source stopped (failure detection on the
host, no GPU involved)."""
from paper_2602_03529_b300.serve import Server, StreamSpec


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeExec:
    """Each chunk takes `dur[(H, W)]` seconds; lanes run in parallel."""

    def __init__(self, clock, dur):
        self.clock, self.dur = clock, dur
        self.finish = {}
        self.log = []
        self.attached = []

    def attach(self, spec, slot):
        self.attached.append((spec.sid, slot, self.clock()))

    def release(self, spec, slot):
        pass

    def submit(self, li, spec, slot, k):
        self.finish[li] = self.clock() + self.dur[(spec.H, spec.W)]
        self.log.append((self.clock(), spec.sid, k, li))

    def done(self, li):
        return self.clock() >= self.finish.get(li, 0.0)


def _server(clock, ex, lanes=2, slots=None, budget=1e30):
    return Server(ex, lanes, slots or {(8, 8): 4}, budget, target_latency=0.033, stall_timeout=0.2,
                  clock=clock, sleep=clock.sleep)


def test_all_chunks_in_order_and_latency_alone():
    c = Clock()
    ex = FakeExec(c, {(8, 8): 0.010})
    specs = [StreamSpec(0, 8, 8, start=0.0, n_chunks=5)]
    rep = _server(c, ex).run(specs, horizon=1.0, poll_s=1e-3)
    ks = [k for _, sid, k, _ in ex.log]
    assert ks == [0, 1, 2, 3, 4]
    assert rep["chunks"] == 5 and rep["frames"] == 17
    assert 9.0 <= rep["p50_ms"] <= 12.0 and rep["p99_ms"] <= 12.0


def test_admission_waits_for_a_free_slot_then_admits():
    c = Clock()
    ex = FakeExec(c, {(8, 8): 0.005})
    specs = [StreamSpec(i, 8, 8, start=0.01 * i, n_chunks=3) for i in range(5)]
    rep = _server(c, ex, lanes=2, slots={(8, 8): 2}).run(specs, horizon=2.0, poll_s=1e-3)
    assert rep["admitted_total"] == 5 and rep["max_concurrent"] <= 2 and rep["never_admitted"] == 0
    waits = rep["admission_wait_s"]
    assert waits[0] < 0.01 and max(waits.values()) > 0.05   # later streams waited for slots
    assert len({slot for _, slot, _ in ex.attached}) == 2    # the two slots were reused


def test_compute_budget_limits_concurrency():
    c = Clock()
    ex = FakeExec(c, {(8, 8): 0.002})
    spec = lambda i: StreamSpec(i, 8, 8, start=0.0, n_chunks=2)  # noqa: E731
    one = spec(0).demand_flops()
    rep = _server(c, ex, lanes=4, slots={(8, 8): 4}, budget=2.5 * one).run([spec(i) for i in range(4)],
                                                                         horizon=2.0, poll_s=1e-3)
    assert rep["max_concurrent"] == 2 and rep["admitted_total"] == 4


def test_earliest_deadline_first():
    c = Clock()
    ex = FakeExec(c, {(8, 8): 0.050})
    specs = [StreamSpec(i, 8, 8, start=0.0, n_chunks=1) for i in (2, 0, 1)]
    _server(c, ex, lanes=1).run(specs, horizon=1.0, poll_s=1e-3)
    assert [sid for _, sid, _, _ in ex.log] == [0, 1, 2]


def test_stalled_source_times_out_and_frees_its_slot():
    c = Clock()
    ex = FakeExec(c, {(8, 8): 0.005})
    specs = [StreamSpec(0, 8, 8, start=0.0, n_chunks=50, stop_after=2),
             StreamSpec(1, 8, 8, start=0.01, n_chunks=2)]
    rep = _server(c, ex, lanes=1, slots={(8, 8): 1}).run(specs, horizon=3.0, poll_s=1e-3)
    assert rep["timed_out"] == 1
    assert rep["admitted_total"] == 2           # the second stream got the freed slot
    assert [k for _, sid, k, _ in ex.log if sid == 0] == [0, 1]
    assert [k for _, sid, k, _ in ex.log if sid == 1] == [0, 1]
