"""Host-side scheduling of the streaming server, on the CPU with a fake executor
and a virtual clock: continuous admission as slots and compute free up,
earliest-deadline-first dispatch, in-order chunks per stream, urgent and
background lanes, deadline-bounded batching, and the stall timeout that
releases a stream whose source stopped (failure detection on the host, no GPU
involved)."""
from paper_2602_03529_b300.serve import Server, StreamSpec


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeExec:
    """Each chunk takes `dur[(H, W)]` seconds, a batch the sum of its chunks; lanes run
    in parallel."""

    def __init__(self, clock, dur):
        self.clock, self.dur = clock, dur
        self.finish = {}
        self.log = []
        self.batches = []
        self.attached = []

    def attach(self, spec, slot):
        self.attached.append((spec.sid, slot, self.clock()))

    def release(self, spec, slot):
        pass

    def submit(self, li, jobs):
        self.finish[li] = self.clock() + sum(self.dur[(spec.H, spec.W)] for spec, _, _ in jobs)
        for spec, slot, k in jobs:
            self.log.append((self.clock(), spec.sid, k, li))
        self.batches.append((li, [spec.sid for spec, _, _ in jobs]))

    def done(self, li):
        return self.clock() >= self.finish.get(li, 0.0)


def _server(clock, ex, lanes=2, slots=None, budget=1e30, service_time=None, max_batch=1, align=False):
    return Server(ex, lanes, slots or {(8, 8): 4}, budget, target_latency=0.033, stall_timeout=0.2,
                  clock=clock, sleep=clock.sleep, service_time=service_time, max_batch=max_batch,
                  align_phases=align)


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


def test_urgent_lane_takes_only_chunks_that_can_meet_the_target():
    """Small streams (10 ms a chunk) are urgent and run on lane 0; large ones (50 ms,
    above the 33 ms target) run on the background lane and never delay lane 0."""
    c = Clock()
    dur = {(8, 8): 0.010, (16, 16): 0.050}
    ex = FakeExec(c, dur)
    svc = lambda spec: dur[(spec.H, spec.W)]  # noqa: E731
    specs = [StreamSpec(0, 16, 16, start=0.0, n_chunks=4), StreamSpec(1, 8, 8, start=0.001, n_chunks=4),
             StreamSpec(2, 16, 16, start=0.002, n_chunks=4), StreamSpec(3, 8, 8, start=0.003, n_chunks=4)]
    rep = _server(c, ex, lanes=2, slots={(8, 8): 2, (16, 16): 2}, service_time=svc, max_batch=4).run(
        specs, horizon=2.0, poll_s=1e-3)
    assert rep["chunks"] == 16
    for _, sid, _, li in ex.log:
        assert li == (0 if sid in (1, 3) else 1)
    small = rep["by_resolution"]["8x8"]
    assert small["p99_ms"] <= 33.0          # never queued behind a 50 ms chunk
    assert rep["by_resolution"]["16x16"]["chunks"] == 8


def test_urgent_batches_keep_every_deadline():
    """Three urgent chunks ready together, 12 ms each: a batch of three would end at
    36 ms, past the first deadline (33 ms), so lane 0 runs two, then one."""
    c = Clock()
    dur = {(8, 8): 0.012, (16, 16): 0.050}
    ex = FakeExec(c, dur)
    svc = lambda spec: dur[(spec.H, spec.W)]  # noqa: E731
    specs = [StreamSpec(i, 8, 8, start=0.0, n_chunks=1) for i in range(3)]
    _server(c, ex, lanes=2, slots={(8, 8): 3, (16, 16): 1}, service_time=svc, max_batch=8).run(
        specs, horizon=1.0, poll_s=1e-3)
    assert [len(b) for _, b in ex.batches] == [2, 1]
    assert all(li == 0 for li, _ in ex.batches)


def test_background_lane_batches_up_to_max_batch():
    c = Clock()
    dur = {(8, 8): 0.005, (16, 16): 0.050}
    ex = FakeExec(c, dur)
    svc = lambda spec: dur[(spec.H, spec.W)]  # noqa: E731
    specs = [StreamSpec(i, 16, 16, start=0.0, n_chunks=1) for i in range(5)]
    _server(c, ex, lanes=2, slots={(8, 8): 1, (16, 16): 5}, service_time=svc, max_batch=3).run(
        specs, horizon=1.0, poll_s=1e-3)
    assert [len(b) for _, b in ex.batches] == [3, 2]
    assert all(li == 1 for li, _ in ex.batches)


def test_phase_alignment_removes_collisions_between_urgent_streams():
    """Four urgent streams of 20 ms chunks arriving together: unaligned, their chunks
    queue behind each other on the urgent lane (up to 80 ms); aligned, each stream
    starts in its own 20 ms window of the 133 ms period and no chunk waits."""
    dur = {(8, 8): 0.020, (16, 16): 0.050}
    svc = lambda spec: dur[(spec.H, spec.W)]  # noqa: E731
    reps = {}
    for align in (False, True):
        c = Clock()
        ex = FakeExec(c, dur)
        specs = [StreamSpec(i, 8, 8, start=0.0005 * i, n_chunks=6) for i in range(4)]
        reps[align] = _server(c, ex, lanes=2, slots={(8, 8): 4, (16, 16): 1}, service_time=svc,
                              align=align).run(specs, horizon=3.0, poll_s=5e-4)
    assert reps[False]["p99_ms"] > 60.0
    assert reps[True]["p99_ms"] <= 22.0 and reps[True]["chunks"] == 24
    waits = sorted(reps[True]["admission_wait_s"].values())
    assert waits[-1] < 4 / 30.0                 # every offset is within one period
    assert min(b - a for a, b in zip(waits, waits[1:])) >= 0.020   # disjoint windows


def test_urgent_stream_without_a_free_window_waits_for_admission():
    """Seven urgent streams of 20 ms chunks: only six disjoint 22 ms windows fit in
    the 133 ms period, so the seventh waits until a stream retires."""
    c = Clock()
    dur = {(8, 8): 0.020, (16, 16): 0.050}
    ex = FakeExec(c, dur)
    svc = lambda spec: dur[(spec.H, spec.W)]  # noqa: E731
    specs = [StreamSpec(i, 8, 8, start=0.0, n_chunks=3) for i in range(7)]
    rep = _server(c, ex, lanes=2, slots={(8, 8): 7, (16, 16): 1}, service_time=svc, align=True).run(
        specs, horizon=3.0, poll_s=5e-4)
    assert rep["chunks"] == 21 and rep["p99_ms"] <= 22.0
    waits = sorted(rep["admission_wait_s"].values())
    assert waits[5] < 4 / 30.0 and waits[6] > 0.2   # the 7th waited for a retirement


class FakeMemExec(FakeExec):
    """FakeExec with device memory: a stream of (H, W) holds H * W bytes; slots are
    opened and closed on demand."""

    def __init__(self, clock, dur):
        super().__init__(clock, dur)
        self.opened, self.closed = [], []
        self.n = {}

    def stream_bytes(self, res):
        return res[0] * res[1]

    def open_slot(self, res):
        self.n[res] = self.n.get(res, 0) + 1
        self.opened.append(res)
        return self.n[res] - 1

    def close_slot(self, res, slot):
        self.closed.append((res, slot))


def test_admission_by_memory_reuses_and_reclaims_slots():
    """Memory budget 200 bytes; 8x8 streams take 64, 12x12 streams 144. Three 8x8
    streams fit together (192), the fourth waits for one to end and takes its slot
    (no new allocation); a 12x12 stream that arrives when only free 8x8 slots remain
    closes all three of them to fit (144 + 64 > 200)."""
    from paper_2602_03529_b300.serve import MemoryPool
    c = Clock()
    ex = FakeMemExec(c, {(8, 8): 0.005, (12, 12): 0.005})
    pool = MemoryPool(ex, 200)
    specs = [StreamSpec(i, 8, 8, start=0.001 * i, n_chunks=3) for i in range(4)]
    specs.append(StreamSpec(9, 12, 12, start=1.0, n_chunks=2))
    rep = Server(ex, 2, pool, 1e30, stall_timeout=0.2, clock=c, sleep=c.sleep).run(specs, horizon=2.0,
                                                                                    poll_s=1e-3)
    assert rep["admitted_total"] == 5 and rep["never_admitted"] == 0
    assert rep["max_concurrent"] == 3
    waits = rep["admission_wait_s"]
    assert max(waits[i] for i in range(3)) < 0.01 and waits[3] > 0.1   # the 4th waited for memory
    assert ex.opened == [(8, 8)] * 3 + [(12, 12)]                      # its slot was reused
    assert len(ex.closed) == 3 and all(r == (8, 8) for r, _ in ex.closed)
    assert pool.allocated <= 200


def test_compute_admission_by_measured_chunk_time():
    """With service times and a load bound, a stream demands service x chunks per second
    of the GPU: 30 ms chunks at 7.5 chunks/s are 0.225 each, so a 0.5 bound admits two."""
    c = Clock()
    dur = {(8, 8): 0.030}
    ex = FakeExec(c, dur)
    svc = lambda spec: dur[(spec.H, spec.W)]  # noqa: E731
    specs = [StreamSpec(i, 8, 8, start=0.0, n_chunks=3) for i in range(4)]
    rep = Server(ex, 2, {(8, 8): 4}, 0.0, stall_timeout=0.2, clock=c, sleep=c.sleep, service_time=svc,
                 load=0.5).run(specs, horizon=2.0, poll_s=1e-3)
    assert rep["max_concurrent"] == 2 and rep["admitted_total"] == 4
