"""Continuous-batching streaming server for the tokenizer (encode -> drop -> decode per chunk).

Each video stream delivers frames at `fps`; chunk 0 is its first frame, chunk
k >= 1 frames 4k-3..4k (ready when frame 4k has arrived). A chunk is encoded
with the stream's on-device conv caches, its tokens are dropped at a per-chunk
rate (zero fill, Sec. 6.2) and decoded back, again through the stream's
caches. Latency of a chunk = time its decoded frames are ready on the device
minus the time its last frame arrived.

Scheduling:
  * lanes: L executors (tokenizer contexts with their own workspace and CUDA
    stream). A lane runs one batch at a time: up to `max_batch` chunks of
    different streams in one grouped pass (one conv launch per layer over all
    of them); chunks on different lanes overlap on the GPU. Requests that
    arrive while others run take a lane as soon as one frees up (continuous
    batching), never waiting for a batch to fill.
  * priority classes (when a per-chunk service-time estimate is given): a
    chunk that can meet the latency target on its own is urgent; the others
    (a resolution too large for the target) are background. Lane 0 runs
    urgent chunks only, on the highest-priority CUDA stream, so an urgent
    chunk waits at most for one background kernel, never for a whole
    background chunk; it batches urgent chunks only while the batch still
    meets every member's deadline. The other lanes run background chunks at
    low priority. Without an estimate every lane takes any chunk.
  * phase alignment (`align_phases`): urgent streams are periodic (a chunk
    every 4/fps s), and a stream's source starts sending when the server
    admits it, so admission may choose the start within one period: the
    earliest offset whose chunk window [offset, offset + service) does not
    overlap the windows of the urgent streams already admitted (modulo the
    period). An urgent stream for which no such window exists waits for
    admission, like one that finds no free slot. The offset is part of the
    reported admission wait; chunk latencies are still counted from each
    chunk's last frame.
  * admission: a stream is admitted when its conv caches fit in device memory
    and its compute demand fits the compute budget; otherwise it waits in
    arrival order. Memory: with a byte budget (from free device memory,
    cudaMemGetInfo, in GpuExecutor.memory_budget) a stream of H x W takes
    tok_stream_bytes(H, W); a stream's caches (a slot) are opened when no
    free slot of its resolution exists and the bytes fit, kept when the
    stream ends and handed to the next stream of that resolution, and free
    slots of other resolutions are closed when a new one does not fit
    otherwise (MemoryPool); a fixed slot table per resolution is the other
    form. Compute: with per-chunk service times and a load bound, a stream
    demands service time x chunks per second of the GPU and is admitted
    while the admitted streams' sum stays within the bound (the service
    times are measured on chunks, not derived from clip throughput);
    otherwise FLOP/s at its frame rate against a FLOP/s budget.
  * dispatch: among ready chunks of admitted streams (one in flight per
    stream, in order), earliest deadline first (deadline = ready + target).
  * a stream whose next chunk has not arrived `stall_timeout` after it was
    due is closed and its slot released (host-side failure detection).

The executor is injected: `GpuExecutor` drives the CUDA library; tests use a
fake with simulated durations to check the scheduling logic on the CPU.
"""
from __future__ import annotations

import dataclasses
import heapq
import time
from typing import Callable

FLOP_PER_PIXEL = 3.94e6  # encoder + decoder of the default tokenizer, per input pixel


@dataclasses.dataclass
class StreamSpec:
    sid: int
    H: int
    W: int
    start: float            # arrival time of frame 0 (s, relative to the run start)
    n_chunks: int           # chunk 0 plus n_chunks-1 chunks of 4 frames
    fps: float = 30.0
    stop_after: int | None = None  # the source stops delivering after this many chunks (stall)

    def ready_time(self, k: int, t0: float | None = None) -> float:
        """When chunk k's last frame has arrived; the source starts sending at t0 (its
        admission; a stream is not sent before the server accepts it)."""
        base = self.start if t0 is None else t0
        return base + (0.0 if k == 0 else 4 * k / self.fps)

    def demand_flops(self) -> float:
        return FLOP_PER_PIXEL * self.H * self.W * self.fps


@dataclasses.dataclass
class StreamState:
    spec: StreamSpec
    slot: object = None
    next_chunk: int = 0
    in_flight: bool = False
    admitted_at: float | None = None
    done: bool = False
    timed_out: bool = False
    latencies: list = dataclasses.field(default_factory=list)
    waits: list = dataclasses.field(default_factory=list)   # ready -> dispatched
    runs: list = dataclasses.field(default_factory=list)    # dispatched -> done


class SlotTable:
    """A fixed number of preallocated cache slots per resolution."""

    def __init__(self, slots_per_res: dict):
        self.free = {res: list(range(n)) for res, n in slots_per_res.items()}

    def acquire(self, res):
        return self.free[res].pop() if self.free.get(res) else None

    def release(self, res, slot):
        self.free[res].append(slot)


class MemoryPool:
    """Cache slots admitted by device memory. A stream of resolution `res` needs
    `ex.stream_bytes(res)` bytes; the slots ever opened (`ex.open_slot(res)`) may
    hold at most `budget` bytes together. A released slot stays open for the next
    stream of its resolution; a new slot that does not fit closes free slots of
    other resolutions (largest first, `ex.close_slot`) before giving up."""

    def __init__(self, ex, budget_bytes: float):
        self.ex = ex
        self.budget = budget_bytes
        self.allocated = 0.0
        self.free: dict = {}
        self.opened: dict = {}

    def acquire(self, res):
        if self.free.get(res):
            return self.free[res].pop()
        need = self.ex.stream_bytes(res)
        while self.allocated + need > self.budget:
            others = sorted((r for r, v in self.free.items() if v and r != res),
                            key=lambda r: -self.ex.stream_bytes(r))
            if not others:
                return None
            r = others[0]
            self.ex.close_slot(r, self.free[r].pop())
            self.allocated -= self.ex.stream_bytes(r)
            self.opened[r] -= 1
        slot = self.ex.open_slot(res)
        self.allocated += need
        self.opened[res] = self.opened.get(res, 0) + 1
        return slot

    def release(self, res, slot):
        self.free.setdefault(res, []).append(slot)


class Server:
    def __init__(self, executor, n_lanes: int, slots_per_res, budget_flops: float,
                 target_latency: float = 0.033, stall_timeout: float = 0.5,
                 clock: Callable[[], float] | None = None, sleep: Callable[[float], None] | None = None,
                 service_time: Callable[[StreamSpec], float] | None = None, max_batch: int = 1,
                 align_phases: bool = False, guard_s: float = 0.002, load: float | None = None):
        """slots_per_res: {(H, W): n} (a fixed slot table) or a MemoryPool.
        load: with service_time, admit while the admitted streams' GPU time per
        second (chunk service time x chunks per second) stays within `load`
        (budget_flops is then unused)."""
        self.ex = executor
        self.n_lanes = n_lanes
        self.service_time = service_time
        self.max_batch = max(1, max_batch)
        self.align = align_phases and service_time is not None
        self.guard = guard_s
        self.windows: dict[int, tuple[float, float, float]] = {}  # sid -> (start, length, period)
        self.slots = slots_per_res if hasattr(slots_per_res, "acquire") else SlotTable(slots_per_res)
        self.load = load if service_time is not None else None
        self.budget = budget_flops
        self.target = target_latency
        self.stall_timeout = stall_timeout
        self.clock = clock or time.perf_counter
        self.sleep = sleep or time.sleep

    def run(self, specs: list[StreamSpec], horizon: float, poll_s: float = 2e-4, hard_stop: float | None = None):
        t0 = self.clock()
        now = lambda: self.clock() - t0  # noqa: E731
        states = {s.sid: StreamState(s) for s in specs}
        arrivals = sorted(specs, key=lambda s: s.start)
        ai = 0
        waiting: list[StreamState] = []
        active: list[StreamState] = []
        lanes: list = [None] * self.n_lanes      # list of (state, chunk, ready_t) or None
        used = 0.0
        max_admitted = 0
        admitted_total = 0
        hard = hard_stop if hard_stop is not None else horizon * 3 + 10
        while True:
            t = now()
            # 1. completions
            for li, jobs in enumerate(lanes):
                if jobs is None or not self.ex.done(li):
                    continue
                tdone = now()
                for st, k, ready, tsub in jobs:
                    st.latencies.append(tdone - ready)
                    st.waits.append(tsub - ready)
                    st.runs.append(tdone - tsub)
                    st.in_flight = False
                    st.next_chunk = k + 1
                    if st.next_chunk >= st.spec.n_chunks:
                        st.done = True
                lanes[li] = None
            # 2. retire finished / stalled streams
            for st in list(active):
                if st.in_flight:
                    continue
                stalled = (not st.done and st.spec.stop_after is not None and st.next_chunk >= st.spec.stop_after
                           and t > st.spec.ready_time(st.next_chunk, st.admitted_at) + self.stall_timeout)
                if st.done or stalled:
                    st.timed_out = stalled
                    st.done = True
                    active.remove(st)
                    self.windows.pop(st.spec.sid, None)
                    used -= self._demand(st.spec)
                    self.ex.release(st.spec, st.slot)
                    self.slots.release((st.spec.H, st.spec.W), st.slot)
            # 3. arrivals and admission (arrival order)
            while ai < len(arrivals) and arrivals[ai].start <= t and arrivals[ai].start <= horizon:
                waiting.append(states[arrivals[ai].sid])
                ai += 1
            while waiting:
                st = waiting[0]
                res = (st.spec.H, st.spec.W)
                cap = self.load if self.load is not None else self.budget
                if used + self._demand(st.spec) > cap:
                    break
                off = self._offset(st.spec, t, commit=False)
                if off is None:
                    break
                slot = self.slots.acquire(res)
                if slot is None:
                    break
                self._offset(st.spec, t)
                waiting.pop(0)
                st.slot = slot
                self.ex.attach(st.spec, st.slot)
                st.admitted_at = t + off
                used += self._demand(st.spec)
                active.append(st)
                admitted_total += 1
            max_admitted = max(max_admitted, len(active))
            # 4. dispatch: earliest deadline first
            ready = []
            for st in active:
                k = st.next_chunk
                if st.in_flight or st.done or k >= st.spec.n_chunks:
                    continue
                if st.spec.stop_after is not None and k >= st.spec.stop_after:
                    continue
                rt = st.spec.ready_time(k, st.admitted_at)
                if rt <= t:
                    heapq.heappush(ready, (rt + self.target, st.spec.sid, st, k, rt))
            ready.sort(key=lambda e: (e[0], e[1]))
            for li in range(self.n_lanes):
                if lanes[li] is not None or not ready:
                    continue
                batch = self._pick(li, ready, t)
                if not batch:
                    continue
                picked = {id(e) for e in batch}
                ready = [e for e in ready if id(e) not in picked]
                for e in batch:
                    e[2].in_flight = True
                lanes[li] = [(e[2], e[3], e[4], t) for e in batch]
                self.ex.submit(li, [(e[2].spec, e[2].slot, e[3]) for e in batch])
            # 5. termination
            idle = all(j is None for j in lanes)
            if ai >= len(arrivals) and not waiting and not active and idle:
                break
            if t > hard:
                break
            if t > horizon and idle and not active:
                break
            self.sleep(poll_s)
        return self._report(states, max_admitted, admitted_total, now())

    def _demand(self, spec) -> float:
        """A stream's share of the compute budget: GPU seconds per second (with a load
        bound and service times) or FLOP/s."""
        if self.load is not None:
            return self.service_time(spec) * spec.fps / 4.0
        return spec.demand_flops()

    def _offset(self, spec, t, commit: bool = True) -> float | None:
        """Start offset (s) of a newly admitted stream: 0 unless phases are aligned; then
        the earliest offset in [0, period) whose window avoids every admitted urgent
        stream's window, or None when there is none (the stream waits). commit=False
        only looks."""
        if not self.align or not self.urgent(spec):
            return 0.0
        period = 4.0 / spec.fps
        d = self.service_time(spec) + self.guard

        def clear(a0):
            for b0, db, pb in self.windows.values():
                if abs(pb - period) > 1e-9:
                    continue
                if (b0 - a0) % period < d or (a0 - b0) % period < db:
                    return False
            return True

        cands = sorted({0.0} | {(b0 + db - t) % period for b0, db, _ in self.windows.values()})
        off = next((c for c in cands if clear(t + c)), None)
        if off is not None and commit:
            self.windows[spec.sid] = (t + off, d, period)
        return off

    def urgent(self, spec) -> bool:
        """A chunk that can meet the latency target when it runs alone."""
        return self.service_time is None or self.service_time(spec) <= self.target

    def _pick(self, li, ready, t):
        """Chunks (EDF-sorted entries of `ready`) for free lane li."""
        if self.service_time is None or self.n_lanes == 1:
            return ready[:self.max_batch]
        if li == 0:
            # urgent lane: EDF, batched only while every member still meets its deadline
            batch, total = [], 0.0
            for e in ready:
                if not self.urgent(e[2].spec):
                    continue
                d = self.service_time(e[2].spec)
                if batch and (len(batch) >= self.max_batch or t + total + d > min(x[0] for x in batch)):
                    break
                batch.append(e)
                total += d
            return batch
        return [e for e in ready if not self.urgent(e[2].spec)][:self.max_batch]

    def _report(self, states, max_admitted, admitted_total, elapsed):
        import statistics as stats
        lat_all = [x for s in states.values() for x in s.latencies]
        by_res, waits, runs = {}, {}, {}
        for s in states.values():
            r = f"{s.spec.H}x{s.spec.W}"
            by_res.setdefault(r, []).extend(s.latencies)
            waits.setdefault(r, []).extend(s.waits)
            runs.setdefault(r, []).extend(s.runs)

        def pct(v, q):
            if not v:
                return None
            v = sorted(v)
            return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]

        frames = sum((1 + 4 * (len(s.latencies) - 1)) if s.latencies else 0 for s in states.values())
        return {
            "streams": len(states), "admitted_total": admitted_total, "max_concurrent": max_admitted,
            "timed_out": sum(1 for s in states.values() if s.timed_out),
            "never_admitted": sum(1 for s in states.values() if s.admitted_at is None),
            "chunks": len(lat_all), "frames": frames, "elapsed_s": elapsed,
            "frames_per_s": frames / elapsed if elapsed > 0 else None,
            "p50_ms": 1e3 * pct(lat_all, 0.5) if lat_all else None,
            "p99_ms": 1e3 * pct(lat_all, 0.99) if lat_all else None,
            "mean_ms": 1e3 * stats.fmean(lat_all) if lat_all else None,
            "by_resolution": {r: {"chunks": len(v), "p50_ms": 1e3 * pct(v, 0.5) if v else None,
                                  "p90_ms": 1e3 * pct(v, 0.9) if v else None,
                                  "p99_ms": 1e3 * pct(v, 0.99) if v else None,
                                  "over_target": sum(1 for x in v if x > self.target),
                                  "wait_p50_ms": 1e3 * pct(waits[r], 0.5) if waits[r] else None,
                                  "wait_p99_ms": 1e3 * pct(waits[r], 0.99) if waits[r] else None,
                                  "run_p50_ms": 1e3 * pct(runs[r], 0.5) if runs[r] else None,
                                  "run_p99_ms": 1e3 * pct(runs[r], 0.99) if runs[r] else None}
                              for r, v in by_res.items()},
            "admission_wait_s": {s.spec.sid: (s.admitted_at - s.spec.start) for s in states.values()
                                 if s.admitted_at is not None},
            "admission_wait_p50_s": pct([s.admitted_at - s.spec.start for s in states.values()
                                         if s.admitted_at is not None], 0.5),
        }


class GpuExecutor:
    """Runs chunks through the CUDA library: one tokenizer context + CUDA stream per lane
    (lane 0 on the highest stream priority when `priorities`), stream-cache slots per
    resolution (preallocated from `slots_per_res`, or opened and closed by a MemoryPool
    on the executor's stream_bytes / open_slot / close_slot), one content loop per
    stream. A submitted batch is one grouped encode, a drop mask per chunk and one
    grouped decode."""

    def __init__(self, n_lanes: int, params: dict, slots_per_res: dict | None = None, drop_seed: int = 1000,
                 drop_range=(0.0, 0.30), content_frames: int = 9, keep_outputs: bool = False,
                 arch: dict | None = None, content_fn=None, max_batch: int = 1, priorities: bool = False,
                 resolutions=None):
        import numpy as np
        import torch

        from . import _lib
        from . import tokenizer as tkz
        self.torch = torch
        self.tkz = tkz
        self.lib = _lib
        arch = arch or {}
        self.lanes = []
        for li in range(n_lanes):
            tk = tkz.Tokenizer("bf16", **arch)
            tk.set_params(params)
            # lower number = higher priority; out-of-range values map to the nearest valid one
            prio = -100 if (priorities and li == 0) else 0
            if priorities and li > 0:
                tk.set_cta_tiles(1)  # background conv CTAs of one tile: SMs free up every few tens of us
            self.lanes.append({"tk": tk, "stream": torch.cuda.Stream(priority=prio), "event": None})
        tk0 = self.lanes[0]["tk"]
        self.levels = tk0.levels
        self.s_t = tk0.s_t
        self.slots = {}
        self.max_batch = max(1, max_batch)
        res = list(slots_per_res) if slots_per_res else list(resolutions)
        big = max(res, key=lambda r: r[0] * r[1])
        nb = min(self.max_batch, sum(slots_per_res.values())) if slots_per_res else self.max_batch
        for lane in self.lanes:
            lane["tk"].reserve_batch([(1, self.s_t, *big)] * nb)
        for (H, W), n in (slots_per_res or {}).items():
            self.slots[(H, W)] = [tk0.stream_open(H, W) for _ in range(n)]
        self.bufs = {}
        self.drop_seed = drop_seed
        self.drop_range = drop_range
        self.content_frames = content_frames
        self.content_fn = content_fn
        self.content = {}
        self.content_ready = {}
        self.side = torch.cuda.Stream()  # content preparation, off the lanes and off the host
        self.keep = keep_outputs
        self.outputs = {}
        self.tokens = {}
        self._np = np

    # -- memory admission (MemoryPool) ------------------------------------------
    def stream_bytes(self, res) -> int:
        """Device bytes one stream of resolution res holds: its conv caches
        (tok_stream_bytes) plus its source frames and its chunk's token and output
        buffers."""
        H, W = res
        caches = self.lanes[0]["tk"].stream_bytes(H, W)
        Tq, Hq, Wq = self.lanes[0]["tk"].latent_shape(1, H, W)
        bufs = 3 * Hq * Wq * 4 + (self.s_t + 1) * H * W * 3 * 4
        return caches + bufs + self.content_frames * H * W * 3 * 2

    def open_slot(self, res) -> int:
        hs = self.slots.setdefault(res, [])
        for i, h in enumerate(hs):
            if h is None:
                hs[i] = self.lanes[0]["tk"].stream_open(*res)
                return i
        hs.append(self.lanes[0]["tk"].stream_open(*res))
        return len(hs) - 1

    def close_slot(self, res, slot) -> None:
        self.torch.cuda.synchronize()  # no lane may still run a chunk on these caches
        self.lanes[0]["tk"].stream_close(self.slots[res][slot])
        self.slots[res][slot] = None
        self.bufs.pop((res[0], res[1], slot), None)

    def memory_budget(self, reserve_bytes: float = 4e9, fraction: float = 0.9) -> float:
        """Bytes of stream state the device can still hold: the free device memory
        (cudaMemGetInfo) after the lanes' workspaces, less a reserve, times `fraction`."""
        self.torch.cuda.synchronize()
        free, _ = self.torch.cuda.mem_get_info()
        return max(0.0, (free - reserve_bytes) * fraction)

    def _content(self, spec):
        """The stream's source frames on the device, made on a side stream (an event marks
        them ready; the lanes wait for it on the device, the host never blocks)."""
        key = spec.sid
        if key not in self.content:
            torch = self.torch
            with torch.cuda.stream(self.side):
                if self.content_fn is not None:
                    clip = self.content_fn(spec)
                else:
                    import synthetic as S
                    clip = S.moving_rects_clip(100 + spec.sid, self.content_frames, spec.H, spec.W)
                if not isinstance(clip, torch.Tensor):
                    clip = torch.from_numpy(clip)
                clip = clip.to("cuda", torch.bfloat16, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.side)
            self.content[key] = clip
            self.content_ready[key] = ev
        return self.content[key]

    def attach(self, spec, slot):
        self._content(spec)
        self.lanes[0]["tk"].stream_reset(self.slots[(spec.H, spec.W)][slot])

    def release(self, spec, slot):
        self.content.pop(spec.sid, None)
        self.content_ready.pop(spec.sid, None)

    def _bufs(self, H, W, slot):
        """Token and output buffers of one stream slot (one chunk of a stream is in flight
        at a time, so a slot's buffers are never shared by two running chunks)."""
        key = (H, W, slot)
        if key not in self.bufs:
            torch = self.torch
            Tq, Hq, Wq = self.lanes[0]["tk"].latent_shape(1, H, W)
            self.bufs[key] = {
                "idx": torch.empty((1, 1, Hq, Wq), device="cuda", dtype=torch.int32),
                "idx_d": torch.empty((1, 1, Hq, Wq), device="cuda", dtype=torch.int32),
                "kb": torch.empty((1, 1, Hq, (Wq + 31) // 32), device="cuda", dtype=torch.int32),
                "xh": torch.empty((1, self.s_t, H, W, 3), device="cuda", dtype=torch.float32),
                "xh1": torch.empty((1, 1, H, W, 3), device="cuda", dtype=torch.float32),
            }
        return self.bufs[key]

    def calibrate(self, reps: int = 5, resolutions=None) -> dict:
        """Seconds one chunk of each resolution takes alone on lane 0 (median of `reps`
        steady-state chunks through a stream slot opened for it and closed after)."""
        torch = self.torch
        out = {}
        for (H, W) in (resolutions or list(self.slots)):
            spec = StreamSpec(-1 - len(out), H, W, 0.0, reps + 1)
            slot = self.open_slot((H, W))
            self.attach(spec, slot)
            times = []
            for k in range(reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(self.lanes[0]["stream"])
                self.submit(0, [(spec, slot, k)])
                e1.record(self.lanes[0]["stream"])
                e1.synchronize()
                if k > 0:
                    times.append(e0.elapsed_time(e1) / 1e3)
            self.release(spec, slot)
            self.close_slot((H, W), slot)
            out[(H, W)] = sorted(times)[len(times) // 2]
        return out

    def chunk_frames(self, spec, k):
        clip = self._content(spec)
        n = clip.shape[0]
        if k == 0:
            ids = [0]
        else:
            ids = [(4 * k - 3 + i) % n for i in range(4)]
        return clip[ids][None].contiguous()

    def submit(self, li, jobs):
        """jobs: list of (spec, slot, chunk index) of distinct streams, run as one batch."""
        torch = self.torch
        lane = self.lanes[li]
        tk = lane["tk"]
        st = lane["stream"]
        L = self.lib
        with torch.cuda.stream(st):
            enc, dec, drops = [], [], []
            for spec, _, _ in jobs:
                self._content(spec)
                st.wait_event(self.content_ready[spec.sid])
            for spec, slot, k in jobs:
                vid = self.slots[(spec.H, spec.W)][slot]
                b = self._bufs(spec.H, spec.W, slot)
                x = self.chunk_frames(spec, k)
                b["x"] = x  # keep the chunk alive until the batch has run
                T = x.shape[1]
                enc.append((x.data_ptr(), 1, T, spec.H, spec.W, None, b["idx"].data_ptr(), vid))
                Tq, Hq, Wq = b["idx"].shape[1:]
                xh = b["xh"] if k > 0 else b["xh1"]
                dec.append((b["idx_d"].data_ptr(), 1, Tq, Hq, Wq, spec.H, spec.W, xh.data_ptr(), vid))
                drops.append((spec, k, b))
            L.tok_encode_batch(tk.ctx, enc, st.cuda_stream)
            for spec, k, b in drops:
                rate = float(self._np.random.default_rng([self.drop_seed + spec.sid, k]).uniform(*self.drop_range))
                self.tkz.drop_mask(b["idx"], rate, seed=self.drop_seed + spec.sid, stream_id=spec.sid, chunk_id=k,
                                   levels=self.levels, out=b["idx_d"], keep_bits=b["kb"], stream=st)
            L.tok_decode_batch(tk.ctx, dec, st.cuda_stream)
            if self.keep:
                for spec, k, b in drops:
                    self.outputs.setdefault(spec.sid, []).append((b["xh"] if k > 0 else b["xh1"]).clone())
                    self.tokens.setdefault(spec.sid, []).append(b["idx_d"].clone())
            ev = torch.cuda.Event()
            ev.record(st)
        lane["event"] = ev

    def done(self, li):
        ev = self.lanes[li]["event"]
        return ev is None or ev.query()

    def status(self):
        return [lane["tk"].status() for lane in self.lanes]

    def close(self):
        for (H, W), hs in self.slots.items():
            for h in hs:
                if h is not None:
                    self.lanes[0]["tk"].stream_close(h)
        for lane in self.lanes:
            lane["tk"].close()
