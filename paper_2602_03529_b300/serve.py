"""Continuous-batching streaming server for the tokenizer (encode -> drop -> decode per chunk).

Each video stream delivers frames at `fps`; chunk 0 is its first frame, chunk
k >= 1 frames 4k-3..4k (ready when frame 4k has arrived). A chunk is encoded
with the stream's on-device conv caches, its tokens are dropped at a per-chunk
rate (zero fill, Sec. 6.2) and decoded back, again through the stream's
caches. Latency of a chunk = time its decoded frames are ready on the device
minus the time its last frame arrived.

Scheduling:
  * lanes: L executors (tokenizer contexts with their own workspace and CUDA
    stream). A lane runs one chunk at a time; chunks of different streams on
    different lanes overlap on the GPU. Requests that arrive while others run
    take a lane as soon as one frees up (continuous batching), never waiting
    for a "batch" to fill.
  * admission: a stream is admitted when a cache slot of its resolution is
    free (memory: tok_stream_bytes per slot, preallocated) and its compute
    demand (FLOP/s at its frame rate) fits the compute budget; otherwise it
    waits in arrival order.
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


class Server:
    def __init__(self, executor, n_lanes: int, slots_per_res: dict, budget_flops: float,
                 target_latency: float = 0.033, stall_timeout: float = 0.5,
                 clock: Callable[[], float] | None = None, sleep: Callable[[float], None] | None = None):
        self.ex = executor
        self.n_lanes = n_lanes
        self.free_slots = {res: list(range(n)) for res, n in slots_per_res.items()}
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
        lanes: list = [None] * self.n_lanes      # (state, chunk, ready_t) or None
        used = 0.0
        max_admitted = 0
        admitted_total = 0
        hard = hard_stop if hard_stop is not None else horizon * 3 + 10
        while True:
            t = now()
            # 1. completions
            for li, job in enumerate(lanes):
                if job is None:
                    continue
                st, k, ready = job
                if self.ex.done(li):
                    st.latencies.append(now() - ready)
                    st.in_flight = False
                    st.next_chunk = k + 1
                    lanes[li] = None
                    if st.next_chunk >= st.spec.n_chunks:
                        st.done = True
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
                    used -= st.spec.demand_flops()
                    self.free_slots[(st.spec.H, st.spec.W)].append(st.slot)
                    self.ex.release(st.spec, st.slot)
            # 3. arrivals and admission (arrival order)
            while ai < len(arrivals) and arrivals[ai].start <= t and arrivals[ai].start <= horizon:
                waiting.append(states[arrivals[ai].sid])
                ai += 1
            while waiting:
                st = waiting[0]
                res = (st.spec.H, st.spec.W)
                if not self.free_slots.get(res) or used + st.spec.demand_flops() > self.budget:
                    break
                waiting.pop(0)
                st.slot = self.free_slots[res].pop()
                self.ex.attach(st.spec, st.slot)
                st.admitted_at = t
                used += st.spec.demand_flops()
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
            for li in range(self.n_lanes):
                if lanes[li] is None and ready:
                    _, _, st, k, rt = heapq.heappop(ready)
                    st.in_flight = True
                    lanes[li] = (st, k, rt)
                    self.ex.submit(li, st.spec, st.slot, k)
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

    def _report(self, states, max_admitted, admitted_total, elapsed):
        import statistics as stats
        lat_all = [x for s in states.values() for x in s.latencies]
        by_res = {}
        for s in states.values():
            by_res.setdefault(f"{s.spec.H}x{s.spec.W}", []).extend(s.latencies)

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
                                  "p99_ms": 1e3 * pct(v, 0.99) if v else None} for r, v in by_res.items()},
            "admission_wait_s": {s.spec.sid: (s.admitted_at - s.spec.start) for s in states.values()
                                 if s.admitted_at is not None},
            "admission_wait_p50_s": pct([s.admitted_at - s.spec.start for s in states.values()
                                         if s.admitted_at is not None], 0.5),
        }


class GpuExecutor:
    """Runs chunks through the CUDA library: one tokenizer context + CUDA stream per lane,
    preallocated stream-cache slots per resolution, one content loop per stream."""

    def __init__(self, n_lanes: int, params: dict, slots_per_res: dict, drop_seed: int = 1000,
                 drop_range=(0.0, 0.30), content_frames: int = 9, keep_outputs: bool = False,
                 arch: dict | None = None, content_fn=None):
        import numpy as np
        import torch

        from . import tokenizer as tkz
        self.torch = torch
        self.tkz = tkz
        arch = arch or {}
        self.lanes = []
        for _ in range(n_lanes):
            tk = tkz.Tokenizer("bf16", **arch)
            tk.set_params(params)
            self.lanes.append({"tk": tk, "stream": torch.cuda.Stream(), "event": None, "bufs": {}})
        tk0 = self.lanes[0]["tk"]
        self.levels = tk0.levels
        self.s_t = tk0.s_t
        self.slots = {}
        for (H, W), n in slots_per_res.items():
            for lane in self.lanes:
                lane["tk"].reserve(1, self.s_t, H, W)
            self.slots[(H, W)] = [tk0.stream_open(H, W) for _ in range(n)]
        self.drop_seed = drop_seed
        self.drop_range = drop_range
        self.content_frames = content_frames
        self.content_fn = content_fn
        self.content = {}
        self.keep = keep_outputs
        self.outputs = {}
        self.tokens = {}
        self._np = np

    def _content(self, spec):
        key = spec.sid
        if key not in self.content:
            if self.content_fn is not None:
                clip = self.content_fn(spec)
            else:
                import synthetic as S
                clip = S.moving_rects_clip(100 + spec.sid, self.content_frames, spec.H, spec.W)
            if not isinstance(clip, self.torch.Tensor):
                clip = self.torch.from_numpy(clip)
            self.content[key] = clip.to("cuda", self.torch.bfloat16)
        return self.content[key]

    def attach(self, spec, slot):
        self._content(spec)
        self.torch.cuda.current_stream().synchronize()  # content is on the device before lanes read it
        self.lanes[0]["tk"].stream_reset(self.slots[(spec.H, spec.W)][slot])

    def release(self, spec, slot):
        self.content.pop(spec.sid, None)

    def _bufs(self, lane, H, W):
        key = (H, W)
        if key not in lane["bufs"]:
            torch = self.torch
            Tq, Hq, Wq = lane["tk"].latent_shape(1, H, W)
            lane["bufs"][key] = {
                "idx": torch.empty((1, 1, Hq, Wq), device="cuda", dtype=torch.int32),
                "idx_d": torch.empty((1, 1, Hq, Wq), device="cuda", dtype=torch.int32),
                "kb": torch.empty((1, 1, Hq, (Wq + 31) // 32), device="cuda", dtype=torch.int32),
                "xh": torch.empty((1, self.s_t, H, W, 3), device="cuda", dtype=torch.float32),
            }
        return lane["bufs"][key]

    def chunk_frames(self, spec, k):
        clip = self._content(spec)
        n = clip.shape[0]
        if k == 0:
            ids = [0]
        else:
            ids = [(4 * k - 3 + i) % n for i in range(4)]
        return clip[ids][None].contiguous()

    def submit(self, li, spec, slot, k):
        torch = self.torch
        lane = self.lanes[li]
        tk = lane["tk"]
        vid = self.slots[(spec.H, spec.W)][slot]
        b = self._bufs(lane, spec.H, spec.W)
        rate = float(self._np.random.default_rng([self.drop_seed + spec.sid, k]).uniform(*self.drop_range))
        with torch.cuda.stream(lane["stream"]):
            x = self.chunk_frames(spec, k)
            tk.encode(x, idx=b["idx"], want_z=False, video=vid, stream=lane["stream"])
            self.tkz.drop_mask(b["idx"], rate, seed=self.drop_seed + spec.sid, stream_id=spec.sid, chunk_id=k,
                               levels=self.levels, out=b["idx_d"], keep_bits=b["kb"], stream=lane["stream"])
            T = 1 if k == 0 else self.s_t
            xh = b["xh"][:, :T]
            tk.decode(b["idx_d"], spec.H, spec.W, out=xh if T == self.s_t else b["xh"][:, :1].contiguous(),
                      video=vid, first_chunk=(k == 0), stream=lane["stream"])
            if self.keep:
                out = b["xh"][:, :T].clone()
                self.outputs.setdefault(spec.sid, []).append(out)
                self.tokens.setdefault(spec.sid, []).append(b["idx_d"].clone())
            ev = torch.cuda.Event()
            ev.record(lane["stream"])
        lane["event"] = ev

    def done(self, li):
        ev = self.lanes[li]["event"]
        return ev is None or ev.query()

    def status(self):
        return [lane["tk"].status() for lane in self.lanes]

    def close(self):
        for (H, W), hs in self.slots.items():
            for h in hs:
                self.lanes[0]["tk"].stream_close(h)
        for lane in self.lanes:
            lane["tk"].close()
