"""a9: serving APSP requests with continuous batching on one GPU.

Requests (a cost matrix each, int32 or float32) arrive over time.  The server
* admits them by HBM footprint: every admitted matrix lives in one device arena whose size is
  the admission budget, placed by a first-fit allocator; a request that does not fit waits
  (requests behind a blocked large one may still be admitted if they fit -- small requests
  are not held up by a large head);
* keeps admitted matrices on the device from the host-to-device copy until the closed result
  has been copied back;
* batches continuously: whenever a launch slot frees up, all admitted small requests of one
  dtype (n <= small_max) are closed together by one apsp_batched launch over the arena, and
  a large request is closed alone with the plan the planner picks for it.  Requests that
  arrive while others are on the GPU join the next launch; launches run concurrently on
  several CUDA streams, with copies overlapping the closures;
* records, per request, the time from arrival to its result being back on the host, and
  reports p50/p99 latency and graphs/s.

Results do not depend on the mix: a request's plan depends only on its own size, density and
dtype, and the batched kernel closes each graph exactly as apsp_fw does.

The scheduling policy (Arena, Scheduler) is plain Python and is tested without a GPU.
"""
from __future__ import annotations

import bisect
import collections
import time
from dataclasses import dataclass

import numpy as np

ALIGN = 64  # elements (256 bytes): every arena offset keeps rows 16-byte aligned


class Arena:
    """First-fit allocator over [0, capacity) elements with coalescing free lists."""

    def __init__(self, capacity: int, align: int = ALIGN):
        self.capacity = int(capacity)
        self.align = align
        self.free_list = [(0, self.capacity)]  # sorted (offset, size)
        self.live = {}
        self.used = 0
        self.peak = 0

    def alloc(self, size: int):
        size = -(-int(size) // self.align) * self.align
        if size <= 0:
            size = self.align
        for i, (off, sz) in enumerate(self.free_list):
            if sz >= size:
                if sz == size:
                    self.free_list.pop(i)
                else:
                    self.free_list[i] = (off + size, sz - size)
                self.live[off] = size
                self.used += size
                self.peak = max(self.peak, self.used)
                return off
        return None

    def free(self, off: int):
        size = self.live.pop(off)
        self.used -= size
        i = bisect.bisect_left(self.free_list, (off, 0))
        self.free_list.insert(i, (off, size))
        # coalesce with the right, then the left neighbour
        if i + 1 < len(self.free_list) and off + size == self.free_list[i + 1][0]:
            self.free_list[i] = (off, size + self.free_list[i + 1][1])
            self.free_list.pop(i + 1)
        if i > 0 and self.free_list[i - 1][0] + self.free_list[i - 1][1] == off:
            self.free_list[i - 1] = (self.free_list[i - 1][0], self.free_list[i - 1][1] + self.free_list[i][1])
            self.free_list.pop(i)


@dataclass
class Request:
    rid: int
    n: int
    dtype: str               # "int32" or "float32"
    arrival: float           # seconds after the start of the stream
    host: object = None      # pinned host tensor holding the cost matrix
    density: float = 0.0
    off: int = -1            # arena offset once admitted
    ld: int = 0
    plan: tuple = ("batched", 0)
    t_admit: float = -1.0
    t_done: float = -1.0
    result: object = None
    ready: bool = True       # False until a Feeder has made the host matrix
    host_off: object = None  # the matrix's offset in the Feeder's HostArena

    @property
    def footprint(self) -> int:
        return self.n * self.ld


class Scheduler:
    """Admission and launch grouping, independent of the GPU."""

    def __init__(self, arena: Arena, small_max: int = 1024, max_batch: int = 4096, big_n: int = 2048,
                 big_slots: int = 1):
        self.arena = arena
        self.small_max = small_max
        self.max_batch = max_batch
        self.big_n = big_n          # solo closures this large use the whole GPU ...
        self.big_slots = big_slots  # ... so at most this many run at once (the rest wait in order)
        self.waiting = collections.deque()
        self.ready_small = {"int32": [], "float32": []}
        self.ready_large = collections.deque()

    def arrive(self, r: Request):
        r.ld = -(-r.n // 4) * 4
        self.waiting.append(r)

    def admit(self, now: float) -> list:
        """Admit waiting requests that fit, in arrival order; small ones may pass a large head
        that does not fit.  Returns the newly admitted requests."""
        out = []
        blocked_large = False
        keep = collections.deque()
        while self.waiting:
            r = self.waiting.popleft()
            if blocked_large and r.n > self.small_max:
                keep.append(r)
                continue
            off = self.arena.alloc(r.footprint)
            if off is None:
                keep.append(r)
                if r.n > self.small_max:
                    blocked_large = True
                continue
            r.off, r.t_admit = off, now
            out.append(r)
            if r.n <= self.small_max:
                self.ready_small[r.dtype].append(r)
            else:
                self.ready_large.append(r)
        self.waiting = keep
        return out

    def next_launch(self, big_inflight: int = 0):
        """The next unit of work: ("batch", dtype, [requests]) or ("solo", request), or None.
        Large requests go first (they take longest), in arrival order, except that a very large
        one (n >= big_n) waits while big_slots of them are already running -- two such closures
        sharing the GPU would both finish late -- and smaller work flows around it.  Small
        requests are gathered per dtype."""
        for idx, r in enumerate(self.ready_large):
            if r.n >= self.big_n and big_inflight >= self.big_slots:
                continue
            del self.ready_large[idx]
            return ("solo", r)
        best = max(self.ready_small, key=lambda k: len(self.ready_small[k]))
        if self.ready_small[best]:
            group = self.ready_small[best][: self.max_batch]
            self.ready_small[best] = self.ready_small[best][self.max_batch:]
            return ("batch", best, group)
        return None

    def release(self, r: Request):
        self.arena.free(r.off)
        r.off = -1


class HostArena:
    """A page-locked host buffer (huge pages when large, so that copies keep their full rate)
    carved by the first-fit Arena: the host side of requests whose matrices are made while the
    stream runs.  view(off, n, dtype) is an n x n tensor at element offset off."""

    def __init__(self, nbytes: int):
        from . import host_empty
        import torch
        self.buf = host_empty((nbytes // 4,), torch.int32)
        self.arena = Arena(nbytes // 4)

    def view(self, off: int, n: int, dtype: str):
        import torch
        t = self.buf[off:off + n * n].view(n, n)
        return t.view(torch.float32) if dtype == "float32" else t


class Feeder:
    """Makes the request matrices of a stream ahead of their arrival, on a pool of host threads,
    into a HostArena: request i is made once its arrival is within `lead` seconds (all at once
    with lead = None) and its matrix fits the arena; the server releases its slice when done.
    ``make(k, n, p, dtype, out)`` writes request k's matrix into the numpy array ``out``.
    ``stats()`` reports how late, if ever, a matrix became ready after its arrival time."""

    def __init__(self, requests: list, arena: HostArena, make, threads: int = 8, lead: float | None = 1.0,
                 time_scale: float = 1.0):
        import threading
        from concurrent.futures import ThreadPoolExecutor
        self.reqs = sorted(requests, key=lambda r: r.arrival)
        self.arena, self.make, self.lead, self.ts = arena, make, lead, time_scale
        self.cv = threading.Condition()
        self.pool = ThreadPoolExecutor(threads)
        self.t0 = None
        self.late = []
        self.stop = False
        self.thread = threading.Thread(target=self._run, daemon=True)

    def start(self, t0: float):
        self.t0 = t0
        self.thread.start()

    def _run(self):
        for r in self.reqs:
            if self.lead is not None:
                while not self.stop:
                    wait = r.arrival * self.ts - self.lead - (time.perf_counter() - self.t0)
                    if wait <= 0:
                        break
                    time.sleep(min(wait, 0.01))
            with self.cv:
                while not self.stop:
                    r.host_off = self.arena.arena.alloc(r.n * r.n)
                    if r.host_off is not None:
                        break
                    self.cv.wait(0.01)
            if self.stop:
                return
            self.pool.submit(self._fill, r)

    def _fill(self, r):
        v = self.arena.view(r.host_off, r.n, r.dtype)
        self.make(r.rid, r.n, r.density, r.dtype, v.numpy())
        r.host = v
        late = (time.perf_counter() - self.t0) - r.arrival * self.ts
        with self.cv:
            self.late.append(late)
            r.ready = True
            self.cv.notify_all()

    def release(self, r):
        with self.cv:
            self.arena.arena.free(r.host_off)
            r.host, r.host_off = None, None
            self.cv.notify_all()

    def close(self):
        self.stop = True
        self.thread.join(timeout=5)
        self.pool.shutdown(wait=True)

    def stats(self) -> dict:
        late = np.maximum(np.asarray(self.late, np.float64), 0.0) * 1e3
        return {"matrices": len(late), "ready_after_arrival_ms_p99": float(np.percentile(late, 99)) if len(late) else None,
                "ready_after_arrival_ms_max": float(late.max()) if len(late) else None}


def stream_requests(arrivals, ns, ps, dtypes):
    """Requests of a stream whose matrices a Feeder makes: request k has n = ns[k], edge
    probability ps[k] (its density feature) and dtype dtypes[k]; not ready until made."""
    return [Request(rid=k, n=int(ns[k]), dtype=str(dtypes[k]), arrival=float(t), density=float(ps[k]), ready=False)
            for k, t in enumerate(arrivals)]


def make_requests(arrivals, library, density=None):
    """Requests for arrival times `arrivals` (seconds): request k carries library graph
    k mod len(library) (a list of numpy cost matrices), copied once to pinned host memory."""
    import torch
    pinned = [torch.from_numpy(m).pin_memory() for m in library]
    dens = density or [0.0] * len(library)
    out = []
    for k, t in enumerate(arrivals):
        g = k % len(library)
        m = library[g]
        out.append(Request(rid=k, n=m.shape[0], dtype="float32" if m.dtype == np.float32 else "int32",
                           arrival=float(t), host=pinned[g], density=dens[g]))
    return out


def percentiles(lat_ms):
    a = np.sort(np.asarray(lat_ms, dtype=np.float64))
    if a.size == 0:
        return {"p50": None, "p99": None}
    return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "mean": float(a.mean()),
            "max": float(a.max())}


class Server:
    """Continuous-batching APSP server on one GPU (see the module docstring)."""

    def __init__(self, device=None, arena_bytes: int = 8 << 30, small_max: int = 1024, slots: int = 4,
                 planner=None, keep_results: bool = False, big_slots: int = 1):
        """big_slots: how many closures of at least 2048 vertices may share the GPU (1 keeps
        their latency low; 2 lets one's latency-bound block steps overlap the other's work,
        for throughput)."""
        import torch
        self.torch = torch
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.arena_elems = arena_bytes // 4
        self.pool = torch.empty(self.arena_elems, dtype=torch.int32, device=self.dev)
        self.sched = Scheduler(Arena(self.arena_elems), small_max=small_max, big_slots=big_slots)
        self.slots = slots
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(slots)]
        self.copy_in = torch.cuda.Stream(self.dev)
        self.planner = planner
        self.keep_results = keep_results
        self.ws = [torch.empty(256, dtype=torch.uint8, device=self.dev) for _ in range(slots)]
        self._staging = {}

    # -- helpers ---------------------------------------------------------------------------
    def _view(self, r: Request):
        t = self.pool[r.off:r.off + r.n * r.ld].view(r.n, r.ld)[:, :r.n]
        return t.view(self.torch.float32) if r.dtype == "float32" else t

    def _plan(self, r: Request):
        if r.n <= self.sched.small_max:
            return ("batched", 0)
        if self.planner is not None:
            return self.planner.choose(r.n, r.density, r.dtype)
        return ("fw", 0)

    def _result_buffer(self, r: Request):
        torch = self.torch
        dt = torch.float32 if r.dtype == "float32" else torch.int32
        if self.keep_results:
            return torch.empty((r.n, r.n), dtype=dt).pin_memory()
        if r.host_off is not None:
            return r.host  # a Feeder's request: back into its own host slice
        key = (r.n, r.dtype)
        if key not in self._staging:
            self._staging[key] = torch.empty((r.n, r.n), dtype=dt).pin_memory()
        return self._staging[key]

    def _launch(self, work, stream, slot):
        from . import apsp_batched_raw, apsp_batched_staged_workspace_bytes, apsp_fw, apsp_rkleene
        torch = self.torch
        with torch.cuda.stream(stream):
            stream.wait_stream(self.copy_in)
            if work[0] == "batch":
                group = work[2]
                offs = np.array([r.off for r in group], np.int64)
                ns = np.array([r.n for r in group], np.int32)
                lds = np.array([r.ld for r in group], np.int32)
                # room for the staged path (int32 graphs of 257..2048 vertices closed in lockstep
                # on the GEMM engine); grown per slot, allocated on the slot's own stream
                need = apsp_batched_staged_workspace_bytes(ns, torch.int32 if work[1] == "int32" else torch.float32)
                if self.ws[slot].numel() < need:
                    self.ws[slot] = torch.empty(need + need // 4, dtype=torch.uint8, device=self.dev)
                ws = self.ws[slot]
                order = np.argsort(-ns, kind="stable").astype(np.int32)
                meta = torch.from_numpy(np.concatenate([offs.view(np.int32), ns, lds, order])).pin_memory()
                dmeta = meta.to(self.dev, non_blocking=True)
                k = len(group)
                d_off = dmeta[:2 * k].view(torch.int64)
                apsp_batched_raw(self.pool if work[1] == "int32" else self.pool.view(torch.float32), d_off,
                                 dmeta[2 * k:3 * k], dmeta[3 * k:4 * k], dmeta[4 * k:5 * k], k, ws, ns_host=ns)
                reqs = group
                keep = (meta, dmeta)
            else:
                r = work[1]
                algo, param = r.plan
                v = self._view(r)
                if algo == "rkleene":
                    apsp_rkleene(v, cutoff=param)
                elif algo == "cta":
                    from . import apsp_close_cta
                    apsp_close_cta(v)
                elif algo == "squaring":
                    from . import apsp_squaring
                    apsp_squaring(v)
                else:
                    apsp_fw(v)
                reqs = [r]
                keep = None
            for r in reqs:
                r.result = self._result_buffer(r)
                r.result.copy_(self._view(r), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        return ev, reqs, keep

    # -- the loop ----------------------------------------------------------------------------
    def serve(self, requests: list, time_scale: float = 1.0, feeder: Feeder | None = None) -> dict:
        """Serve requests at their arrival times (arrival * time_scale seconds after start).  With
        a feeder, a request enters once its matrix is made, and its host slice is released (the
        result then goes back into it unless keep_results) when it is done."""
        torch = self.torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            r.plan = self._plan(r)
            if r.n * (-(-r.n // 4) * 4) > self.sched.arena.capacity:
                raise ValueError(f"request {r.rid} (n={r.n}) can never fit the {self.arena_elems * 4} B arena")
        total = len(reqs)
        t0 = time.perf_counter()
        if feeder is not None:
            feeder.start(t0)
        nxt, done = 0, 0
        inflight = []  # (event, reqs, keepalive, slot)
        free_slots = list(range(self.slots))
        big = self.sched.big_n
        launches = {"batch": 0, "solo": 0}
        while done < total:
            now = time.perf_counter() - t0
            while nxt < total and reqs[nxt].arrival * time_scale <= now and reqs[nxt].ready:
                self.sched.arrive(reqs[nxt])
                nxt += 1
            for r in self.sched.admit(now):
                with torch.cuda.stream(self.copy_in):
                    self._view(r).copy_(r.host, non_blocking=True)
            progressed = False
            while free_slots:
                big_inflight = sum(1 for _, rs, _, _ in inflight if len(rs) == 1 and rs[0].n >= big
                                   and rs[0].plan[0] != "batched")
                work = self.sched.next_launch(big_inflight)
                if work is None:
                    break
                slot = free_slots.pop()
                ev, rs, keep = self._launch(work, self.streams[slot], slot)
                inflight.append((ev, rs, keep, slot))
                launches[work[0]] += 1
                progressed = True
            still = []
            for ev, rs, keep, slot in inflight:
                if ev.query():
                    t = time.perf_counter() - t0
                    for r in rs:
                        r.t_done = t
                        self.sched.release(r)
                        if feeder is not None and not self.keep_results:
                            feeder.release(r)
                        done += 1
                    free_slots.append(slot)
                    progressed = True
                else:
                    still.append((ev, rs, keep, slot))
            inflight = still
            if not progressed:
                time.sleep(50e-6)
        wall = time.perf_counter() - t0
        if feeder is not None:
            feeder.close()
        lat = [(r.t_done - r.arrival * time_scale) * 1e3 for r in reqs]
        st = percentiles(lat)
        st.update({"requests": total, "wall_s": wall, "graphs_per_s": total / wall, "launches": launches,
                   "arena_peak_bytes": self.sched.arena.peak * 4, "arena_bytes": self.arena_elems * 4})
        return st


def serve_one_at_a_time(requests: list, device=None, time_scale: float = 1.0, planner=None,
                        feeder: Feeder | None = None) -> dict:
    """Baseline: each request in arrival order is copied in, closed alone (apsp_fw) and copied
    back before the next one starts (with a feeder: back into its own host slice)."""
    import torch
    from . import apsp_fw
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    reqs = sorted(requests, key=lambda r: r.arrival)
    staging = {}
    t0 = time.perf_counter()
    if feeder is not None:
        feeder.start(t0)
    for r in reqs:
        while time.perf_counter() - t0 < r.arrival * time_scale or not r.ready:
            time.sleep(50e-6)
        d = r.host.to(dev, non_blocking=True)
        apsp_fw(d)
        if r.host_off is not None:  # a Feeder's request: back into its own host slice
            dst = r.host
        else:
            key = (r.n, r.dtype)
            if key not in staging:
                staging[key] = torch.empty_like(r.host).pin_memory()
            dst = staging[key]
        dst.copy_(d, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        r.t_done = time.perf_counter() - t0
        if feeder is not None:
            feeder.release(r)
    wall = time.perf_counter() - t0
    if feeder is not None:
        feeder.close()
    st = percentiles([(r.t_done - r.arrival * time_scale) * 1e3 for r in reqs])
    st.update({"requests": len(reqs), "wall_s": wall, "graphs_per_s": len(reqs) / wall})
    return st
