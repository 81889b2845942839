"""Continuous-batching serving loop for alm2map / map2alm requests.

Requests of mixed resolution, spin and map count arrive at any time. The
server keeps plans (ring, recurrence and FFT tables) resident, groups the
pending requests that share a plan key and an operation into one batch (the
map columns are the GEMM's N side, so a batch fills the tensor-core tiles that
single requests leave empty), admits a batch only while the device memory it
needs (workspace, staging and output buffers), on top of what the executor
keeps resident (plans, captured graphs) and the batches already running, fits
the HBM budget and a stream slot is free, runs it asynchronously, and hands
every request its own slice of the batch output. Batches that arrive while others run are admitted as slots and
memory free up (continuous batching); the results of a request do not depend
on what it was batched with (map columns are independent in every kernel).

Optional CUDA graphs: a batch shape (plan key, operation, batch bucket) is
captured once with static buffers and replayed afterwards; batches are padded
with zero maps up to their bucket.

The scheduling logic is independent of the GPU: `Server` drives an executor
object (`GpuExecutor` on a device; tests use a CPU fake) through four calls:
`prepare(key)`, `batch_bytes(key, n)`, `launch(key, inputs) -> handle` and
`poll(handle) -> outputs or None`, plus optionally `resident_bytes()`.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field


@dataclass(eq=False)          # compared by identity (the payloads are arrays)
class Request:
    op: str                      # "alm2map" or "map2alm"
    nside: int
    spin: int
    data: object                 # alm [n, ncomp, nalm] complex128 / maps [n, ncomp, npix] float64,
                                 # or a list of such arrays (concatenated along the first axis)
    nmaps: int = 0
    lmax: int = -1               # default 2 nside - 1
    t_arrival: float = 0.0
    t_start: float | None = None
    t_done: float | None = None
    result: object = None
    error: str | None = None
    done: threading.Event = field(default_factory=threading.Event)

    def key(self, precision):
        lmax = self.lmax if self.lmax >= 0 else 2 * self.nside - 1
        return (self.op, self.nside, lmax, self.spin, precision)


@dataclass(eq=False)
class _Batch:
    key: tuple
    reqs: list
    nbytes: int
    handle: object
    t_launch: float


class Server:
    """Continuous-batching scheduler over an executor (see module docstring)."""

    def __init__(self, executor, hbm_budget: float = 150e9, max_batch_maps: int = 256, slots: int = 4,
                 precision_for=None, on_complete=None):
        self.ex = executor
        self.budget = float(hbm_budget)
        self.max_batch = int(max_batch_maps)
        self.slots = int(slots)
        self.precision_for = precision_for or (lambda req: "auto")
        self.on_complete = on_complete               # called with each finished request
        self.pending = collections.OrderedDict()     # key -> deque of requests (FIFO per key)
        self.inflight: list[_Batch] = []
        self.used = 0.0
        self.lock = threading.Condition()
        self.completed: list[Request] = []
        self.nbatches = 0
        self.peak_used = 0.0
        self._stop = False
        self._thread = None

    # ---------------------------------------------------------------- intake
    def submit(self, req: Request) -> Request:
        if req.op not in ("alm2map", "map2alm"):
            raise ValueError(f"unknown operation {req.op}")
        if not req.nmaps:
            parts = req.data if isinstance(req.data, (list, tuple)) else [req.data]
            req.nmaps = int(sum(int(x.shape[0]) for x in parts))
        if not req.t_arrival:
            req.t_arrival = time.perf_counter()
        key = req.key(self.precision_for(req))
        with self.lock:
            self.pending.setdefault(key, collections.deque()).append(req)
            self.lock.notify_all()
        return req

    # ------------------------------------------------------------- scheduling
    def _oldest_key(self, skip):
        best, t = None, None
        for k, q in self.pending.items():
            if q and k not in skip and (t is None or q[0].t_arrival < t):
                best, t = k, q[0].t_arrival
        return best

    def step(self) -> bool:
        """One scheduling round: retire finished batches, admit new ones.
        Returns True if anything happened."""
        progressed = False
        # retire
        for b in list(self.inflight):
            outs = self.ex.poll(b.handle)
            if outs is None:
                continue
            now = time.perf_counter()
            for r, o in zip(b.reqs, outs):
                r.result, r.t_done = o, now
                self._finish(r)
            self.inflight.remove(b)
            self.used -= b.nbytes
            progressed = True
        # admit, oldest request first; a key whose batch does not fit is
        # skipped for this round so that smaller work can still start
        skip = set()
        while len(self.inflight) < self.slots:
            with self.lock:
                key = self._oldest_key(skip)
                if key is None:
                    break
                q = self.pending[key]
            self.ex.prepare(key)
            room = self.budget - self._resident()
            with self.lock:
                # grow the batch while it stays within max_batch maps and
                # within the memory left beside the resident plans
                reqs, n = [], 0
                while q and (not reqs or (n + q[0].nmaps <= self.max_batch
                                          and self.ex.batch_bytes(key, n + q[0].nmaps) <= room)):
                    reqs.append(q.popleft())
                    n += reqs[-1].nmaps
            nbytes = self.ex.batch_bytes(key, n)
            # (a batch larger than the whole budget still runs, alone)
            if self.used + self._resident() + nbytes > self.budget and self.inflight:
                with self.lock:                       # put back, in order
                    for r in reversed(reqs):
                        q.appendleft(r)
                skip.add(key)
                continue
            now = time.perf_counter()
            for r in reqs:
                r.t_start = now
            try:
                handle = self.ex.launch(key, [r.data for r in reqs])
            except Exception as e:                    # a failed batch fails its requests, not the server
                msg = f"{type(e).__name__}: {e}"
                for r in reqs:
                    r.error, r.t_done = msg, time.perf_counter()
                    self._finish(r)
                progressed = True
                continue
            # a graph captured by this launch is resident from now on (and in
            # _resident()): the batch itself keeps only what batch_bytes now says
            nbytes = min(nbytes, self.ex.batch_bytes(key, n))
            self.inflight.append(_Batch(key, reqs, nbytes, handle, now))
            self.used += nbytes
            self.peak_used = max(self.peak_used, self.used + self._resident())
            self.nbatches += 1
            progressed = True
        return progressed

    def _resident(self) -> float:
        f = getattr(self.ex, "resident_bytes", None)
        return float(f()) if f else 0.0

    def _finish(self, r):
        r.done.set()
        self.completed.append(r)
        if self.on_complete is not None:
            self.on_complete(r)

    def idle(self) -> bool:
        with self.lock:
            return not self.inflight and not any(self.pending.values())

    def run_until_idle(self, poll_s: float = 1e-4):
        while not self.idle():
            if not self.step():
                time.sleep(poll_s)

    # ------------------------------------------------------- background mode
    def start(self, poll_s: float = 1e-4):
        def loop():
            while not self._stop:
                if not self.step():
                    with self.lock:
                        self.lock.wait(timeout=poll_s)
        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()

    def stop(self):
        self._stop = True
        with self.lock:
            self.lock.notify_all()
        if self._thread is not None:
            self._thread.join()

    # ---------------------------------------------------------------- report
    def stats(self) -> dict:
        lat = sorted((r.t_done - r.t_arrival) for r in self.completed if r.t_done is not None and not r.error)
        maps = sum(r.nmaps for r in self.completed if not r.error)
        errs = [r.error for r in self.completed if r.error]
        if not lat:
            return {"requests": 0, "errors": len(errs), "first_error": errs[0] if errs else None}
        t0 = min(r.t_arrival for r in self.completed)
        t1 = max(r.t_done for r in self.completed)

        def pct(p):
            return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]
        return {"requests": len(lat), "maps": maps, "batches": self.nbatches,
                "p50_ms": 1e3 * pct(50), "p99_ms": 1e3 * pct(99), "maps_per_s": maps / max(t1 - t0, 1e-9),
                "peak_admitted_bytes": self.peak_used,
                "errors": len(errs), "first_error": errs[0] if errs else None}


class GpuExecutor:
    """Runs batches on one GPU with libsht: resident plans (LRU), one CUDA
    stream per slot, optional CUDA-graph replay per (key, batch bucket).

    Memory. A batch of n maps (without a graph) is run as consecutive library calls of at most
    `chunk` maps on its stream, with one workspace sized for the chunk, so
    that workspace + input staging + the batch output stay within `mem_cap`
    (the server's HBM budget). Each request's result is a view of the batch
    output (no copies). Graphs are kept only for batch buckets whose static
    buffers (input, output, workspace) are at most `graph_max_bytes`, up to
    `graph_cache_bytes` in all (LRU); a captured graph serves one batch at a
    time (a batch that finds its graph busy runs without it). Plans and graph
    buffers are reported by `resident_bytes()` for admission; a batch that
    will capture a graph also counts the capture's buffers. Batches below
    `small_work` map values run on high-priority streams (`small_slots` of
    them)."""

    def __init__(self, device: int = 0, slots: int = 4, use_graphs: bool = False, plan_cache: int = 32,
                 mem_cap: float = 150e9, graph_max_bytes: float = 0.5e9, graph_cache_bytes: float = 24e9,
                 small_work: float = 2e9, small_slots: int = 2):
        import torch
        from . import sht
        self.torch, self.sht = torch, sht
        self.device = device
        # batches of less than `small_work` (map pixels x components x maps)
        # run on high-priority streams: the GPU schedules their CTAs ahead of
        # those of large batches already running, so small requests do not
        # wait behind a batch that takes seconds
        self.small_work = float(small_work)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        hi = torch.cuda.Stream.priority_range()[1] if hasattr(torch.cuda.Stream, "priority_range") else -1
        self.streams_hi = [torch.cuda.Stream(device=device, priority=hi) for _ in range(small_slots)]
        self.free_streams = list(range(slots))
        self.free_hi = list(range(small_slots))
        self.plans = collections.OrderedDict()
        self.plan_cache = plan_cache
        self.use_graphs = use_graphs
        self.mem_cap = float(mem_cap)
        self.graph_max_bytes = float(graph_max_bytes)
        self.graph_cache_bytes = float(graph_cache_bytes)
        self.graphs = collections.OrderedDict()      # (key, bucket) -> (graph, xin, yout, ws, bytes)
        self.graph_busy = set()
        self.graph_replays = 0

    # ------------------------------------------------------------- plans
    def _precision(self, key):
        op, nside, lmax, spin, prec = key
        if prec != "auto":
            return prec
        # the split form's limits (libsht returns SHT_EUNSUPPORTED beyond them)
        ok = lmax <= 2047 and nside <= (4096 if spin == 0 else 2048)
        return "split" if ok else "fp64"

    def prepare(self, key):
        pk = key[1:4] + (self._precision(key),)
        if pk not in self.plans:
            self.plans[pk] = self.sht.Plan(pk[0], pk[1], None, pk[2], pk[3], device=self.device)
            while len(self.plans) > self.plan_cache:
                old, _ = self.plans.popitem(last=False)
                for gk in [g for g in self.graphs if g[0][1:4] == old[:3] and g not in self.graph_busy]:
                    del self.graphs[gk]
        self.plans.move_to_end(pk)
        return self.plans[pk]

    _plan = prepare

    def resident_bytes(self) -> float:
        return float(sum(p.device_bytes() for p in self.plans.values())
                     + sum(v[4] for v in self.graphs.values()))

    # ------------------------------------------------------------ memory
    @staticmethod
    def _sizes(p, op):
        """(input, output) bytes per map of one operation."""
        alm_b, map_b = p.ncomp * p.nalm * 16, p.ncomp * p.npix * 8
        return (alm_b, map_b) if op == "alm2map" else (map_b, alm_b)

    def _chunk(self, p, op, n):
        """Maps per library call: all n if they fit the memory cap (less what
        the executor keeps resident), else the largest halving of n that does
        (at least 1)."""
        ib, ob = self._sizes(p, op)
        cap = self.mem_cap - self.resident_bytes()
        c = n
        while c > 1 and p.workspace_bytes(c) + c * ib + n * ob > cap:
            c = (c + 1) // 2
        return c

    def batch_bytes(self, key, n):
        p = self._plan(key)
        ib, ob = self._sizes(p, key[0])
        g = self._graph_bytes(key, p, n)
        if g:                                          # the output is copied out of the graph's buffers,
            cached = (key, self._bucket(n)) in self.graphs   # which are resident once captured
            return n * ob + (0 if cached else g)
        c = self._chunk(p, key[0], n)
        return p.workspace_bytes(c) + c * ib + n * ob

    def _graph_bytes(self, key, p, n):
        """Static bytes of the graph a batch of n maps would replay, or 0 if
        it would run without one."""
        if not self.use_graphs:
            return 0
        b = self._bucket(n)
        ib, ob = self._sizes(p, key[0])
        nbytes = p.workspace_bytes(b) + b * (ib + ob)
        return nbytes if nbytes <= self.graph_max_bytes else 0

    @staticmethod
    def _bucket(n):
        b = 1
        while b < n:
            b *= 2
        return b

    # ------------------------------------------------------------ launch
    def launch(self, key, inputs):
        torch = self.torch
        p = self._plan(key)
        op = key[0]
        dev = f"cuda:{self.device}"
        counts, pieces = [], []
        for x in inputs:
            parts = list(x) if isinstance(x, (list, tuple)) else [x]
            counts.append(sum(int(t.shape[0]) for t in parts))
            pieces.extend(parts)
        n = sum(counts)
        if n * p.ncomp * p.npix < self.small_work and self.free_hi:
            sid = ("hi", self.free_hi.pop())
            st = self.streams_hi[sid[1]]
        elif self.free_streams:
            sid = ("lo", self.free_streams.pop())
            st = self.streams[sid[1]]
        else:                                          # every slot busy: queue on stream 0 (not freed again)
            sid = ("shared", 0)
            st = self.streams[0]
        ib, ob = self._sizes(p, op)
        out_len = p.npix if op == "alm2map" else p.nalm
        out_dt = torch.float64 if op == "alm2map" else torch.complex128
        gk = None
        with torch.cuda.stream(st):
            pieces = [t.to(dev, non_blocking=True) for t in pieces]
            if self.use_graphs:
                gk = self._graph_for(key, p, op, n, st)
            if gk is not None:
                out = self._replay(gk, pieces, n, out_len, out_dt)
            else:
                out = torch.empty((n, p.ncomp, out_len), dtype=out_dt, device=dev)
                c = self._chunk(p, op, n)
                ws = torch.empty(p.workspace_bytes(c) + 256, dtype=torch.uint8, device=dev)
                ws = ws[(-ws.data_ptr()) % 256:]
                stage = None
                for c0 in range(0, n, c):
                    c1 = min(n, c0 + c)
                    x = self._rows(pieces, c0, c1)
                    if x is None:                      # rows span several pieces: gather
                        if stage is None:
                            in_len = p.nalm if op == "alm2map" else p.npix
                            in_dt = torch.complex128 if op == "alm2map" else torch.float64
                            stage = torch.empty((c, p.ncomp, in_len), dtype=in_dt, device=dev)
                        x = stage[:c1 - c0]
                        self._gather(pieces, c0, c1, x)
                    if op == "alm2map":
                        p.alm2map(x, out=out[c0:c1], workspace=ws)
                    else:
                        p.map2alm(x, out=out[c0:c1], workspace=ws)
            outs, o = [], 0
            for cnt in counts:
                outs.append(out[o:o + cnt])
                o += cnt
            ev = torch.cuda.Event()
            ev.record(st)
        # buffers allocated on st are only reused by later work on st: stream order keeps them valid
        return (ev, outs, sid, gk)

    @staticmethod
    def _rows(pieces, c0, c1):
        """Rows c0..c1 of the concatenated pieces as one contiguous view, or None."""
        o = 0
        for t in pieces:
            k = int(t.shape[0])
            if o <= c0 and c1 <= o + k:
                v = t[c0 - o:c1 - o]
                return v if v.is_contiguous() else None
            o += k
        return None

    @staticmethod
    def _gather(pieces, c0, c1, dst):
        o = 0
        for t in pieces:
            k = int(t.shape[0])
            a, b = max(c0, o), min(c1, o + k)
            if a < b:
                dst[a - c0:b - c0].copy_(t[a - o:b - o])
            o += k

    # ------------------------------------------------------------ graphs
    def _graph_for(self, key, p, op, n, st):
        """The (key, bucket) graph to replay for n maps, captured on first
        use; None if its buffers exceed the limits or it is busy."""
        torch = self.torch
        b = self._bucket(n)
        gk = (key, b)
        if gk in self.graph_busy:
            return None
        ib, ob = self._sizes(p, op)
        nbytes = p.workspace_bytes(b) + b * (ib + ob)
        if nbytes > self.graph_max_bytes:
            return None
        if gk not in self.graphs:
            while self.graphs and sum(v[4] for v in self.graphs.values()) + nbytes > self.graph_cache_bytes:
                old = next((g for g in self.graphs if g not in self.graph_busy), None)
                if old is None:
                    return None
                del self.graphs[old]
            dev = f"cuda:{self.device}"
            shape_in = (b, p.ncomp, p.nalm if op == "alm2map" else p.npix)
            dt_in = torch.complex128 if op == "alm2map" else torch.float64
            xin = torch.zeros(shape_in, dtype=dt_in, device=dev)
            yout = torch.empty((b, p.ncomp, p.npix if op == "alm2map" else p.nalm),
                               dtype=torch.float64 if op == "alm2map" else torch.complex128, device=dev)
            ws = torch.empty(p.workspace_bytes(b) + 256, dtype=torch.uint8, device=dev)
            ws = ws[(-ws.data_ptr()) % 256:]
            if op == "alm2map":
                def run():
                    p.alm2map(xin, out=yout, workspace=ws)
            else:
                def run():
                    p.map2alm(xin, out=yout, workspace=ws)
            run()                                      # warm-up outside the capture (sets kernel attributes)
            st.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st, capture_error_mode="thread_local"):
                run()
            self.graphs[gk] = (g, xin, yout, ws, nbytes)
        self.graphs.move_to_end(gk)
        self.graph_busy.add(gk)
        return gk

    def _replay(self, gk, pieces, n, out_len, out_dt):
        torch = self.torch
        g, xin, yout, ws, _ = self.graphs[gk]
        self._gather(pieces, 0, n, xin[:n])
        if n < xin.shape[0]:
            xin[n:].zero_()
        g.replay()
        self.graph_replays += 1
        # the graph's output buffer is reused by its next replay: copy out
        return yout[:n].clone()

    def poll(self, handle):
        ev, outs, sid, gk = handle
        if not ev.query():
            return None
        if sid[0] == "hi":
            self.free_hi.append(sid[1])
        elif sid[0] == "lo":
            self.free_streams.append(sid[1])
        if gk is not None:
            self.graph_busy.discard(gk)
        return outs
