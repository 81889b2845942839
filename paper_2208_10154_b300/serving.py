"""Continuous-batching serving loop for alm2map / map2alm requests.

Requests of mixed resolution, spin and map count arrive at any time. The
server keeps plans (ring, recurrence and FFT tables) resident, groups the
pending requests that share a plan key and an operation into one batch (the
map columns are the GEMM's N side, so a batch fills the tensor-core tiles that
single requests leave empty), admits a batch only while the device memory it
needs (workspace + batch buffers) fits the HBM budget and a stream slot is
free, runs it asynchronously, and hands every request its own slice of the
batch output. Batches that arrive while others run are admitted as slots and
memory free up (continuous batching); the results of a request do not depend
on what it was batched with (map columns are independent in every kernel).

Optional CUDA graphs: a batch shape (plan key, operation, batch bucket) is
captured once with static buffers and replayed afterwards; batches are padded
with zero maps up to their bucket.

The scheduling logic is independent of the GPU: `Server` drives an executor
object (`GpuExecutor` on a device; tests use a CPU fake) through four calls:
`prepare(key)`, `batch_bytes(key, n)`, `launch(key, inputs) -> handle` and
`poll(handle) -> outputs or None`.
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
    data: object                 # alm [n, ncomp, nalm] complex128 / maps [n, ncomp, npix] float64
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
                 precision_for=None):
        self.ex = executor
        self.budget = float(hbm_budget)
        self.max_batch = int(max_batch_maps)
        self.slots = int(slots)
        self.precision_for = precision_for or (lambda req: "auto")
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
            req.nmaps = int(req.data.shape[0])
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
                r.done.set()
                self.completed.append(r)
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
                reqs, n = [], 0
                while q and (not reqs or n + q[0].nmaps <= self.max_batch):
                    reqs.append(q.popleft())
                    n += reqs[-1].nmaps
            self.ex.prepare(key)
            nbytes = self.ex.batch_bytes(key, n)
            # (a batch larger than the whole budget still runs, alone)
            if self.used + nbytes > self.budget and self.inflight:
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
                for r in reqs:
                    r.error, r.t_done = str(e), time.perf_counter()
                    r.done.set()
                    self.completed.append(r)
                progressed = True
                continue
            self.inflight.append(_Batch(key, reqs, nbytes, handle, now))
            self.used += nbytes
            self.peak_used = max(self.peak_used, self.used)
            self.nbatches += 1
            progressed = True
        return progressed

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
        if not lat:
            return {"requests": 0}
        t0 = min(r.t_arrival for r in self.completed)
        t1 = max(r.t_done for r in self.completed)

        def pct(p):
            return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]
        return {"requests": len(lat), "maps": maps, "batches": self.nbatches,
                "p50_ms": 1e3 * pct(50), "p99_ms": 1e3 * pct(99), "maps_per_s": maps / max(t1 - t0, 1e-9),
                "peak_admitted_bytes": self.peak_used,
                "errors": sum(1 for r in self.completed if r.error)}


class GpuExecutor:
    """Runs batches on one GPU with libsht: resident plans, one CUDA stream per
    slot, optional CUDA-graph replay per (key, bucket)."""

    def __init__(self, device: int = 0, slots: int = 4, use_graphs: bool = False, plan_cache: int = 32):
        import torch
        from . import sht
        self.torch, self.sht = torch, sht
        self.device = device
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.free_streams = list(range(slots))
        self.plans = collections.OrderedDict()
        self.plan_cache = plan_cache
        self.use_graphs = use_graphs
        self.graphs = {}

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
                self.plans.popitem(last=False)
        self.plans.move_to_end(pk)
        return self.plans[pk]

    def _plan(self, key):
        return self.prepare(key)

    def batch_bytes(self, key, n):
        p = self._plan(key)
        io = n * p.ncomp * (p.npix * 8 + p.nalm * 16)
        return p.workspace_bytes(n) + io

    @staticmethod
    def _bucket(n):
        b = 1
        while b < n:
            b *= 2
        return b

    def launch(self, key, inputs):
        torch = self.torch
        p = self._plan(key)
        op = key[0]
        sid = self.free_streams.pop() if self.free_streams else 0
        st = self.streams[sid]
        counts = [int(x.shape[0]) for x in inputs]
        n = sum(counts)
        with torch.cuda.stream(st):
            xs = [x.to(f"cuda:{self.device}", non_blocking=True) for x in inputs]
            if self.use_graphs:
                out = self._replay(key, p, op, xs, n, st)
            else:
                x = xs[0] if len(xs) == 1 else torch.cat(xs, dim=0)
                ws = torch.empty(p.workspace_bytes(n) + 256, dtype=torch.uint8, device=x.device)
                ws = ws[(-ws.data_ptr()) % 256:]
                out = p.alm2map(x, workspace=ws) if op == "alm2map" else p.map2alm(x, workspace=ws)
            outs, o = [], 0
            for c in counts:
                outs.append(out[o:o + c].clone())
                o += c
            ev = torch.cuda.Event()
            ev.record(st)
        # buffers allocated on st are only reused by later work on st: stream order keeps them valid
        return (ev, outs, sid)

    def _replay(self, key, p, op, xs, n, st):
        torch = self.torch
        b = self._bucket(n)
        gk = (key, b)
        if gk not in self.graphs:
            shape_in = (b, p.ncomp, p.nalm if op == "alm2map" else p.npix)
            dt_in = torch.complex128 if op == "alm2map" else torch.float64
            xin = torch.zeros(shape_in, dtype=dt_in, device=f"cuda:{self.device}")
            ws = torch.empty(p.workspace_bytes(b) + 256, dtype=torch.uint8, device=xin.device)
            ws = ws[(-ws.data_ptr()) % 256:]
            run = (lambda: p.alm2map(xin, workspace=ws)) if op == "alm2map" else (lambda: p.map2alm(xin, workspace=ws))
            run()                                      # warm-up outside the capture (sets kernel attributes)
            torch.cuda.current_stream().synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st, capture_error_mode="thread_local"):
                yout = run()
            self.graphs[gk] = (g, xin, yout, ws)
        g, xin, yout, ws = self.graphs[gk]
        o = 0
        for x in xs:
            xin[o:o + x.shape[0]].copy_(x)
            o += x.shape[0]
        if o < b:
            xin[o:].zero_()
        g.replay()
        return yout[:n]

    def poll(self, handle):
        ev, outs, sid = handle
        if not ev.query():
            return None
        self.free_streams.append(sid)
        return outs
