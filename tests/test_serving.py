"""Serving loop: continuous batching, HBM admission and per-request routing
(CPU, with a fake executor), and on the GPU: each result is the same alone
and in the mix."""
import numpy as np
import pytest

from paper_2208_10154_b300.serving import Request, Server


class FakeExecutor:
    """Batches finish after `lag` polls; output of a request = 2 x its input."""

    def __init__(self, lag=2, bytes_per_map=1000):
        self.lag, self.bpm = lag, bytes_per_map
        self.launched = []

    def prepare(self, key):
        return key

    def batch_bytes(self, key, n):
        return n * self.bpm

    def launch(self, key, inputs):
        self.launched.append((key, sum(len(x) for x in inputs)))
        return {"left": self.lag, "outs": [2 * x for x in inputs]}

    def poll(self, h):
        h["left"] -= 1
        return h["outs"] if h["left"] < 0 else None


def _req(op, nside, n, rng):
    return Request(op=op, nside=nside, spin=0, data=rng.standard_normal((n, 1, 3)))


def test_batches_group_by_key_and_route_results():
    rng = np.random.default_rng(0)
    ex = FakeExecutor()
    srv = Server(ex, hbm_budget=1e9, max_batch_maps=8, slots=2)
    reqs = [srv.submit(_req(op, ns, int(rng.integers(1, 4)), rng))
            for op, ns in [("alm2map", 8), ("map2alm", 8), ("alm2map", 16)] * 5]
    srv.run_until_idle()
    for r in reqs:
        assert r.done.is_set() and r.error is None
        np.testing.assert_array_equal(r.result, 2 * r.data)
    assert all(n <= 8 for _, n in ex.launched)
    assert len(ex.launched) < len(reqs)             # requests of a key share batches
    for key, _ in ex.launched:
        assert key[0] in ("alm2map", "map2alm")
    st = srv.stats()
    assert st["requests"] == len(reqs) and st["errors"] == 0 and st["p99_ms"] >= st["p50_ms"]


def test_admission_respects_budget_and_slots():
    rng = np.random.default_rng(1)
    ex = FakeExecutor(lag=3, bytes_per_map=100)
    srv = Server(ex, hbm_budget=1000, max_batch_maps=6, slots=3)
    for i in range(12):
        srv.submit(_req("alm2map", 8 * (1 + i % 3), 5, rng))
    while not srv.idle():
        srv.step()
        assert len(srv.inflight) <= 3
        assert srv.used <= 1000
    assert srv.peak_used <= 1000


def test_batches_fit_the_budget_beside_resident_memory():
    """A batch grows only while it fits the budget left beside what the
    executor keeps resident; the admitted total never exceeds the budget."""
    class Resident(FakeExecutor):
        def resident_bytes(self):
            return 400.0
    rng = np.random.default_rng(5)
    ex = Resident(lag=2, bytes_per_map=100)
    srv = Server(ex, hbm_budget=1000, max_batch_maps=64, slots=2)
    for i in range(6):
        srv.submit(_req("alm2map", 8, 3, rng))
    while not srv.idle():
        srv.step()
        assert srv.used + 400.0 <= 1000
    assert all(n <= 6 for _, n in ex.launched)       # (1000 - 400) / 100 maps per batch
    assert srv.peak_used <= 1000


def test_graph_captured_at_launch_is_counted_once():
    """A batch that captures a CUDA graph is admitted with the graph's bytes;
    once launched those bytes are resident (reported by resident_bytes) and
    no longer the batch's, so the admitted peak stays within the budget."""
    class Graphs(FakeExecutor):
        def __init__(self):
            super().__init__(lag=2, bytes_per_map=100)
            self.cached = set()

        def resident_bytes(self):
            return 150.0 * len(self.cached)

        def batch_bytes(self, key, n):
            return n * self.bpm + (0 if key in self.cached else 150)

        def launch(self, key, inputs):
            self.cached.add(key)
            return super().launch(key, inputs)
    rng = np.random.default_rng(6)
    ex = Graphs()
    srv = Server(ex, hbm_budget=1000, max_batch_maps=8, slots=2)
    for i in range(8):
        srv.submit(_req("alm2map", 8 * (1 + i % 2), 4, rng))
    while not srv.idle():
        srv.step()
        assert srv.used + ex.resident_bytes() <= 1000
    assert srv.peak_used <= 1000


def test_continuous_admission_while_busy():
    rng = np.random.default_rng(2)
    ex = FakeExecutor(lag=5)
    srv = Server(ex, hbm_budget=1e9, max_batch_maps=64, slots=2)
    first = srv.submit(_req("map2alm", 8, 2, rng))
    srv.step()
    assert len(srv.inflight) == 1
    late = srv.submit(_req("alm2map", 8, 3, rng))    # arrives while the first batch runs
    srv.step()
    assert len(srv.inflight) == 2                     # admitted into the free slot
    srv.run_until_idle()
    assert first.done.is_set() and late.done.is_set()


def test_failed_batch_fails_only_its_requests():
    class Boom(FakeExecutor):
        def launch(self, key, inputs):
            if key[1] == 16:
                raise RuntimeError("no plan")
            return super().launch(key, inputs)
    rng = np.random.default_rng(3)
    srv = Server(Boom(), hbm_budget=1e9)
    a = srv.submit(_req("alm2map", 16, 1, rng))
    b = srv.submit(_req("alm2map", 8, 1, rng))
    srv.run_until_idle()
    assert a.error and b.error is None and b.result is not None


def test_batches_finishing_out_of_order():
    """A later batch can finish first; retiring it must not compare the
    array payloads of the others."""
    class Lifo(FakeExecutor):
        def launch(self, key, inputs):
            h = super().launch(key, inputs)
            h["left"] = 10 - len(self.launched)      # later launches finish sooner
            return h
    rng = np.random.default_rng(4)
    ex = Lifo()
    srv = Server(ex, hbm_budget=1e9, max_batch_maps=3, slots=4)
    reqs = [srv.submit(_req("alm2map", 8, 3, rng)) for i in range(4)]    # one key, one batch each
    srv.run_until_idle()
    for r in reqs:
        assert r.error is None
        np.testing.assert_array_equal(r.result, 2 * r.data)
    assert srv.completed != reqs                      # retired out of order


def test_executor_rows_and_gather_cpu():
    """Row ranges of a list of pieces: a contiguous view when the range lies
    in one piece, else a gather in order (GpuExecutor helpers, CPU tensors)."""
    import torch
    from paper_2208_10154_b300.serving import GpuExecutor
    pieces = [torch.arange(3 * 2 * 4, dtype=torch.float64).reshape(3, 2, 4) + 100 * i for i in range(3)]
    cat = torch.cat(pieces)
    v = GpuExecutor._rows(pieces, 3, 5)
    assert v is not None and torch.equal(v, cat[3:5])
    assert GpuExecutor._rows(pieces, 2, 4) is None
    dst = torch.empty((5, 2, 4), dtype=torch.float64)
    GpuExecutor._gather(pieces, 2, 7, dst)
    assert torch.equal(dst, cat[2:7])


def test_executor_chunk_fits_the_cap():
    """Chunk selection: the whole batch when it fits, else halvings until
    workspace + staging + output fit the memory cap."""
    from paper_2208_10154_b300.serving import GpuExecutor

    class P:
        ncomp, nalm, npix = 1, 10, 100

        def workspace_bytes(self, n):
            return 1000 * n
    ex = GpuExecutor.__new__(GpuExecutor)
    ex.resident_bytes = lambda: 0.0
    ex.mem_cap = 1e9
    assert ex._chunk(P(), "alm2map", 64) == 64
    ex.mem_cap = 64 * 800 + 8 * (1000 + 160)            # output of 64 maps + 8 maps of the rest
    c = ex._chunk(P(), "alm2map", 64)
    assert c == 8 and 1000 * c + 160 * c + 64 * 800 <= ex.mem_cap


@pytest.mark.gpu
@pytest.mark.parametrize("graphs,chunked", [(False, False), (True, False), (False, True)])
def test_gpu_results_same_alone_and_in_the_mix(graphs, chunked):
    import torch
    from paper_2208_10154_b300 import build, inputs, sht
    from paper_2208_10154_b300.serving import GpuExecutor
    build.build()
    rng = np.random.default_rng(7)
    # chunked: a memory cap that forces batches through several library calls
    ex = GpuExecutor(slots=3, use_graphs=graphs, mem_cap=2e6 if chunked else 150e9)
    srv = Server(ex, hbm_budget=4e9, max_batch_maps=16, slots=3)
    reqs = []
    for i in range(18):
        nside = [8, 16, 32][i % 3]
        spin = 2 if i % 5 == 4 else 0
        op = "alm2map" if i % 2 == 0 else "map2alm"
        n = int(rng.integers(1, 5))
        lmax = 2 * nside - 1
        ncomp = 2 if spin else 1
        if op == "alm2map":
            a = inputs.gaussian_alm(100 + i, n, ncomp, lmax, cls=inputs.cl_inv_llp1(lmax))
            data = torch.from_numpy(a).cuda()
        else:
            data = torch.from_numpy(rng.standard_normal((n, ncomp, 12 * nside * nside))).cuda()
        if chunked and n > 1:                         # a request given as a list of pieces
            data = [data[:1], data[1:]]
        reqs.append(srv.submit(Request(op=op, nside=nside, spin=spin, data=data)))
    srv.run_until_idle()
    torch.cuda.synchronize()
    assert srv.stats()["errors"] == 0
    for r in reqs:
        p = ex.prepare(r.key("auto"))
        x = torch.cat(list(r.data)) if isinstance(r.data, list) else r.data
        alone = p.alm2map(x) if r.op == "alm2map" else p.map2alm(x)
        d = (r.result - alone).abs().max().item()
        s = alone.abs().max().item()
        assert d <= 1e-12 * s, (r.op, r.nside, r.spin, d, s)
