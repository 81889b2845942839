#!/usr/bin/env python
"""Benchmark: batched HEALPix spherical harmonic transforms on B300.

One step = alm2map + map2alm (spin 0) of one batch of maps at nside 512,
lmax 1023, 1000 maps per GPU (the paper's batched-SHT scheme, Sec. 2.1-2.2),
on synthetic Gaussian skies with C_l = 1/(l(l+1)) plus 1% white noise.
Prints ONE JSON line. Single-GPU only: the split-form contraction shares
lambda pieces inside thread-block clusters with TMA multicast loads, which
this library keeps out of processes that drive more than one GPU. With
--gpus N > 1 or WORLD_SIZE > 1 it prints an "unavailable" line and exits
(maps are independent columns, so N GPUs serve N separate single-GPU
processes; there is no exchange step to measure).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision auto|fp64|split]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the serving run allocates and frees batches of very different sizes on
# several streams: growable segments keep the allocator from fragmenting
os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "expandable_segments:True")

METRIC = "maps/s batched vs per-map on one B300 at <=1e-6 rel err; served p50/p99 latency"
WORKLOAD = "t_nside512"
FP64_PEAK_TFLOPS = 1.25      # nominal B300 FP64 (recipe table); probe measured 1.13 at 2032 MHz
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # FP32 FMA lanes x clock (non-tensor)
SPLIT_PRODUCTS = 10          # tensor-core products per output term in the split form (4 FP16 slices)
# DRAM traffic (read + write) of one launch from an ncu capture of the current
# kernel build at nside 512, lmax 1023, 128 maps (256 columns); at fixed nside
# and lmax it grows in proportion to the map columns. Empty while the kernel
# has changed since the last capture (the line then reports null).
TRAFFIC_NCU = {"k_leg_a2m_tc": 4.956e9, "k_leg_m2a_tc": 4.711e9}
TRAFFIC_NCU_AT = {"nside": 512, "lmax": 1023, "ncol": 256}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "split"])
    ap.add_argument("--nside", type=int, default=512)
    ap.add_argument("--lmax", type=int, default=None)
    ap.add_argument("--nmaps", type=int, default=1000)
    ap.add_argument("--per-map-samples", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--qu1024-pairs", type=int, default=200,
                    help="Q/U pairs of the spin-2 measurement at nside 1024, lmax 2047 (0 skips it)")
    ap.add_argument("--qu-maps", type=int, default=500,
                    help="Q/U map pairs of the spin-2 (polarization) measurement at the same nside; 0 skips it")
    ap.add_argument("--no-context", action="store_true",
                    help="skip the context run (nside 256, lmax 767, 1000 maps, Legendre only)")
    ap.add_argument("--no-next-rows", action="store_true",
                    help="skip the compact-storage and E-projection measurements")
    ap.add_argument("--serve-requests", type=int, default=400,
                    help="requests of the serving measurement, drawn from the serving workload's mix (0: skip)")
    ap.add_argument("--serve-loads", default="0.5,0.8,0.95",
                    help="offered loads of the open-loop serving runs, as fractions of closed-loop saturation")
    ap.add_argument("--serve-no-graphs", action="store_true")
    a = ap.parse_args()
    if a.lmax is None:
        a.lmax = 2 * a.nside - 1
    return a


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


MULTI_GPU_UNAVAILABLE = ("single-GPU only: the split-form contraction multicasts lambda pieces inside "
                         "thread-block clusters (TMA multicast from this GPU's own memory), which is kept out "
                         "of multi-GPU processes; maps are independent columns with no exchange step")


def multi_gpu_requested(a) -> bool:
    """True when the run asks for more than one GPU (flag or torchrun environment)."""
    _, world, _ = dist_info()
    return a.gpus > 1 or world > 1


def unavailable_line(a) -> dict:
    return {"metric": METRIC, "n_gpus": max(a.gpus, dist_info()[1]), "unavailable": MULTI_GPU_UNAVAILABLE}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


def fft_flops_per_map(nside):
    """Nominal flops of one direction's ring FFTs for one spin-0 map: one
    complex FFT of N points per ring pair (the equator ring alone), counted as
    5 N log2 N whatever its length."""
    import math
    tot = 0.0
    for i in range(1, 2 * nside + 1):                 # ring pairs: north ring i with its mirror
        n = 4 * i if i < nside else 4 * nside
        tot += 5.0 * n * math.log2(n)
    return tot


def host_link_gbs(host_buf, torch):
    """Copy bandwidth between pinned host memory and the GPU (GB/s): host to
    device alone, device to host alone, and both at once on two streams (the
    ceiling of the end-to-end measurement)."""
    n = min(host_buf.numel(), 1 << 30)                # up to 8 GB of float64
    h_in = host_buf.view(-1)[:n]
    h_out = torch.empty(n, dtype=host_buf.dtype, pin_memory=True)
    d_a = torch.empty(n, dtype=host_buf.dtype, device="cuda")
    d_b = torch.empty(n, dtype=host_buf.dtype, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    nbytes = n * host_buf.element_size()

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0
    d_a.copy_(h_in, non_blocking=True)
    h_out.copy_(d_b, non_blocking=True)
    t_h2d = timed(lambda: d_a.copy_(h_in, non_blocking=True))
    t_d2h = timed(lambda: h_out.copy_(d_b, non_blocking=True))

    def both():
        with torch.cuda.stream(s1):
            d_a.copy_(h_in, non_blocking=True)
        with torch.cuda.stream(s2):
            h_out.copy_(d_b, non_blocking=True)
    t_both = timed(both)
    out = {"h2d_gbs": nbytes / t_h2d / 1e9, "d2h_gbs": nbytes / t_d2h / 1e9,
           "both_gbs": 2 * nbytes / t_both / 1e9, "bytes_per_copy": nbytes}
    del h_out, d_a, d_b
    return out


def algorithmic_flops(nside, lmax, nmaps, spin=0):
    """Legendre contraction flops per transform (4 per (l, m, ring pair) per map
    for spin 0; x4 for a spin-2 Q/U pair)."""
    R = 2 * nside
    nalm = (lmax + 1) * (lmax + 2) // 2
    return 4.0 * R * nalm * nmaps * (4 if spin else 1)


# ----------------------------------------------------------------------------
def run_reference(a):
    """The CPU oracle (plain FP64, separable tier) on a bounded sample: one map
    per step at the benchmark's nside/lmax (the oracle is timed as it stands)."""
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_2208_10154_b300 import inputs
    oracle.build()
    nside, lmax = a.nside, a.lmax
    alm = inputs.gaussian_alm(1, 1, 1, lmax, cls=inputs.cl_inv_llp1(lmax))
    maps = oracle.alm2map(alm, nside, lmax)
    def step():
        oracle.alm2map(alm, nside, lmax)
        oracle.map2alm(maps, nside, lmax)
    for _ in range(a.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        step()
    dt = time.perf_counter() - t0
    value = a.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "maps/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * dt / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": ref_config(a),
        "cpu_baseline": {"value": value, "unit": "maps/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"1 map per step (alm2map + map2alm, nside {nside}, lmax {lmax})"},
        "e2e": {"value": value, "unit": "maps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def ref_config(a):
    return {"workload": f"{WORKLOAD}: spin-0 alm2map + map2alm, nside {a.nside}, lmax {a.lmax}, "
                        f"{a.nmaps} maps per GPU, C_l = 1/(l(l+1)) + 1% white noise",
            "nside": a.nside, "lmax": a.lmax, "nmaps": a.nmaps, "spin": 0}


# ----------------------------------------------------------------------------
# Serving workload (request mix; see serving_spec)
SERVE_NSIDES = [64, 128, 256, 512, 1024]
SERVE_W = [0.3, 0.3, 0.2, 0.15, 0.05]


def time_eb_only(plan, maps, alm_out, ws, npairs):
    """E-only and B-only spin-2 map2alm beside the full one (events on the current stream)."""
    import torch
    e_only = plan.map2alm_eb(maps, "E", workspace=ws)
    torch.cuda.synchronize()
    t_ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t_ev[0].record()
    plan.map2alm(maps, out=alm_out, workspace=ws)
    t_ev[1].record()
    plan.map2alm_eb(maps, "E", out=e_only, workspace=ws)
    t_ev[2].record()
    plan.map2alm_eb(maps, "B", out=e_only, workspace=ws)
    t_ev[3].record()
    torch.cuda.synchronize()
    t_full, t_e, t_b = (t_ev[i].elapsed_time(t_ev[i + 1]) for i in range(3))
    eb_only = {"pairs": npairs, "map2alm_full_ms": t_full, "map2alm_E_ms": t_e, "map2alm_B_ms": t_b,
               "E_over_full": t_e / t_full, "device_status": plan.device_status(),
               "note": "ring FFTs of Q and U in full; the Legendre contraction forms one component"}
    del e_only
    return eb_only


def run_qu(nside, lmax, npairs, steps, warmup, precision, eb=True):
    """Spin-2 (Q/U <-> E/B) alm2map + map2alm of `npairs` Q/U map pairs per step,
    E/B a_lm Gaussian with C_EE = 1/(l(l+1)), C_BB = 0.01 C_EE, beside the
    per-pair FP64 form; kernel times from libsht's own profiler. eb: also time
    the E-only / B-only map2alm (its output does not fit beside the nside-1024
    batch)."""
    import torch
    from paper_2208_10154_b300 import sht
    plan = sht.Plan(nside, lmax, None, 2, precision)
    ls = torch.arange(lmax + 1, dtype=torch.float64)
    cl = torch.zeros(lmax + 1, dtype=torch.float64)
    cl[2:] = 1.0 / (ls[2:] * (ls[2:] + 1.0))
    from paper_2208_10154_b300 import inputs
    lsa, msa = inputs.lm_arrays(lmax)
    sd = torch.sqrt(cl[torch.from_numpy(lsa)] / torch.where(torch.from_numpy(msa) == 0, 1.0, 2.0)).cuda()
    sd = torch.stack([sd, 0.1 * sd])[None, :, :]
    g = torch.Generator(device="cuda")
    g.manual_seed(2)
    re = torch.randn((npairs, 2, plan.nalm), generator=g, dtype=torch.float64, device="cuda") * sd
    im = torch.randn((npairs, 2, plan.nalm), generator=g, dtype=torch.float64, device="cuda") * sd
    im[..., torch.from_numpy(msa == 0).cuda()] = 0.0
    alm = torch.complex(re, im).contiguous()
    del re, im
    ws = torch.empty(plan.workspace_bytes(npairs) + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    maps = plan.alm2map(alm, workspace=ws)
    alm_out = torch.empty_like(alm)

    def step():
        plan.alm2map(alm, out=maps, workspace=ws)
        plan.map2alm(maps, out=alm_out, workspace=ws)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sht.sht_profile_begin()
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    prof = sht.sht_profile_end()
    ms = e0.elapsed_time(e1) / steps
    status = plan.device_status()
    # E-only map2alm (Sec. 3.1: one of a_E, a_B) beside the full spin-2 map2alm
    eb_only = None
    if eb:
        eb_only = time_eb_only(plan, maps, alm_out, ws, npairs)
    # per-pair FP64 form
    p64 = sht.Plan(nside, lmax, None, 2, "fp64")
    a1 = alm[:1].contiguous()
    m1 = p64.alm2map(a1)
    p64.map2alm(m1)
    torch.cuda.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(2):
        m1 = p64.alm2map(a1)
        p64.map2alm(m1)
    s1.record()
    torch.cuda.synchronize()
    per = 2 / (s0.elapsed_time(s1) / 1e3)
    out = {"value": npairs / (ms / 1e3), "unit": "Q/U map pairs/s", "ms_per_step": ms, "steps": steps,
           "config": {"workload": "qu", "nside": nside, "lmax": lmax, "npairs": npairs, "spin": 2,
                      "precision": precision, "cl": "EE 1/(l(l+1)), BB 0.01 EE", "seed": 2},
           "per_map": {"value": per, "unit": "Q/U map pairs/s", "form": "fp64, one pair"},
           "batched_over_per_map": npairs / (ms / 1e3) / per, "device_status": status, "eb_only": eb_only,
           "kernels": {k: {"launches": v["launches"], "ms": v["ms"] / steps} for k, v in prof.items()}}
    del plan, p64, ws, maps, alm, alm_out
    torch.cuda.empty_cache()
    return out


def run_next_rows(nside, lmax, nmaps, npairs, precision):
    """The widening rows: the compact square a_lm storage (Sec. 5) converted
    both ways for the benchmark's batch (bytes moved / time against HBM), the
    pixel-domain E projection (Sec. 2.3) of npairs Q/U pairs, and Algorithm 3
    against Algorithm 2 at the paper's setting of that comparison."""
    import torch
    from paper_2208_10154_b300 import sht
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    p0 = sht.Plan(nside, lmax, None, 0, "fp64")
    alm = torch.view_as_complex(torch.randn((nmaps, 1, p0.nalm, 2), generator=g, dtype=torch.float64,
                                            device="cuda")).contiguous()
    sq = p0.alm_to_square(alm)
    back = p0.square_to_alm(sq)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    p0.alm_to_square(alm, out=sq)
    e1.record()
    p0.square_to_alm(sq, out=back)
    e2.record()
    torch.cuda.synchronize()
    t_sq, t_back = e0.elapsed_time(e1), e1.elapsed_time(e2)
    ref = alm.clone()
    ref[..., :lmax + 1] = ref[..., :lmax + 1].real.to(torch.complex128)     # Im a_l0 is not stored
    exact = bool(torch.equal(back, ref))
    del ref
    nbytes = alm.numel() * 16 + sq.numel() * 8
    peaks, _ = measured_peaks()
    layout = {"maps": nmaps, "lmax": lmax, "to_square_ms": t_sq, "to_alm_ms": t_back,
              "to_square_gbs": nbytes / (t_sq / 1e3) / 1e9, "to_alm_gbs": nbytes / (t_back / 1e3) / 1e9,
              "hbm_peak_gbs": peaks["hbm_gbs"], "round_trip_exact": exact}
    del alm, sq, back
    torch.cuda.empty_cache()
    p2 = sht.Plan(nside, lmax, None, 2, precision)
    qu = torch.randn((npairs, 2, p2.npix), generator=g, dtype=torch.float64, device="cuda")
    out = p2.eb_project(qu, "E", 0)
    torch.cuda.synchronize()
    e0.record()
    p2.eb_project(qu, "E", 0, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    status = p2.device_status()
    proj = {"pairs": npairs, "which": "E", "niter": 0, "precision": precision, "ms": ms,
            "pairs_per_s": npairs / (ms / 1e3), "device_status": status}
    return {"square_storage": layout, "eb_projection": proj, "immediate": time_immediate()}


def time_immediate(passes=3):
    """Algorithm 3 (immediate iteration, Sec. 4) at the paper's setting of that
    comparison: nside 128, lmax 383 (< 3 nside), 3 passes, FP64 form, 1000
    maps (spin 0) and 500 Q/U pairs (spin 2), beside Algorithm 2 with the
    same number of passes (niter = passes - 1). CUDA events, one call each
    after one untimed call; Gaussian white-noise maps (the cost does not
    depend on the values)."""
    import torch
    from paper_2208_10154_b300 import sht
    nside, lmax = 128, 383
    out = {"nside": nside, "lmax": lmax, "passes": passes, "precision": "fp64"}
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    for spin, nmaps in ((0, 1000), (2, 500)):
        plan = sht.Plan(nside, lmax, None, spin, "fp64")
        x = torch.randn((nmaps, plan.ncomp, plan.npix), generator=g, dtype=torch.float64, device="cuda")
        res = {"maps": nmaps}
        for name, fn in (("immediate_ms", lambda: plan.map2alm_immediate(x, passes)),
                         ("traditional_ms", lambda: plan.map2alm(x, niter=passes - 1))):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = fn()
            e1.record()
            torch.cuda.synchronize()
            res[name] = e0.elapsed_time(e1)
            del r
        plan.device_status()
        res["immediate_maps_per_s"] = nmaps / (res["immediate_ms"] / 1e3)
        out["spin%d" % spin] = res
        del plan, x
        torch.cuda.empty_cache()
    return out


def run_context(precision, steps=3):
    """Context run beside the paper's Appendix B timing model: spin 0, nside 256,
    lmax 767, 1000 maps; the Legendre contractions alone (one alm2map and one
    map2alm per step, their kernel times from libsht's profiler) against the
    paper's t1 = 0.222 s for one Legendre-only transform of 1000 maps on an
    A100 in FP64. Also map2alm with 3 iteration rounds (Algorithm 2) against
    the same without: the paper's round costs 2 t1 = 0.444 s."""
    import torch
    from paper_2208_10154_b300 import sht
    nside, lmax, nmaps = 256, 767, 1000
    plan = sht.Plan(nside, lmax, None, 0, precision)
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    alm = torch.view_as_complex(torch.randn((nmaps, 1, plan.nalm, 2), generator=g, dtype=torch.float64,
                                            device="cuda")).contiguous()
    ws = torch.empty(plan.workspace_bytes(nmaps, 3) + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    maps = plan.alm2map(alm, workspace=ws)
    alm_out = torch.empty_like(alm)
    plan.map2alm(maps, out=alm_out, workspace=ws)
    torch.cuda.synchronize()
    sht.sht_profile_begin()
    for _ in range(steps):
        plan.alm2map(alm, out=maps, workspace=ws)
        plan.map2alm(maps, out=alm_out, workspace=ws)
    torch.cuda.synchronize()
    prof = sht.sht_profile_end()
    plan.device_status()
    leg = {k: v["ms"] / steps for k, v in prof.items() if "leg" in k}
    per_transform = sum(leg.values()) / 2.0
    iter_ms = {}
    for niter in (0, 3):
        plan.map2alm(maps, out=alm_out, niter=niter, workspace=ws)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.map2alm(maps, out=alm_out, niter=niter, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        iter_ms[niter] = e0.elapsed_time(e1)
    plan.device_status()
    out = {"config": {"nside": nside, "lmax": lmax, "nmaps": nmaps, "spin": 0, "precision": precision},
           "legendre_ms_per_transform": per_transform, "legendre_kernels_ms": leg,
           "paper_t1_ms": 222.0, "paper_hw": "one A100, FP64 (App. B)",
           "ratio_paper_over_ours": 222.0 / per_transform,
           "map2alm_ms": {"niter0": iter_ms[0], "niter3": iter_ms[3]},
           "iteration_round_ms": (iter_ms[3] - iter_ms[0]) / 3.0, "paper_round_ms": 444.0}
    del plan, ws, maps, alm, alm_out
    torch.cuda.empty_cache()
    return out


def serving_spec(n_req, seed=3):
    """Requests of the serving workload: op alm2map / map2alm 50/50, spin 2
    with probability 0.3, nside from {64, 128, 256, 512, 1024} with weights
    {0.3, 0.3, 0.2, 0.15, 0.05}, lmax = 2 nside - 1, maps uniform in 1..256."""
    import numpy as np
    rng = np.random.default_rng(seed)
    w = np.array(SERVE_W) / np.sum(SERVE_W)
    spec = []
    for _ in range(n_req):
        nside = int(rng.choice(SERVE_NSIDES, p=w))
        spin = 2 if rng.random() < 0.3 else 0
        op = "alm2map" if rng.random() < 0.5 else "map2alm"
        spec.append((op, nside, spin, int(rng.integers(1, 257))))
    return spec, rng


def run_serving(n_req, loads, device, use_graphs=True):
    """The serving workload through the continuous-batching server: closed
    loop (all requests at once: saturation), then Poisson arrivals at each
    offered load (a fraction of saturation). Inputs: one pool of maps per
    (op, nside, spin), 256 maps (64 for nside >= 512); a request of n maps
    takes the pool's first n, or repeats of the pool passed as a list of
    pieces. Results are dropped as requests finish (the caller would take
    them); the split form within its limits, HBM budget 150 GB."""
    import numpy as np
    import torch
    from paper_2208_10154_b300.serving import GpuExecutor, Request, Server
    spec, rng = serving_spec(n_req)
    pool = {}
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    for op, nside, spin, _ in spec:
        k = (op, nside, spin)
        if k in pool:
            continue
        ncomp = 2 if spin else 1
        lmax = 2 * nside - 1
        npool = 64 if nside >= 512 else 256
        if op == "alm2map":
            nalm = (lmax + 1) * (lmax + 2) // 2
            x = torch.randn((npool, ncomp, nalm, 2), generator=g, dtype=torch.float64, device="cuda")
            pool[k] = torch.view_as_complex(x).contiguous()
            del x
        else:
            pool[k] = torch.randn((npool, ncomp, 12 * nside * nside), generator=g, dtype=torch.float64,
                                  device="cuda")

    def data(k, n):
        p = pool[k]
        if n <= p.shape[0]:
            return p[:n]
        q, r = divmod(n, p.shape[0])
        return [p] * q + ([p[:r]] if r else [])

    budget = 150e9
    ex = GpuExecutor(device=device, slots=4, use_graphs=use_graphs, mem_cap=budget, small_slots=2)

    def drop(r):
        r.result = None
    srv = Server(ex, hbm_budget=budget, max_batch_maps=256, slots=6, on_complete=drop)

    def run(sp, arrivals):
        srv.completed.clear()
        srv.nbatches = 0
        srv.peak_used = 0.0
        t0 = time.perf_counter()
        i = 0
        while i < len(sp) or not srv.idle():
            now = time.perf_counter() - t0
            while i < len(sp) and arrivals[i] <= now:
                op, nside, spin, n = sp[i]
                srv.submit(Request(op=op, nside=nside, spin=spin, data=data((op, nside, spin), n),
                                   t_arrival=t0 + arrivals[i]))
                i += 1
            if not srv.step():
                time.sleep(1e-4)
        torch.cuda.synchronize()
        st = srv.stats()
        st["peak_admitted_gb"] = srv.peak_used / 1e9
        return st

    for op, nside, spin, _ in spec:                         # every plan before any timing
        ex.prepare(Request(op=op, nside=nside, spin=spin, data=pool[(op, nside, spin)][:1]).key("auto"))
    warm = spec[:min(len(spec), 64)]                       # kernel attributes, first graphs
    run(warm, np.zeros(len(warm)))
    closed = run(spec, np.zeros(len(spec)))
    mean_maps = sum(s[3] for s in spec) / len(spec)
    out = {"requests": len(spec), "saturation": {k: closed.get(k) for k in (
               "maps_per_s", "p50_ms", "p99_ms", "batches", "errors", "first_error", "peak_admitted_gb")},
           "open_loop": [], "graphs": use_graphs, "graph_replays": ex.graph_replays,
           "workload": "serving mix: Poisson arrivals; alm2map/map2alm 50/50; nside 64/128/256/512/1024 "
                       "(0.3/0.3/0.2/0.15/0.05), lmax = 2 nside - 1; spin 2 in 30%; 1-256 maps per request; "
                       "split form; HBM budget 150 GB; seed 3; "
                       f"{len(spec)} of the workload's 20000 requests"}
    errors = closed.get("errors", 0) or 0
    first = closed.get("first_error")
    peak = closed.get("peak_admitted_gb", 0.0) or 0.0
    for load in loads:
        rate = load * closed["maps_per_s"] / mean_maps
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(spec)))
        o = run(spec, arrivals)
        out["open_loop"].append({"offered_load": load, "offered_requests_per_s": rate,
                                 "p50_ms": o.get("p50_ms"), "p99_ms": o.get("p99_ms"),
                                 "maps_per_s": o.get("maps_per_s"), "batches": o.get("batches"),
                                 "errors": o.get("errors"), "first_error": o.get("first_error"),
                                 "peak_admitted_gb": o.get("peak_admitted_gb")})
        errors += o.get("errors", 0) or 0
        first = first or o.get("first_error")
        peak = max(peak, o.get("peak_admitted_gb", 0.0) or 0.0)
    ref = next((x for x in out["open_loop"] if x["offered_load"] == 0.8), out["open_loop"][-1] if loads else {})
    out.update({"p50_ms": ref.get("p50_ms"), "p99_ms": ref.get("p99_ms"), "maps_per_s": ref.get("maps_per_s"),
                "errors": errors, "first_error": first, "peak_admitted_gb": peak,
                "resident_gb_at_end": ex.resident_bytes() / 1e9})
    del srv, ex, pool
    gc.collect()
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------
def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if multi_gpu_requested(a):
        if dist_info()[0] == 0:
            print(json.dumps(unavailable_line(a)), flush=True)
        return 0
    import numpy as np
    import torch
    from paper_2208_10154_b300 import build, sht
    torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    build.build()
    sht.load()
    nside, lmax, nmaps = a.nside, a.lmax, a.nmaps
    precision = a.precision
    if precision == "auto":
        try:
            p = sht.Plan(4, 7, None, 0, "split")
            p.close()
            precision = "split"
        except sht.ShtError:
            precision = "fp64"

    # ---- inputs: Gaussian a_lm (seed 1), maps = alm2map(a) + 1% noise ----
    t0 = time.perf_counter()
    plan64 = sht.Plan(nside, lmax, None, 0, "fp64")
    plan = plan64 if precision == "fp64" else sht.Plan(nside, lmax, None, 0, precision)
    plan_s = time.perf_counter() - t0
    from paper_2208_10154_b300 import inputs
    ls, ms = inputs.lm_arrays(lmax)
    cl = inputs.cl_inv_llp1(lmax)[ls]
    sd = torch.from_numpy(np.where(ms == 0, np.sqrt(cl), np.sqrt(cl / 2.0))).cuda()
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    re = torch.randn((nmaps, 1, plan.nalm), generator=g, dtype=torch.float64, device="cuda") * sd
    im = torch.randn((nmaps, 1, plan.nalm), generator=g, dtype=torch.float64, device="cuda") * sd
    im[..., torch.from_numpy(ms == 0).cuda()] = 0.0
    alm = torch.complex(re, im).contiguous()
    del re, im
    maps_in = plan64.alm2map(alm)
    rms = maps_in.square().mean(dim=-1, keepdim=True).sqrt()
    maps_in += 0.01 * rms * torch.randn(maps_in.shape, generator=g, dtype=torch.float64, device="cuda")
    plan64._ws = None
    maps_out = torch.empty_like(maps_in)
    alm_out = torch.empty_like(alm)
    wsb = max(plan.workspace_bytes(nmaps), 1)
    ws = torch.empty(wsb + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    torch.cuda.synchronize()

    launches = [0]

    def step():
        plan.alm2map(alm, out=maps_out, workspace=ws)
        launches[0] += sht.sht_last_launch_count()
        plan.map2alm(maps_in, out=alm_out, workspace=ws)
        launches[0] += sht.sht_last_launch_count()

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    launches[0] = 0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    sht.sht_profile_begin()
    with ClockSampler(dev) as clk:
        e0.record()
        for _ in range(a.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
    prof = sht.sht_profile_end()
    plan.device_status()                 # raises if a bounded device wait gave up
    ms_step = e0.elapsed_time(e1) / a.steps
    value = nmaps / (ms_step / 1e3)
    gpu_launches = launches[0]

    # ---- per-map FP64 form (the paper's "one map at a time" baseline) ----
    per_map = None
    if a.per_map_samples > 0:
        plan1 = plan64
        P = min(a.per_map_samples, nmaps)
        for i in range(1):
            plan1.alm2map(alm[i:i + 1].contiguous())
            plan1.map2alm(maps_in[i:i + 1].contiguous())
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        views = [(alm[i:i + 1].contiguous(), maps_in[i:i + 1].contiguous()) for i in range(P)]
        s0.record()
        for av, mv in views:
            plan1.alm2map(av)
            plan1.map2alm(mv)
        s1.record()
        torch.cuda.synchronize()
        per_map = {"value": P / (s0.elapsed_time(s1) / 1e3), "unit": "maps/s", "form": "fp64, nmaps=1",
                   "samples": P}
        plan1._ws = None

    # ---- roofline of the dominant Legendre kernel ----
    peaks, peak_src = measured_peaks()
    legs = {k: v for k, v in prof.items() if "leg" in k} if prof else {}
    dom = max((legs or prof).items(), key=lambda kv: kv[1]["ms"]) if prof else None
    roofline = None
    if dom:
        name, rec = dom
        avg_ms = rec["ms"] / max(rec["launches"], 1)
        flops = algorithmic_flops(nside, lmax, nmaps)
        if "leg" in name and "f64" in name:
            ach = flops / (avg_ms / 1e3) / 1e12
            roofline = {"kernel": name, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                        "peak_source": "nominal FP64 of the profiling recipe (no measured FP64 peak)",
                        "avg_launch_ms": avg_ms, "algorithmic_flops_per_launch": flops}
        elif "leg" in name:
            # split form: `achieved` counts the method's own flops (4 per (l, m,
            # ring pair, map), every term); the tensor cores execute
            # SPLIT_PRODUCTS FP16 slice products per term they evaluate
            # (kind::f16 runs at the bf16 rate), which `executed` reports
            # against the same peak; the ring optimisation leaves out the
            # share 1 - kept of the terms (negligible lambda on polar rings)
            ach = flops / (avg_ms / 1e3) / 1e12
            kept = plan.terms_kept()
            pk = peaks.get("bf16_tflops_sustained", 1400.0)
            traffic = None
            if name in TRAFFIC_NCU and (nside, lmax) == (TRAFFIC_NCU_AT["nside"], TRAFFIC_NCU_AT["lmax"]):
                traffic = TRAFFIC_NCU[name] * (2 * nmaps) / TRAFFIC_NCU_AT["ncol"]
            roofline = {"kernel": name, "bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                        "frac": ach / pk, "traffic": traffic,
                        "traffic_source": "ncu capture at 128 maps, scaled by map columns" if traffic else None,
                        "peak_source": f"bf16 dense sustained ({peak_src}); the kernel runs inside a long step",
                        "algorithmic_flops_per_launch": flops, "avg_launch_ms": avg_ms,
                        "executed": {"products_per_term": SPLIT_PRODUCTS, "terms_kept": kept,
                                     "flops_per_launch": SPLIT_PRODUCTS * kept * flops,
                                     "achieved": SPLIT_PRODUCTS * kept * ach,
                                     "frac": SPLIT_PRODUCTS * kept * ach / pk}}
        else:
            byts = 8.0 * nmaps * plan.npix * 2
            ach = byts / (avg_ms / 1e3) / 1e9
            roofline = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                        "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None,
                        "peak_source": peak_src, "avg_launch_ms": avg_ms}

    # ---- ring FFTs: against HBM (algorithmic bytes of both directions per
    # step: maps read and written in FP64, T written as FP32 hi/lo pairs, G
    # read in FP32) and against the FP32 ALU (5 N log2 N flops per complex
    # ring-pair FFT of N points, both directions), over their summed time ----
    fft_roofline = None
    fft_ms = sum(v["ms"] for k, v in prof.items() if "fft" in k) / max(a.steps, 1) if prof else 0.0
    if fft_ms > 0:
        nring = 4 * nside - 1
        fft_bytes_map = 16.0 * plan.npix * plan.ncomp + (plan.mmax + 1) * nring * plan.ncomp * (16.0 + 8.0)
        ach = fft_bytes_map * nmaps / (fft_ms / 1e3) / 1e9
        fft_flops = 2.0 * fft_flops_per_map(nside) * nmaps
        ach_alu = fft_flops / (fft_ms / 1e3) / 1e12
        fft_roofline = {"kernels": "ring FFTs (all size classes, both directions)", "bound": "hbm",
                        "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                        "ms_per_step": fft_ms, "algorithmic_bytes_per_step": fft_bytes_map * nmaps,
                        "alu": {"bound": "alu", "achieved": ach_alu, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                "frac": ach_alu / FP32_PEAK_TFLOPS, "algorithmic_flops_per_step": fft_flops,
                                "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz",
                                "note": "each flop runs as several compensated FP32 operations"}}

    # ---- end to end through the host-buffer C-ABI entry points: the two
    # directions of a step from two host threads, one plan each (the host
    # entry points are not for concurrent calls on one plan), so that the
    # host->device copies of one overlap the device->host copies of the
    # other (PCIe is full duplex) ----
    e2e = None
    if not a.no_e2e:
        alm_h = torch.empty(alm.shape, dtype=torch.complex128, pin_memory=True)
        alm_h.copy_(alm)
        maps_h = torch.empty(maps_in.shape, dtype=torch.float64, pin_memory=True)
        maps_h.copy_(maps_in)
        mo_h = torch.empty(maps_in.shape, dtype=torch.float64, pin_memory=True)
        ao_h = torch.empty(alm.shape, dtype=torch.complex128, pin_memory=True)
        del maps_out, alm_out, ws
        maps_out = alm_out = ws = None
        torch.cuda.empty_cache()
        plan_b = sht.Plan(nside, lmax, None, 0, precision)
        sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
        errs = []

        def a2m():
            try:
                with torch.cuda.stream(sa):
                    plan.alm2map_host(alm_h.numpy(), out_host=mo_h.numpy())
            except Exception as ex:                  # surfaced after the join
                errs.append(ex)

        def m2a():
            try:
                with torch.cuda.stream(sb):
                    plan_b.map2alm_host(maps_h.numpy(), out_host=ao_h.numpy())
            except Exception as ex:
                errs.append(ex)

        def both():
            th = [threading.Thread(target=a2m), threading.Thread(target=m2a)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            if errs:
                raise errs[0]
        both()                                       # staging buffers, kernel attributes
        t0 = time.perf_counter()
        ke = max(1, min(a.steps, 2))
        for _ in range(ke):
            both()
        dt = (time.perf_counter() - t0) / ke
        nb_alm = alm_h.numel() * 16
        nb_map = maps_h.numel() * 8
        e2e = {"value": nmaps / dt, "unit": "maps/s", "h2d_bytes_per_step": nb_alm + nb_map,
               "d2h_bytes_per_step": nb_map + nb_alm, "api": "sht_alm2map_host + sht_map2alm_host",
               "directions": "concurrent: two host threads, one plan each",
               "host_link": host_link_gbs(maps_h, torch)}
        e2e["host_link"]["e2e_gbs"] = (nb_alm + nb_map) * 2 / dt / 1e9
        plan_b.close()
        del plan_b

    # ---- CPU baseline: the oracle on one map ----
    cpu = None
    if not a.no_cpu_baseline:
        import oracle
        oracle.build()
        a1 = alm[:1].cpu().numpy()
        m1 = maps_in[:1].cpu().numpy()
        t0 = time.perf_counter()
        oracle.alm2map(a1, nside, lmax)
        oracle.map2alm(m1, nside, lmax)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "maps/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"1 map (alm2map + map2alm, nside {nside}, lmax {lmax}), separable tier"}

    del alm, maps_in, maps_out, alm_out, ws
    # the step's plans hold the host entry points' device buffers (up to 48 GB)
    for pl in {id(plan): plan, id(plan64): plan64}.values():
        pl.close()
    del plan, plan64
    gc.collect()
    torch.cuda.empty_cache()
    context = None
    if not a.no_context:
        context = run_context(precision)
    qu = None
    if a.qu_maps > 0:
        qu = run_qu(nside, lmax, a.qu_maps, max(1, min(a.steps, 3)), max(1, min(a.warmup, 2)), precision)
    qu1024 = None
    if a.qu1024_pairs > 0:
        gc.collect()
        torch.cuda.empty_cache()
        qu1024 = run_qu(1024, 2047, a.qu1024_pairs, 2, 1, precision, eb=False)

    next_rows = None
    if not a.no_next_rows:
        next_rows = run_next_rows(nside, lmax, nmaps, 100, precision)

    serving = None
    if a.serve_requests > 0:
        # the serving run admits up to 150 GB of batches: release the step's
        # plans (and their host-path staging buffers) and cached blocks first
        plan = plan64 = None
        gc.collect()
        torch.cuda.empty_cache()
        serving = run_serving(a.serve_requests, [float(x) for x in a.serve_loads.split(",") if x],
                              dev, use_graphs=not a.serve_no_graphs)

    line = {
        "metric": METRIC, "value": value, "unit": "maps/s", "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "f16+f64",
        "data": "synthetic",
        "config": dict(ref_config(a), precision=precision, direction="alm2map+map2alm per step",
                       l2="inputs larger than L2 (maps 25.2 GB per GPU), no flush",
                       parallelism="single GPU"),
        "clocks": clk.summary(), "gpu_launches": gpu_launches, "roofline": roofline,
        "roofline_fft": fft_roofline,
        "cpu_baseline": cpu, "e2e": e2e, "per_map": per_map,
        "batched_over_per_map": value / per_map["value"] if per_map else None,
        "kernels": prof, "plan_create_s": plan_s, "qu": qu, "qu_nside1024": qu1024, "context": context,
        "next_rows": next_rows,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
