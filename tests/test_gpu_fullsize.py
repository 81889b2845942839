"""GPU parity against the CPU oracle at the full benchmark sizes.

* Spin 0, nside 512, lmax 1023, 1000 maps in one batch (2000 map columns:
  16 column tiles, clusters of 8 and the small-cluster fill launch in the
  split form; the alm2map contraction runs 8 spans of 128 along l): both
  directions, FP64 form at 1e-10 and split form at 1e-6, the oracle on three
  whole map columns (exact metric: max |err| / RMS over the column).
* Spin 2 (Q/U <-> E/B), nside 1024, lmax 2047, 200 Q/U pairs (deep-underflow
  lambda, the split form's double-float steps from its FP64 checkpoints at
  the largest planned size): both directions and both forms, the oracle on
  two pairs, at sampled outputs the oracle can compute one by one (alm2map
  on 15 rings from pole to pole, map2alm for 95 orders m), normalised by an
  estimate of the column RMS made from oracle-side data only (below).

Inputs are seeded and synthetic. The a_lm of every column are drawn on the
GPU by a seeded torch generator (C_l = 1/(l(l+1)); C_BB = 0.01 C_EE); the
checked columns are copied to the host for the oracle. The map2alm input of
a checked column is the oracle's own alm2map of its a_lm plus 1% white noise
(nside 1024: a band-limited sky of lmax 511, the full-band synthesis being
too slow for a test); unchecked columns carry the GPU's alm2map output plus
noise and are never seen by the oracle."""
import math

import numpy as np
import pytest
import torch

from paper_2208_10154_b300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "split": 1e-6}
# Accuracy budget of the split form at these sizes, beside the 1e-6 contract:
# its measured errors (nside 512: alm2map 1.36e-7, limited by the FP32 output
# of the contraction, 2^-24 per value; map2alm 1.47e-8; nside 1024 spin 2:
# alm2map 1.13e-7, map2alm 4.44e-7, relative to the ten times smaller B
# component) with a margin of 1.5. A change of the arithmetic that loses
# precision below the contract (the compensated ring FFT without its lo
# renormalisation gave 2.4e-7 and 2.6e-8 at nside 512) fails here.
BUDGET = {512: (2.0e-7, 2.2e-8), 1024: (1.7e-7, 6.7e-7)}      # (alm2map, map2alm)


@pytest.fixture(scope="module")
def sht():
    from paper_2208_10154_b300 import build, sht as s
    build.build()
    s.load()
    return s


def _free():
    import gc
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _add_noise(maps, seed, frac=0.01, chunk=8):
    """maps += frac * RMS(map) * N(0, 1) per map, a few maps at a time (no
    full-size temporaries); seeded torch generator."""
    g = torch.Generator(device=maps.device)
    g.manual_seed(int(seed))
    for i in range(0, maps.shape[0], chunk):
        x = maps[i:i + chunk]
        x += frac * x.square().mean(dim=-1, keepdim=True).sqrt() * torch.randn(
            x.shape, generator=g, dtype=x.dtype, device=x.device)


def _colerr(got, want):
    """max |err| / RMS(oracle) per (map, component) over whole columns."""
    g = np.asarray(got).reshape(-1, np.asarray(want).shape[-1])
    w = np.asarray(want).reshape(g.shape)
    den = np.sqrt(np.mean(np.abs(w) ** 2, axis=1))
    return float(np.max(np.max(np.abs(g - w), axis=1) / den))


# ----------------------------------------------------------------- spin 0
NS0, LM0, NM0 = 512, 1023, 1000
PICK0 = [0, 501, 999]          # first, middle and last (ragged) column tile


@pytest.fixture(scope="module")
def spin0_oracle(orc):
    """The checked columns' a_lm, the oracle's maps of them, the noisy map2alm
    inputs and the oracle's a_lm of those inputs."""
    alm = inputs.gaussian_alm_torch(101, NM0, 1, LM0)
    a_s = alm[PICK0].cpu().numpy()
    del alm
    _free()
    m_s = orc.alm2map(a_s, NS0, LM0)
    rng = np.random.default_rng(102)
    t_s = m_s + 0.01 * np.sqrt(np.mean(m_s ** 2, axis=-1, keepdims=True)) * rng.standard_normal(m_s.shape)
    return {"a": a_s, "maps": m_s, "t": t_s, "alm_of_t": orc.map2alm(t_s, NS0, LM0)}


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_spin0_nside512_1000_maps(sht, spin0_oracle, prec):
    ref = spin0_oracle
    NAME = "spin 0, nside 512, lmax 1023, 1000 maps"
    plan = sht.Plan(NS0, LM0, None, 0, prec)
    alm = inputs.gaussian_alm_torch(101, NM0, 1, LM0)
    maps = plan.alm2map(alm)
    torch.cuda.synchronize()
    plan.device_status()
    err_a2m = _colerr(maps[PICK0].cpu().numpy(), ref["maps"])
    # map2alm input: the oracle's noisy maps in the checked columns, the GPU
    # maps plus noise elsewhere (unchecked)
    del alm
    plan._ws = None
    _free()
    _add_noise(maps, 103)
    maps[PICK0] = torch.from_numpy(ref["t"]).cuda()
    out = plan.map2alm(maps)
    torch.cuda.synchronize()
    plan.device_status()
    err_m2a = _colerr(out[PICK0].cpu().numpy(), ref["alm_of_t"])
    plan.close()
    del maps, out, plan
    _free()
    print(f"\n{NAME} {prec}: alm2map {err_a2m:.3e}, map2alm {err_m2a:.3e} (bar {TOL[prec]:.0e})")
    assert err_a2m < TOL[prec], ("alm2map", prec, err_a2m)
    assert err_m2a < TOL[prec], ("map2alm", prec, err_m2a)
    if prec == "split":
        assert err_a2m < BUDGET[NS0][0] and err_m2a < BUDGET[NS0][1], ("budget", err_a2m, err_m2a)


# ----------------------------------------------------------------- spin 2
NS2, LM2, NP2 = 1024, 2047, 200
PICK2 = [0, 199]
LM_IN = 511                    # band limit of the oracle-synthesised map2alm inputs
RINGS2 = [1, 2, 3, 255, 511, 1023, 1024, 1536, 2048, 2560, 3072, 3073, 3584, 4094, 4095]
MSEL2 = list(range(32)) + [32 * k + 16 for k in range(1, 64)] + [2047]


def _idx(lmax, l, m):
    return m * (2 * lmax + 1 - m) // 2 + l


def _rms_qu_parseval(a_pair, lmax):
    """RMS of Q (and of U) from the a_lm of one pair: the integral of Q^2 + U^2
    over the sphere is sum_l [a_E,l0^2 + a_B,l0^2 + 2 sum_{m>0} (|a_E|^2 + |a_B|^2)]
    (orthonormal +-2Y_lm), split evenly between Q and U."""
    _, ms = inputs.lm_arrays(lmax)
    w = np.where(ms == 0, 1.0, 2.0)
    tot = float(np.sum(w * (np.abs(a_pair[0]) ** 2 + np.abs(a_pair[1]) ** 2)))
    return math.sqrt(tot / (8.0 * math.pi))


def _rms_alm_from_msel(blocks, nalm):
    """Column RMS of a_lm estimated from the sampled orders: m < 32 exactly,
    each m = 32k + 16 standing for the 32 orders 32k .. 32k + 31 (the last
    sampled order, mmax, is not counted)."""
    tot = 0.0
    for m, b in zip(MSEL2, blocks):
        if m == 2047:
            continue
        tot += float(np.sum(np.abs(b) ** 2)) * (1 if m < 32 else 32)
    return math.sqrt(tot / nalm)


@pytest.fixture(scope="module")
def spin2_oracle(orc):
    cl = inputs.cl_inv_llp1(LM2)
    alm = inputs.gaussian_alm_torch(201, NP2, 2, LM2, cls=np.stack([cl, 0.01 * cl]))
    a_s = alm[PICK2].cpu().numpy()
    del alm
    _free()
    ring_vals = orc.alm2map_rings(a_s, NS2, LM2, RINGS2, spin=2)          # per ring [pair, comp, N]
    rms_qu = [_rms_qu_parseval(a_s[k], LM2) for k in range(len(PICK2))]
    # map2alm inputs of the checked pairs: a band-limited sky (lmax 511, same
    # spectra) synthesised by the oracle, plus 1% white noise
    cl_in = inputs.cl_inv_llp1(LM_IN)
    a_in = inputs.gaussian_alm(202, len(PICK2), 2, LM_IN, cls=np.stack([cl_in, 0.01 * cl_in]))
    t_s = orc.alm2map(a_in, NS2, LM_IN, spin=2)
    rng = np.random.default_rng(203)
    t_s += 0.01 * np.sqrt(np.mean(t_s ** 2, axis=-1, keepdims=True)) * rng.standard_normal(t_s.shape)
    blocks = orc.map2alm_msel(t_s, NS2, LM2, MSEL2, spin=2)                # per m [pair, comp, lmax-m+1]
    nalm = (LM2 + 1) * (LM2 + 2) // 2
    rms_eb = [[_rms_alm_from_msel([b[k, c] for b in blocks], nalm) for c in range(2)]
              for k in range(len(PICK2))]
    return {"rings": ring_vals, "rms_qu": rms_qu, "t": t_s, "blocks": blocks, "rms_eb": rms_eb}


@pytest.mark.parametrize("prec", ["split", "fp64"])
def test_spin2_nside1024_200_pairs(orc, sht, spin2_oracle, prec):
    ref = spin2_oracle
    _, _, _, n, st = orc.ring_info(NS2)
    NAME = "spin 2, nside 1024, lmax 2047, 200 pairs"
    plan = sht.Plan(NS2, LM2, None, 2, prec)
    cl = inputs.cl_inv_llp1(LM2)
    alm = inputs.gaussian_alm_torch(201, NP2, 2, LM2, cls=np.stack([cl, 0.01 * cl]))
    maps = plan.alm2map(alm)
    torch.cuda.synchronize()
    plan.device_status()
    del alm
    err_a2m = 0.0
    for k, p in enumerate(PICK2):
        for j, r in enumerate(RINGS2):
            got = maps[p, :, st[r - 1]:st[r - 1] + n[r - 1]].cpu().numpy()
            err_a2m = max(err_a2m, float(np.max(np.abs(got - ref["rings"][j][k]))) / ref["rms_qu"][k])
    plan._ws = None
    _free()
    _add_noise(maps, 204)
    maps[PICK2] = torch.from_numpy(ref["t"]).cuda()
    out = plan.map2alm(maps)
    torch.cuda.synchronize()
    plan.device_status()
    del maps
    err_m2a = 0.0
    for k, p in enumerate(PICK2):
        for j, m in enumerate(MSEL2):
            i0 = _idx(LM2, m, m)
            got = out[p, :, i0:i0 + LM2 - m + 1].cpu().numpy()
            for c in range(2):
                e = float(np.max(np.abs(got[c] - ref["blocks"][j][k, c]))) / ref["rms_eb"][k][c]
                err_m2a = max(err_m2a, e)
    plan.close()
    del out, plan
    _free()
    print(f"\n{NAME} {prec}: alm2map {err_a2m:.3e}, map2alm {err_m2a:.3e} (bar {TOL[prec]:.0e})")
    assert err_a2m < TOL[prec], ("alm2map", prec, err_a2m)
    assert err_m2a < TOL[prec], ("map2alm", prec, err_m2a)
    if prec == "split":
        assert err_a2m < BUDGET[NS2][0] and err_m2a < BUDGET[NS2][1], ("budget", err_a2m, err_m2a)
