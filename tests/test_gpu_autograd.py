"""Autograd wrappers (differentiable alm2map / map2alm with the libsht
adjoints) against central finite differences and against the oracle's
explicit transposes, on the refinement loss of the differentiable workload
(three Algorithm-2 steps, squared residual to a fixed target map)."""
import numpy as np
import pytest
import torch

from paper_2208_10154_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2208_10154_b300 import build, sht, autograd
    build.build()
    sht.load()
    return sht, autograd


def _ri(a):
    return torch.view_as_real(torch.from_numpy(a)).cuda().clone()


def test_gradcheck_linear_maps(mods):
    sht, ag = mods
    nside, lmax = 4, 7
    plan = sht.Plan(nside, lmax, None, 0, "fp64")
    a = _ri(inputs.gaussian_alm(11, 2, 1, lmax, cls=np.ones(lmax + 1))).requires_grad_(True)
    m = torch.randn((2, 1, 12 * nside * nside), dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: ag.alm2map(x, plan), (a,), eps=1e-6, atol=1e-8)
    assert torch.autograd.gradcheck(lambda x: ag.map2alm(x, plan), (m,), eps=1e-6, atol=1e-8)


def _loss(ag, plan, a_ri, target, niter=3):
    a3 = ag.refine(a_ri, target, plan, niter)
    return (ag.alm2map(a3, plan) - target).square().sum()


def test_refinement_loss_finite_differences(mods):
    sht, ag = mods
    nside, lmax, nmaps = 32, 63, 4
    plan = sht.Plan(nside, lmax, None, 0, "fp64")
    rng = np.random.default_rng(4)
    a0 = _ri(inputs.gaussian_alm(4, nmaps, 1, lmax, cls=inputs.cl_inv_llp1(lmax)))
    target = torch.from_numpy(rng.standard_normal((nmaps, 1, 12 * nside * nside)) * 0.1).cuda()
    a = a0.clone().requires_grad_(True)
    loss = _loss(ag, plan, a, target)
    loss.backward()
    g = a.grad.detach()
    flat = a0.view(-1)
    idx = rng.choice(flat.numel(), 64, replace=False)
    h = 1e-6
    ls_, ms_ = inputs.lm_arrays(lmax)
    for i in idx:
        ap = a0.clone().view(-1); ap[i] += h
        am = a0.clone().view(-1); am[i] -= h
        with torch.no_grad():
            fd = (_loss(ag, plan, ap.view_as(a0), target) - _loss(ag, plan, am.view_as(a0), target)) / (2 * h)
        an = g.view(-1)[i]
        # Im a_l0 is not a parameter: both sides are zero there
        assert abs(float(fd) - float(an)) <= 1e-5 * max(1.0, abs(float(fd))), (int(i), float(fd), float(an))


def test_refinement_gradient_matches_oracle_transposes(orc, mods):
    sht, ag = mods
    nside, lmax, nmaps = 8, 15, 2
    plan = sht.Plan(nside, lmax, None, 0, "fp64")
    rng = np.random.default_rng(5)
    a0 = inputs.gaussian_alm(6, nmaps, 1, lmax, cls=np.ones(lmax + 1))
    target = rng.standard_normal((nmaps, 1, 12 * nside * nside))
    a = _ri(a0).requires_grad_(True)
    _loss(ag, plan, a, torch.from_numpy(target).cuda()).backward()
    got = torch.view_as_complex(a.grad.detach().contiguous()).cpu().numpy()
    # reverse mode with the oracle's transposes: a_{k+1} = a_k + M (T - A a_k)
    a_k = [a0]
    for _ in range(3):
        a_k.append(a_k[-1] + orc.map2alm(target - orc.alm2map(a_k[-1], nside, lmax), nside, lmax))
    r = orc.alm2map(a_k[3], nside, lmax) - target
    g = orc.alm2map_adjoint(2 * r, nside, lmax)
    for _ in range(3):
        g = g - orc.alm2map_adjoint(orc.map2alm_adjoint(g, nside, lmax), nside, lmax)
    scale = np.abs(g).max()
    assert np.max(np.abs(got - g)) <= 1e-10 * scale


def test_refinement_gradient_at_nside256_256_maps(orc, mods):
    """The differentiable workload's own shape: nside 256, lmax 511, 256 maps,
    FP64, loss = squared residual after three Algorithm-2 steps. The gradient
    comes from one backward pass over the whole batch. The loss is a sum of
    per-map terms and every transform acts on each map alone, so the
    derivative by a coefficient of map k is that of map k's term: central
    differences (step 1e-6) on 64 random components evaluate map k's term
    alone (free of the other maps' rounding), and the oracle's explicit
    transposes check two whole maps (to 2e-9 of the gradient's largest
    entry: a chain of 14 FP64 transforms)."""
    sht, ag = mods
    nside, lmax, nmaps = 256, 511, 256
    plan = sht.Plan(nside, lmax, None, 0, "fp64")
    rng = np.random.default_rng(4)
    a0 = _ri(inputs.gaussian_alm(4, nmaps, 1, lmax, cls=inputs.cl_inv_llp1(lmax)))
    t_np = rng.standard_normal((nmaps, 1, 12 * nside * nside)) * 0.05
    target = torch.from_numpy(t_np).cuda()
    a = a0.clone().requires_grad_(True)
    _loss(ag, plan, a, target).backward()
    g = a.grad.detach()
    per = g[0].numel()
    idx = rng.choice(a0.numel(), 64, replace=False)
    h = 1e-6
    for i in idx:
        k, j = divmod(int(i), per)
        ak = a0[k:k + 1].clone()
        ap = ak.clone().view(-1); ap[j] += h
        am = ak.clone().view(-1); am[j] -= h
        with torch.no_grad():
            fd = (_loss(ag, plan, ap.view_as(ak), target[k:k + 1]) -
                  _loss(ag, plan, am.view_as(ak), target[k:k + 1])) / (2 * h)
        an = float(g.view(-1)[i])
        assert abs(float(fd) - an) <= 1e-5 * max(1.0, abs(float(fd))), (int(i), float(fd), an)
    # reverse mode with the oracle's transposes on two maps
    got = torch.view_as_complex(g.contiguous()).cpu().numpy()
    for k in (0, nmaps - 1):
        ak0 = torch.view_as_complex(a0[k:k + 1].contiguous()).cpu().numpy()
        tk = t_np[k:k + 1]
        a_k = [ak0]
        for _ in range(3):
            a_k.append(a_k[-1] + orc.map2alm(tk - orc.alm2map(a_k[-1], nside, lmax), nside, lmax))
        r = orc.alm2map(a_k[3], nside, lmax) - tk
        gk = orc.alm2map_adjoint(2 * r, nside, lmax)
        for _ in range(3):
            gk = gk - orc.alm2map_adjoint(orc.map2alm_adjoint(gk, nside, lmax), nside, lmax)
        # the gradient chains 14 FP64 transforms (three refinement steps
        # forward and back, the final synthesis and its adjoint), each held
        # to 1e-10: their rounding adds up, so the chain is held to 2e-9
        assert np.max(np.abs(got[k:k + 1] - gk)) <= 2e-9 * np.abs(gk).max()
