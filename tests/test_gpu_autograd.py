"""Differentiation form: the registration energy as a torch.autograd.Function
whose backward is the library's adjoint kernel chain, with the state kept only
every 4 of 20 time steps and recomputed segment by segment in the backward.

Checked on a 64^3 phantom pair (band 32^3, 20 steps) against the FP64 oracle's
gradient, against FP64 central finite differences of the oracle energy (step
1e-4, 32 random smooth directions), the Gauss-Newton HVP against central
differences of the FP64 gradient at zero residual, and checkpointed against
non-checkpointed runs bit for bit at 64^3 and at the full 256^3 size."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import blr_oracle as O  # noqa: E402
from paper_1807_05117_gb300 import synth  # noqa: E402

N64, BAND, NT, CK = (64, 64, 64), (32, 32, 32), 20, 4


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def mods():
    from paper_1807_05117_gb300 import blr
    from paper_1807_05117_gb300.autograd import registration_energy
    return blr, registration_energy


@pytest.fixture(scope="module")
def inst():
    I0, I1, _ = synth.phantom_pair(N64, 5001, max_disp=4.0)
    vt = synth.random_coefficients(BAND, 5002, 160.0)      # about 0.4 voxel per step
    (I0f, I0d), (I1f, I1d), (vtf, vtd) = synth.as_device_inputs(I0, I1, vt)
    return dict(I0f=I0f, I1f=I1f, I0d=I0d, I1d=I1d, vtf=vtf, vtd=vtd,
                p=O.Params(N64, BAND, NT))


def _plan(blr, n, I0f, I1f, ckpt):
    plan = blr.Plan(n, BAND, NT, ckpt_every=ckpt)
    plan.set_images(torch.from_numpy(I0f).cuda(), torch.from_numpy(I1f).cuda())
    return plan


def _grad(energy_fn, plan, vtf):
    vt = torch.from_numpy(vtf).cuda().requires_grad_(True)
    E = energy_fn(vt, plan)
    E.backward()
    return float(E.detach()), vt.grad.detach()


def test_energy_and_gradient_match_oracle(mods, inst):
    blr, energy_fn = mods
    plan = _plan(blr, N64, inst["I0f"], inst["I1f"], CK)
    E, g = _grad(energy_fn, plan, inst["vtf"])
    assert plan.status() == 0
    pt = O.Point(inst["vtd"], inst["I0d"], inst["I1d"], inst["p"])
    assert abs(E - pt.energy) <= 1e-5 * pt.energy
    assert rel(g.cpu().numpy(), pt.gradient()[0]) <= 1e-4


def test_gradient_matches_fp64_central_differences(mods, inst):
    blr, energy_fn = mods
    plan = _plan(blr, N64, inst["I0f"], inst["I1f"], CK)
    _, g = _grad(energy_fn, plan, inst["vtf"])
    g = g.cpu().numpy().astype(np.complex128)
    eps = 1e-4
    errs = []
    for s in range(32):
        dv = synth.random_coefficients(BAND, 6000 + s, 1.0)
        dv /= np.linalg.norm(dv)
        ep = O.energy(inst["vtd"] + eps * dv, inst["I0d"], inst["I1d"], inst["p"])
        em = O.energy(inst["vtd"] - eps * dv, inst["I0d"], inst["I1d"], inst["p"])
        fd = (ep - em) / (2 * eps)
        dd = O.inner(g, dv)
        errs.append(abs(fd - dd) / abs(fd))
    assert max(errs) <= 1e-3, errs


def test_gn_hessvec_matches_fp64_differences_of_the_gradient(mods, inst):
    """At zero residual the dropped Gauss-Newton terms vanish, so H_GN dv equals
    the central difference of the FP64 gradient."""
    blr, _ = mods
    I1z = O.Point(inst["vtd"], inst["I0d"], inst["I0d"], inst["p"]).m[-1]
    (I1zf, I1zd), = synth.as_device_inputs(I1z)
    plan = _plan(blr, N64, inst["I0f"], I1zf, CK)
    vt = torch.from_numpy(inst["vtf"]).cuda()
    plan.state(vt)
    eps = 1e-4
    for s in range(4):
        dv = synth.random_coefficients(BAND, 7000 + s, 1.0)
        dv /= np.linalg.norm(dv)
        (dvf, dvd), = synth.as_device_inputs(dv)
        h = torch.empty_like(vt)
        plan.hessvec(torch.from_numpy(dvf).cuda(), h)
        gp = O.Point(inst["vtd"] + eps * dvd, inst["I0d"], I1zd, inst["p"]).gradient()[0]
        gm = O.Point(inst["vtd"] - eps * dvd, inst["I0d"], I1zd, inst["p"]).gradient()[0]
        assert rel(h.cpu().numpy(), (gp - gm) / (2 * eps)) <= 1e-3


@pytest.mark.parametrize("n", [N64, (256, 256, 256)], ids=["64cube", "256cube"])
def test_checkpointing_is_bit_identical(mods, n):
    blr, energy_fn = mods
    I0, I1, _ = synth.phantom_pair(n, 5003, max_disp=8.0)
    vt = synth.random_coefficients(BAND, 5004, 160.0)      # same voxel displacement at any grid
    dv = synth.random_direction(BAND, 5005)
    (I0f, _), (I1f, _), (vtf, _), (dvf, _) = synth.as_device_inputs(I0, I1, vt, dv)
    out = []
    for ck in (0, CK):
        plan = _plan(blr, n, I0f, I1f, ck)
        E, g = _grad(energy_fn, plan, vtf)
        h = torch.empty_like(g)
        plan.hessvec(torch.from_numpy(dvf).cuda(), h)
        assert plan.status() == 0
        out.append((E, g, h))
        plan.close()
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2], out[1][2])


def test_backward_composes_and_survives_another_forward(mods, inst):
    blr, energy_fn = mods
    plan = _plan(blr, N64, inst["I0f"], inst["I1f"], CK)
    _, g_ref = _grad(energy_fn, plan, inst["vtf"])
    v1 = torch.from_numpy(inst["vtf"]).cuda().requires_grad_(True)
    v2 = (0.5 * torch.from_numpy(inst["vtf"]).cuda()).requires_grad_(True)
    E1 = energy_fn(v1, plan)
    E2 = energy_fn(v2, plan)          # moves the plan's current point
    loss = E1 + (v1.abs() ** 2).sum()
    loss.backward()
    assert torch.allclose(v1.grad, g_ref + 2 * v1.detach(), rtol=1e-6, atol=0)
    E2.backward()
    assert v2.grad is not None and torch.isfinite(v2.grad).all()
