"""Full Newton Hessian (Eqs. 44-46 without the drops of Section 3.4) through the
C-ABI against the FP64 oracle.  Tolerances (relative L2) as for the
Gauss-Newton path: FP32 1e-4, mixed 5e-4 on the Hessian-vector product; the
cases use sigma = 0.5 so that the terms the Gauss-Newton step drops change the
product by far more than the tolerance.  Also: the adjoint states are kept per
point (gradient_at_state and blr_adjoint repeat bit-exactly after a
Hessian-vector product), truncated PCG on an indefinite Hessian, and a full
Newton registration against the oracle's."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import blr_oracle as O  # noqa: E402
from paper_1807_05117_gb300 import synth  # noqa: E402


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


TOL = {"fp32": 1e-4, "mixed": 5e-4}

CASES = {
    "ragged": dict(n=(40, 36, 52), band=(8, 6, 10), nt=5, seed=131, bound=13.0),
    "64cube": dict(n=(64, 64, 64), band=(16, 16, 16), nt=10, seed=141, bound=40.0),
    "nt1": dict(n=(16, 12, 20), band=(4, 4, 4), nt=1, seed=151, bound=2.0),
}


@pytest.fixture(scope="module")
def blr():
    from paper_1807_05117_gb300 import blr as _blr
    return _blr


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _coef(band):
    return torch.zeros((3,) + tuple(band), dtype=torch.complex64, device="cuda")


@pytest.fixture(scope="module",
                params=[(c, pr) for c in sorted(CASES) for pr in ("fp32", "mixed")],
                ids=lambda t: f"{t[0]}-{t[1]}")
def case(request, blr):
    name, precision = request.param
    c = CASES[name]
    n, band, nt = c["n"], c["band"], c["nt"]
    I0, I1, _ = synth.blob_pair(n, c["seed"], max_disp=2.0)
    vt = synth.random_coefficients(band, c["seed"] + 1, bound=c["bound"])
    dvt = synth.random_direction(band, c["seed"] + 2)
    (I0f, I0d), (I1f, I1d), (vtf, vtd), (dvf, dvd) = synth.as_device_inputs(I0, I1, vt, dvt)
    p = O.Params(n=n, band=band, nt=nt, sigma=0.5)
    plan = blr.Plan(n, band, nt, sigma=0.5, hessian=blr.BLR_NEWTON,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(_dev(I0f), _dev(I1f))
    pt = O.Point(vtd, I0d, I1d, p)
    return dict(plan=plan, pt=pt, vtf=vtf, dvf=dvf, dvd=dvd, band=band, tol=TOL[precision])


def test_full_hessvec_parity(case, blr):
    plan, pt = case["plan"], case["pt"]
    g, h = _coef(case["band"]), _coef(case["band"])
    plan.gradient(_dev(case["vtf"]), g)
    plan.hessvec(_dev(case["dvf"]), h)
    assert plan.status() == blr.BLR_OK
    h_ref = pt.full_hessvec(case["dvd"])[0]
    h_gn = pt.gn_hessvec(case["dvd"])[0]
    assert rel(h_gn, h_ref) > 10 * case["tol"]        # the full terms matter here
    assert rel(h.cpu().numpy(), h_ref) <= case["tol"]
    assert rel(g.cpu().numpy(), pt.gradient()[0]) <= case["tol"]


def test_full_hessvec_after_state_only_and_deterministic(case):
    """Without a gradient call the product computes the adjoint states itself;
    the result is bit-identical to the one after blr_gradient."""
    plan = case["plan"]
    h1, h2, h3 = (_coef(case["band"]) for _ in range(3))
    plan.state(_dev(case["vtf"]))
    plan.hessvec(_dev(case["dvf"]), h1)
    plan.hessvec(_dev(case["dvf"]), h2)
    plan.gradient(_dev(case["vtf"]), _coef(case["band"]))
    plan.hessvec(_dev(case["dvf"]), h3)
    assert torch.equal(h1, h2) and torch.equal(h1, h3)


@pytest.mark.parametrize("hessian", ["gn", "full"])
def test_adjoint_repeats_after_hessvec(blr, hessian):
    """lambda^nt of the current point is kept apart from the HVP's buffers:
    gradient_at_state and blr_adjoint give bit-identical results when repeated
    and after a Hessian-vector product."""
    n, band, nt = (24, 20, 36), (6, 4, 8), 4
    I0, I1, _ = synth.blob_pair(n, 161, max_disp=2.0)
    vt = synth.random_coefficients(band, 162, bound=6.0)
    dvt = synth.random_direction(band, 163)
    (I0f, _), (I1f, _), (vtf, _), (dvf, _) = synth.as_device_inputs(I0, I1, vt, dvt)
    plan = blr.Plan(n, band, nt, hessian=blr.BLR_NEWTON if hessian == "full"
                    else blr.BLR_GAUSS_NEWTON)
    plan.set_images(_dev(I0f), _dev(I1f))
    g1, g2, g3 = (_coef(band) for _ in range(3))
    plan.gradient(_dev(vtf), g1)
    plan.gradient_at_state(g2)
    plan.hessvec(_dev(dvf), _coef(band))
    plan.gradient_at_state(g3)
    assert torch.equal(g1, g2) and torch.equal(g1, g3)
    b1 = torch.zeros((3,) + n, dtype=torch.float32, device="cuda")
    b2 = torch.zeros_like(b1)
    plan.adjoint(b1)
    plan.hessvec(_dev(dvf), _coef(band))
    plan.adjoint(b2)
    assert torch.equal(b1, b2)


def test_truncated_pcg_on_indefinite_hessian(blr):
    """Weak regulariser (alpha = 0, gamma = 0.1, s = 1): the full Hessian is
    indefinite here.  blr_pcg reports the non-positive curvature near the
    iteration where the oracle meets it, and a Newton step (truncated PCG) is
    accepted with a lower energy, as in the oracle."""
    n, band, nt = (12, 12, 12), (4, 4, 4), 5
    I0, I1, _ = synth.blob_pair(n, 51, max_disp=2.0)
    vt = synth.random_coefficients(band, 52, bound=2.0)
    (I0f, I0d), (I1f, I1d), (vtf, vtd) = synth.as_device_inputs(I0, I1, vt)
    p = O.Params(n=n, band=band, nt=nt, alpha=0.0, gamma=0.1, s=1)
    pt = O.Point(vtd, I0d, I1d, p)
    g_ref = pt.gradient()[0]
    with pytest.raises(O.NegativeCurvature):
        O.pcg(lambda v: pt.full_hessvec(v)[0], -g_ref, 1.0 / pt.A[None], 1e-10, 60)
    _, its_ref, _ = O.pcg(lambda v: pt.full_hessvec(v)[0], -g_ref, 1.0 / pt.A[None], 1e-10, 60,
                          truncate=True)
    plan = blr.Plan(n, band, nt, alpha=0.0, gamma=0.1, s=1, hessian=blr.BLR_NEWTON)
    plan.set_images(_dev(I0f), _dev(I1f))
    g = _coef(band)
    plan.gradient(_dev(vtf), g)
    assert rel(g.cpu().numpy(), g_ref) <= 1e-4
    x = _coef(band)
    with pytest.raises(blr.BlrError) as ei:
        plan.pcg(-g, x, 60, 1e-10)
    assert ei.value.code == blr.BLR_ECURV
    v = _dev(vtf)
    rep = plan.newton(v, 1, 60, 0.0, 1e-10)
    ref = O.newton(vtd, I0d, I1d, p, max_newton=1, max_pcg=60, gtol=0.0, forcing=1e-10,
                   hessian="full")
    assert rep.status == blr.BLR_OK and rep.newton_iters == ref.iterations == 1
    assert abs(rep.pcg_iters - its_ref) <= 1
    assert rep.energy < rep.energy0
    assert abs(rep.energy - ref.energies[-1]) <= 1e-3 * ref.energies[-1]


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_full_newton_registration_matches_oracle(blr, precision):
    n, band, nt = (32, 32, 32), (8, 8, 8), 10
    I0, I1, _ = synth.blob_pair(n, 1201, max_disp=2.0)
    (I0f, I0d), (I1f, I1d) = synth.as_device_inputs(I0, I1)
    plan = blr.Plan(n, band, nt, hessian=blr.BLR_NEWTON,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(_dev(I0f), _dev(I1f))
    vt = torch.zeros((3,) + band, dtype=torch.complex64, device="cuda")
    rep = plan.newton(vt, 5, 10, 1e-6)
    ref = O.newton(np.zeros((3,) + band, complex), I0d, I1d, O.Params(n, band, nt),
                   max_newton=5, max_pcg=10, gtol=1e-6, hessian="full")
    assert rep.status == blr.BLR_OK
    assert rep.newton_iters == ref.iterations
    assert abs(rep.energy0 - ref.energies[0]) <= 1e-5 * ref.energies[0]
    assert abs(rep.energy - ref.energies[-1]) <= 1e-3 * ref.energies[-1]
    assert abs(rep.pcg_iters - sum(ref.pcg_iterations)) <= ref.iterations
    assert rep.energy < 0.5 * rep.energy0
