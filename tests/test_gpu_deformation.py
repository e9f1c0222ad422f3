"""Deformation-state-equation variant (Section 2.3, Eqs. 16-18) through the C-ABI
against the FP64 oracle.  Tolerances (relative L2) as for the image variant:
FP32 1e-5 on m(1) and the energy, 1e-4 on the gradient, the Gauss-Newton HVP and
the PCG iterates; mixed 5e-5 / 5e-4.  Also: the body force of blr_adjoint
(FP32 1e-5; mixed: a bound from the oracle's response to perturbations of the
displacement, see body_force_bound), the full Newton Hessian of the variant,
gradient_at_state repeating bit-exactly after an HVP, the incompressible form,
and a registration against the oracle's."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import blr_oracle as O  # noqa: E402
from paper_1807_05117_gb300 import synth  # noqa: E402


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


TOL = {"fp32": dict(field=1e-5, grad=1e-4), "mixed": dict(field=5e-5, grad=5e-4)}

CASES = {
    "ragged": dict(n=(40, 36, 52), band=(8, 6, 10), nt=5, seed=211, bound=13.0),
    "64cube": dict(n=(64, 64, 64), band=(16, 16, 16), nt=10, seed=321, bound=40.0),
    "nt1": dict(n=(16, 12, 20), band=(4, 4, 4), nt=1, seed=231, bound=2.0),
}


def body_force_bound(pt, vtd, I0d, I1d, p, precision, b_ref):
    """Relative L2 bound for the body force b of blr_adjoint.

    b responds to the displacement d about one to one (a relative change of d
    moves b by about as much), and it jumps where a point x + u^nt of the final
    warp crosses a cell face, since the trilinear gradient of I0 changes there;
    both cell choices are valid discretisations.  The FP32 path's d differs from
    the oracle's by FP32 rounding, so the field bound 1e-5 holds.  The mixed
    path's d carries the BF16 hi+lo DFT error (the expand bound, 5e-5), so its
    bound is the field bound plus twice the oracle's own largest response to two
    random relative changes of d of that size."""
    if precision == "fp32":
        return TOL["fp32"]["field"]
    rng = np.random.default_rng(12345)
    spread = 0.0
    for _ in range(2):
        fac = 1.0 + 5e-5 * rng.standard_normal(size=(3,) + tuple(p.n))
        _, b = O.DeformationPoint(vtd, I0d, I1d, p, displacement_factor=fac).gradient()
        spread = max(spread, rel(b, b_ref))
    return TOL["mixed"]["field"] + 2.0 * spread


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
    p = O.Params(n=n, band=band, nt=nt, state="deformation")
    plan = blr.Plan(n, band, nt, state_equation=blr.BLR_STATE_DEFORMATION,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(_dev(I0f), _dev(I1f))
    pt = O.DeformationPoint(vtd, I0d, I1d, p)
    b_tol = body_force_bound(pt, vtd, I0d, I1d, p, precision, pt.gradient()[1])
    return dict(plan=plan, pt=pt, vtf=vtf, dvf=dvf, dvd=dvd, n=n, band=band,
                tol=TOL[precision], b_tol=b_tol)


def test_state_gradient_and_hessvec_parity(case, blr):
    plan, pt, tol = case["plan"], case["pt"], case["tol"]
    m1 = torch.zeros(case["n"], dtype=torch.float32, device="cuda")
    e = torch.zeros(3, dtype=torch.float64, device="cuda")
    plan.state(_dev(case["vtf"]), m1, e)
    assert plan.status() == blr.BLR_OK
    assert rel(m1.cpu().numpy(), pt.m1) <= tol["field"]
    assert abs(float(e[0]) - pt.energy) <= tol["field"] * pt.energy
    b = torch.zeros((3,) + case["n"], dtype=torch.float32, device="cuda")
    plan.adjoint(b)
    _, b_ref = pt.gradient()
    assert rel(b.cpu().numpy(), b_ref) <= case["b_tol"], case["b_tol"]
    g, h = _coef(case["band"]), _coef(case["band"])
    plan.gradient(_dev(case["vtf"]), g)
    plan.hessvec(_dev(case["dvf"]), h)
    assert rel(g.cpu().numpy(), pt.gradient()[0]) <= tol["grad"]
    assert rel(h.cpu().numpy(), pt.gn_hessvec(case["dvd"])[0]) <= tol["grad"]


def test_pcg_iterates_parity(case):
    plan, pt = case["plan"], case["pt"]
    g = _coef(case["band"])
    plan.gradient(_dev(case["vtf"]), g)
    x = _coef(case["band"])
    its, _ = plan.pcg(-g, x, 4, 0.0)
    rhs = (-g).cpu().numpy().astype(np.complex128)
    x_ref, its_ref, _ = O.pcg(lambda v: pt.gn_hessvec(v)[0], rhs, 1.0 / pt.A[None], 0.0, 4)
    assert its == its_ref == 4
    assert rel(x.cpu().numpy(), x_ref) <= case["tol"]["grad"]


def test_sweep_forms_are_bit_identical(case, blr):
    """Kept state gradients grad u^n_c (read by the adjoint and incremental sweeps)
    against interpolated ones, the gather and march incremental forms, and the
    split adjoint solve (transport steps, then one body-force pass) against the
    per-step one: gradient, Gauss-Newton HVP and blr_adjoint's body force equal
    bit for bit."""
    plan = case["plan"]
    tun = plan.tuning()
    assert tun["grad_kept"] == 1
    splits = (0, 1) if plan.nt > 1 else (0,)
    out = {}
    try:
        for split in splits:
            for useg in (0, 1):
                for inc in (0, 2):
                    plan.set_tuning(adjoint_split=split, adjoint_reads_grad=useg,
                                    incremental_form=inc, adjoint_two_step=0)
                    g, h = _coef(case["band"]), _coef(case["band"])
                    plan.gradient(_dev(case["vtf"]), g)
                    plan.hessvec(_dev(case["dvf"]), h)
                    b = torch.zeros((3,) + case["n"], dtype=torch.float32, device="cuda")
                    plan.adjoint(b)
                    out[(split, useg, inc)] = (g, h, b)
    finally:
        plan.set_tuning(**{k: tun[k] for k in ("adjoint_split", "adjoint_reads_grad",
                                               "incremental_form", "adjoint_two_step")})
    assert plan.status() == blr.BLR_OK
    ref = out[(0, 0, 0)]
    for key, res in out.items():
        for a, r in zip(res, ref):
            assert torch.equal(a, r), key


def test_gradient_repeats_after_hessvec_and_adjoint_arguments(blr):
    n, band, nt = (24, 20, 36), (6, 4, 8), 4
    I0, I1, _ = synth.blob_pair(n, 241, max_disp=2.0)
    vt = synth.random_coefficients(band, 242, bound=6.0)
    dvt = synth.random_direction(band, 243)
    (I0f, _), (I1f, _), (vtf, _), (dvf, _) = synth.as_device_inputs(I0, I1, vt, dvt)
    plan = blr.Plan(n, band, nt, state_equation=blr.BLR_STATE_DEFORMATION)
    plan.set_images(_dev(I0f), _dev(I1f))
    g1, g2, g3 = _coef(band), _coef(band), _coef(band)
    plan.gradient(_dev(vtf), g1)
    plan.gradient_at_state(g2)
    plan.hessvec(_dev(dvf), _coef(band))
    plan.gradient_at_state(g3)
    assert torch.equal(g1, g2) and torch.equal(g1, g3)
    b = torch.zeros((3,) + n, dtype=torch.float32, device="cuda")
    lam0 = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(blr.BlrError) as ei:
        plan.adjoint(b, lam0)
    assert ei.value.code == blr.BLR_EINVAL


def test_incompressible_deformation_parity(blr):
    n, band, nt = (40, 36, 52), (8, 6, 10), 5
    I0, I1, _ = synth.blob_pair(n, 251, max_disp=2.0)
    vt = synth.random_coefficients(band, 252, bound=13.0)
    dvt = synth.random_direction(band, 253)
    (I0f, I0d), (I1f, I1d), (vtf, vtd), (dvf, dvd) = synth.as_device_inputs(I0, I1, vt, dvt)
    p = O.Params(n=n, band=band, nt=nt, s=0.5, incompressible=True, state="deformation")
    plan = blr.Plan(n, band, nt, s=0.5, incompressible=True,
                    state_equation=blr.BLR_STATE_DEFORMATION)
    plan.set_images(_dev(I0f), _dev(I1f))
    g, h = _coef(band), _coef(band)
    plan.gradient(_dev(vtf), g)
    plan.hessvec(_dev(dvf), h)
    pt = O.DeformationPoint(vtd, I0d, I1d, p)
    assert rel(g.cpu().numpy(), pt.gradient()[0]) <= 1e-4
    assert rel(h.cpu().numpy(), pt.gn_hessvec(dvd)[0]) <= 1e-4


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_deformation_registration_matches_oracle(blr, precision):
    n, band, nt = (32, 32, 32), (8, 8, 8), 10
    I0, I1, _ = synth.blob_pair(n, 1401, max_disp=2.0)
    (I0f, I0d), (I1f, I1d) = synth.as_device_inputs(I0, I1)
    plan = blr.Plan(n, band, nt, state_equation=blr.BLR_STATE_DEFORMATION,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(_dev(I0f), _dev(I1f))
    vt = _coef(band)
    rep = plan.newton(vt, 5, 10, 1e-6)
    ref = O.newton(np.zeros((3,) + band, complex), I0d, I1d,
                   O.Params(n, band, nt, state="deformation"), max_newton=5, max_pcg=10,
                   gtol=1e-6)
    assert rep.status == blr.BLR_OK
    assert rep.newton_iters == ref.iterations
    assert abs(rep.energy0 - ref.energies[0]) <= 1e-5 * ref.energies[0]
    assert abs(rep.energy - ref.energies[-1]) <= 1e-3 * ref.energies[-1]
    assert abs(rep.pcg_iters - sum(ref.pcg_iterations)) <= ref.iterations
    assert rep.energy < 0.5 * rep.energy0


# --- the full Newton Hessian of this variant (Eqs. 19-21 without the drops of
# Section 3.4): sigma = 0.5, where the dropped terms change the product by 6 % to
# 45 %, far more than the tolerances -------------------------------------------


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_full_newton_hessvec_parity(blr, name, precision):
    c = CASES[name]
    n, band, nt = c["n"], c["band"], c["nt"]
    I0, I1, _ = synth.blob_pair(n, c["seed"], max_disp=2.0)
    vt = synth.random_coefficients(band, c["seed"] + 1, bound=c["bound"])
    dvt = synth.random_direction(band, c["seed"] + 2)
    (I0f, I0d), (I1f, I1d), (vtf, vtd), (dvf, dvd) = synth.as_device_inputs(I0, I1, vt, dvt)
    p = O.Params(n=n, band=band, nt=nt, sigma=0.5, state="deformation")
    pt = O.DeformationPoint(vtd, I0d, I1d, p)
    h_ref = pt.full_hessvec(dvd)[0]
    tol = TOL[precision]["grad"]
    assert rel(pt.gn_hessvec(dvd)[0], h_ref) > 10 * tol   # the full terms matter here
    plan = blr.Plan(n, band, nt, sigma=0.5, state_equation=blr.BLR_STATE_DEFORMATION,
                    hessian=blr.BLR_NEWTON,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(_dev(I0f), _dev(I1f))
    g, h = _coef(band), _coef(band)
    plan.gradient(_dev(vtf), g)
    plan.hessvec(_dev(dvf), h)
    assert plan.status() == blr.BLR_OK
    assert rel(g.cpu().numpy(), pt.gradient()[0]) <= tol
    assert rel(h.cpu().numpy(), h_ref) <= tol
    # after a forward solve alone the product computes the adjoint states itself,
    # bit for bit the same; the gradient at the state repeats after the product
    h2, g2 = _coef(band), _coef(band)
    plan.state(_dev(vtf))
    plan.hessvec(_dev(dvf), h2)
    plan.gradient_at_state(g2)
    assert torch.equal(h, h2) and torch.equal(g, g2)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_full_newton_deformation_registration_matches_oracle(blr, precision):
    """5 Newton updates (truncated PCG, <= 10 iterations) from zero on the 32^3 blob
    pair: Newton counts equal, final energy within 1e-3, PCG totals within +-1
    per update."""
    n, band, nt = (32, 32, 32), (8, 8, 8), 10
    I0, I1, _ = synth.blob_pair(n, 1411, max_disp=2.0)
    (I0f, I0d), (I1f, I1d) = synth.as_device_inputs(I0, I1)
    plan = blr.Plan(n, band, nt, state_equation=blr.BLR_STATE_DEFORMATION,
                    hessian=blr.BLR_NEWTON,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(_dev(I0f), _dev(I1f))
    vt = _coef(band)
    rep = plan.newton(vt, 5, 10, 1e-6)
    ref = O.newton(np.zeros((3,) + band, complex), I0d, I1d,
                   O.Params(n, band, nt, state="deformation"), max_newton=5, max_pcg=10,
                   gtol=1e-6, hessian="full")
    assert rep.status == blr.BLR_OK
    assert rep.newton_iters == ref.iterations
    assert abs(rep.energy0 - ref.energies[0]) <= 1e-5 * ref.energies[0]
    assert abs(rep.energy - ref.energies[-1]) <= 1e-3 * ref.energies[-1]
    assert abs(rep.pcg_iters - sum(ref.pcg_iterations)) <= ref.iterations
    assert rep.energy < 0.5 * rep.energy0
