"""Non-stationary velocity (one band-limited velocity per time step) through the
C-ABI against the FP64 oracle.  Tolerances (relative L2) as for the stationary
path: FP32 1e-5 on the energy, 1e-4 on the gradient, the HVP and the PCG
iterates; mixed 5e-5 / 5e-4.  Also: a velocity constant in time reproduces the
stationary plan, per-step body forces from blr_adjoint, checkpointed runs
bit-identical to unchecked ones, the incompressible form per step, and a
registration against the oracle's."""

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
    "ragged": dict(n=(40, 36, 52), band=(8, 6, 10), nt=5, seed=171, bound=13.0),
    "64cube": dict(n=(64, 64, 64), band=(16, 16, 16), nt=10, seed=181, bound=40.0),
}


@pytest.fixture(scope="module")
def blr():
    from paper_1807_05117_gb300 import blr as _blr
    return _blr


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _steps(band, nt, seed, bound):
    """Per-step coefficients (nt, 3, B1, B2, B3) with seeds seed .. seed + nt - 1."""
    return np.stack([synth.random_coefficients(band, seed + n, bound=bound) for n in range(nt)])


def _dirs(band, nt, seed):
    return np.stack([synth.random_direction(band, seed + n) for n in range(nt)])


@pytest.fixture(scope="module",
                params=[(c, pr) for c in sorted(CASES) for pr in ("fp32", "mixed")],
                ids=lambda t: f"{t[0]}-{t[1]}")
def case(request, blr):
    name, precision = request.param
    c = CASES[name]
    n, band, nt = c["n"], c["band"], c["nt"]
    I0, I1, _ = synth.blob_pair(n, c["seed"], max_disp=2.0)
    vt = _steps(band, nt, c["seed"] + 100, c["bound"])
    dvt = _dirs(band, nt, c["seed"] + 200)
    (I0f, I0d), (I1f, I1d), (vtf, vtd), (dvf, dvd) = synth.as_device_inputs(I0, I1, vt, dvt)
    p = O.Params(n=n, band=band, nt=nt, stationary=False)
    plan = blr.Plan(n, band, nt, nonstationary=True,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(_dev(I0f), _dev(I1f))
    pt = O.Point(vtd, I0d, I1d, p)
    return dict(plan=plan, pt=pt, vtf=vtf, dvf=dvf, dvd=dvd, band=band, nt=nt,
                tol=TOL[precision])


def _coefs(band, nt):
    return torch.zeros((nt, 3) + tuple(band), dtype=torch.complex64, device="cuda")


def test_gradient_and_hessvec_parity(case):
    plan, pt, tol = case["plan"], case["pt"], case["tol"]
    g, h = _coefs(case["band"], case["nt"]), _coefs(case["band"], case["nt"])
    e = torch.zeros(3, dtype=torch.float64, device="cuda")
    plan.gradient(_dev(case["vtf"]), g, e)
    plan.hessvec(_dev(case["dvf"]), h)
    assert plan.status() == 0
    assert abs(float(e[0]) - pt.energy) <= tol["field"] * pt.energy
    assert abs(float(e[1]) - pt.energy_reg) <= 1e-5 * pt.energy_reg
    assert rel(g.cpu().numpy(), pt.gradient()[0]) <= tol["grad"]
    assert rel(h.cpu().numpy(), pt.gn_hessvec(case["dvd"])[0]) <= tol["grad"]


def test_pcg_iterates_parity(case):
    plan, pt = case["plan"], case["pt"]
    g = _coefs(case["band"], case["nt"])
    plan.gradient(_dev(case["vtf"]), g)
    x = _coefs(case["band"], case["nt"])
    its, _ = plan.pcg(-g, x, 4, 0.0)
    rhs = (-g).cpu().numpy().astype(np.complex128)
    x_ref, its_ref, _ = O.pcg(lambda v: pt.gn_hessvec(v)[0], rhs, 1.0 / pt.A[None], 0.0, 4)
    assert its == its_ref == 4
    assert rel(x.cpu().numpy(), x_ref) <= case["tol"]["grad"]


def test_constant_in_time_matches_stationary_plan(blr):
    """v~^n = v~ for every step: the energies agree, the per-step gradients and
    HVPs sum to the stationary plan's, and the per-step body forces of
    blr_adjoint sum to the stationary body force."""
    n, band, nt = (24, 20, 36), (6, 4, 8), 4
    I0, I1, _ = synth.blob_pair(n, 191, max_disp=2.0)
    vt = synth.random_coefficients(band, 192, bound=6.0)
    dvt = synth.random_direction(band, 193)
    (I0f, _), (I1f, _), (vtf, _), (dvf, _) = synth.as_device_inputs(I0, I1, vt, dvt)
    st = blr.Plan(n, band, nt)
    ns = blr.Plan(n, band, nt, nonstationary=True)
    for pl in (st, ns):
        pl.set_images(_dev(I0f), _dev(I1f))
    g1 = torch.zeros((3,) + band, dtype=torch.complex64, device="cuda")
    h1 = torch.zeros_like(g1)
    e1 = torch.zeros(3, dtype=torch.float64, device="cuda")
    st.gradient(_dev(vtf), g1, e1)
    st.hessvec(_dev(dvf), h1)
    g2, h2 = _coefs(band, nt), _coefs(band, nt)
    e2 = torch.zeros(3, dtype=torch.float64, device="cuda")
    ns.gradient(_dev(np.stack([vtf] * nt)), g2, e2)
    ns.hessvec(_dev(np.stack([dvf] * nt)), h2)
    assert abs(float(e1[0]) - float(e2[0])) <= 1e-6 * float(e1[0])
    assert rel(g2.sum(dim=0).cpu().numpy(), g1.cpu().numpy()) <= 1e-5
    assert rel(h2.sum(dim=0).cpu().numpy(), h1.cpu().numpy()) <= 1e-5
    b1 = torch.zeros((3,) + n, dtype=torch.float32, device="cuda")
    b2 = torch.zeros((nt, 3) + n, dtype=torch.float32, device="cuda")
    st.adjoint(b1)
    ns.adjoint(b2)
    assert rel(b2.sum(dim=0).cpu().numpy(), b1.cpu().numpy()) <= 1e-5


def test_checkpointed_bit_identical_and_incompressible(blr):
    n, band, nt = (24, 20, 36), (6, 4, 8), 5
    I0, I1, _ = synth.blob_pair(n, 195, max_disp=2.0)
    vt = _steps(band, nt, 196, 6.0)
    dvt = _dirs(band, nt, 206)
    (I0f, I0d), (I1f, I1d), (vtf, vtd), (dvf, dvd) = synth.as_device_inputs(I0, I1, vt, dvt)
    out = []
    for ck in (0, 2):
        pl = blr.Plan(n, band, nt, nonstationary=True, ckpt_every=ck)
        pl.set_images(_dev(I0f), _dev(I1f))
        g, h = _coefs(band, nt), _coefs(band, nt)
        pl.gradient(_dev(vtf), g)
        pl.hessvec(_dev(dvf), h)
        out.append((g, h))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    # incompressible form, per step, H^1 regulariser
    p = O.Params(n=n, band=band, nt=nt, stationary=False, incompressible=True, s=0.5)
    pl = blr.Plan(n, band, nt, nonstationary=True, incompressible=True, s=0.5)
    pl.set_images(_dev(I0f), _dev(I1f))
    g, h = _coefs(band, nt), _coefs(band, nt)
    pl.gradient(_dev(vtf), g)
    pl.hessvec(_dev(dvf), h)
    pt = O.Point(vtd, I0d, I1d, p)
    assert rel(g.cpu().numpy(), pt.gradient()[0]) <= 1e-4
    assert rel(h.cpu().numpy(), pt.gn_hessvec(dvd)[0]) <= 1e-4


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_nonstationary_registration_matches_oracle(blr, precision):
    n, band, nt = (32, 32, 32), (8, 8, 8), 10
    I0, I1, _ = synth.blob_pair(n, 1301, max_disp=2.0)
    (I0f, I0d), (I1f, I1d) = synth.as_device_inputs(I0, I1)
    plan = blr.Plan(n, band, nt, nonstationary=True,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(_dev(I0f), _dev(I1f))
    vt = _coefs(band, nt)
    rep = plan.newton(vt, 5, 10, 1e-6)
    ref = O.newton(np.zeros((nt, 3) + band, complex), I0d, I1d,
                   O.Params(n, band, nt, stationary=False), max_newton=5, max_pcg=10, gtol=1e-6)
    assert rep.status == blr.BLR_OK
    assert rep.newton_iters == ref.iterations
    assert abs(rep.energy0 - ref.energies[0]) <= 1e-5 * ref.energies[0]
    assert abs(rep.energy - ref.energies[-1]) <= 1e-3 * ref.energies[-1]
    assert abs(rep.pcg_iters - sum(ref.pcg_iterations)) <= ref.iterations
    assert rep.energy < 0.5 * rep.energy0
