"""Incompressible form (Eq. 4 with gamma = 1, imposed in the band by the Leray
projector) through the C-ABI against the FP64 oracle, with the H^1 regulariser
(s = 1/2).  Tolerances (relative L2) as for the compressible path: FP32 1e-5 on
the energy, 1e-4 on the gradient, the HVP and the PCG iterates; mixed 5e-5 / 5e-4.
The outputs must also lie in the divergence-free subspace (P x = x to FP32
rounding), and a registration's final energy must match within 1e-3."""

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


TOL = {"fp32": dict(field=1e-5, grad=1e-4), "mixed": dict(field=5e-5, grad=5e-4)}

CASES = {
    # several sweep tiles with ragged tails on every axis, anisotropic band
    "ragged": dict(n=(40, 36, 52), band=(8, 6, 10), nt=5, seed=111, bound=13.0),
    "64cube": dict(n=(64, 64, 64), band=(16, 16, 16), nt=10, seed=121, bound=40.0),
}


@pytest.fixture(scope="module")
def blr():
    from paper_1807_05117_gb300 import blr as _blr
    return _blr


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
    p = O.Params(n=n, band=band, nt=nt, s=0.5, incompressible=True)
    plan = blr.Plan(n, band, nt, s=0.5, incompressible=True,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()   # noqa: E731
    plan.set_images(dev(I0f), dev(I1f))
    pt = O.Point(vtd, I0d, I1d, p)
    return dict(plan=plan, p=p, pt=pt, vtf=vtf, dvf=dvf, dvd=dvd, dev=dev, band=band,
                tol=TOL[precision])


def _coef(band):
    return torch.zeros((3,) + tuple(band), dtype=torch.complex64, device="cuda")


def test_gradient_and_hessvec_parity(case):
    g, h = _coef(case["band"]), _coef(case["band"])
    e = torch.zeros(3, dtype=torch.float64, device="cuda")
    case["plan"].gradient(case["dev"](case["vtf"]), g, e)
    case["plan"].hessvec(case["dev"](case["dvf"]), h)
    assert case["plan"].status() == 0
    pt, tol = case["pt"], case["tol"]
    assert abs(float(e[0]) - pt.energy) <= tol["field"] * pt.energy
    assert abs(float(e[1]) - pt.energy_reg) <= 1e-5 * pt.energy_reg
    g_ref = pt.gradient()[0]
    h_ref = pt.gn_hessvec(case["dvd"])[0]
    gn, hn = g.cpu().numpy(), h.cpu().numpy()
    assert rel(gn, g_ref) <= tol["grad"]
    assert rel(hn, h_ref) <= tol["grad"]
    # outputs are divergence-free band fields
    n = case["p"].n
    assert rel(O.leray(gn.astype(np.complex128), n), gn) <= 1e-6
    assert rel(O.leray(hn.astype(np.complex128), n), hn) <= 1e-6


def test_pcg_iterates_parity(case):
    g = _coef(case["band"])
    case["plan"].gradient(case["dev"](case["vtf"]), g)
    x = _coef(case["band"])
    its, relres = case["plan"].pcg(-g, x, 4, 0.0)
    pt = case["pt"]
    rhs = (-g).cpu().numpy().astype(np.complex128)
    x_ref, its_ref, rel_ref = O.pcg(lambda v: pt.gn_hessvec(v)[0], rhs, 1.0 / pt.A[None], 0.0, 4)
    assert its == its_ref == 4
    assert rel(x.cpu().numpy(), x_ref) <= case["tol"]["grad"]


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_incompressible_registration_matches_oracle(blr, precision):
    n, band, nt = (32, 32, 32), (8, 8, 8), 10
    I0, I1, _ = synth.blob_pair(n, 1101, max_disp=2.0)
    (I0f, I0d), (I1f, I1d) = synth.as_device_inputs(I0, I1)
    plan = blr.Plan(n, band, nt, s=0.5, incompressible=True,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(torch.from_numpy(I0f).cuda(), torch.from_numpy(I1f).cuda())
    vt = torch.zeros((3,) + band, dtype=torch.complex64, device="cuda")
    rep = plan.newton(vt, 5, 10, 1e-6)
    p = O.Params(n, band, nt, s=0.5, incompressible=True)
    ref = O.newton(np.zeros((3,) + band, complex), I0d, I1d, p, max_newton=5, max_pcg=10,
                   gtol=1e-6)
    assert rep.status == blr.BLR_OK
    assert rep.newton_iters == ref.iterations
    assert abs(rep.energy0 - ref.energies[0]) <= 1e-5 * ref.energies[0]
    assert abs(rep.energy - ref.energies[-1]) <= 1e-3 * ref.energies[-1]
    assert abs(rep.pcg_iters - sum(ref.pcg_iterations)) <= ref.iterations
    assert rep.energy < rep.energy0
    v = vt.cpu().numpy().astype(np.complex128)
    assert rel(O.leray(v, n), v) <= 1e-5
