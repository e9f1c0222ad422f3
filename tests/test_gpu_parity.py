"""CUDA path (through the C-ABI) against the FP64 oracle on identical seeded
inputs.  Tolerances (relative L2):
  FP32 path : 1e-5 on iota / pi, the state and the adjoint fields; 1e-4 on the
              gradient and the Gauss-Newton HVP; PCG iterates 1e-4;
  mixed path: (BF16 hi+lo split operands on tensor cores, FP32 accumulation in
              the axis-1 DFT stages; everything else FP32) 5e-5 on the fields,
              5e-4 on the gradient, the HVP and the PCG iterates;
a full registration's final energy within 1e-3 with PCG iteration counts within
+-1 per Newton step.  Cases: ragged tiles, a grid smaller than one tile, one
time step, two x2 tiles of the fused transforms, the 32^3 blob registration, the 128^3 phantom (band 32^3) and the
192x224x192 phantom with band 48^3 (gradient and HVP against the oracle in both
precisions; a 10-step registration mixed against FP32)."""

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


@pytest.fixture(scope="module")
def blr():
    from paper_1807_05117_gb300 import blr as _blr
    return _blr


TOL = {"fp32": dict(field=1e-5, grad=1e-4, pcg=1e-4),
       "mixed": dict(field=5e-5, grad=5e-4, pcg=5e-4)}


class Case:
    """Seeded inputs, rounded once to FP32 and given to both sides."""

    def __init__(self, blr, n, band, nt, seed, bound, sigma=1.0, pair="blob", max_disp=2.0,
                 precision="fp32"):
        n, band = tuple(n), tuple(band)
        if pair == "blob":
            I0, I1, _ = synth.blob_pair(n, seed, max_disp=max_disp)
        else:
            I0, I1, _ = synth.phantom_pair(n, seed, max_disp=max_disp)
        vt = synth.random_coefficients(band, seed + 1, bound=bound)
        dvt = synth.random_direction(band, seed + 2)
        (self.I0f, self.I0), (self.I1f, self.I1), (self.vtf, self.vt), (self.dvf, self.dv) = \
            synth.as_device_inputs(I0, I1, vt, dvt)
        self.p = O.Params(n=n, band=band, nt=nt, sigma=sigma)
        self.precision = precision
        self.tol = TOL[precision]
        self.plan = blr.Plan(n, band, nt, sigma=sigma,
                             precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
        self.dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        self.plan.set_images(self.dev(self.I0f), self.dev(self.I1f))
        self.n, self.band = n, band

    def coef(self):
        return torch.zeros((3,) + self.band, dtype=torch.complex64, device="cuda")

    def field(self, comps=3):
        shape = ((3,) if comps == 3 else ()) + self.n
        return torch.zeros(shape, dtype=torch.float32, device="cuda")


# Coefficient bounds are chosen so that the largest per-step displacement is
# 0.6-0.7 voxel (both cell choices and all 27 transpose neighbours are used).
CASES = {
    # spans several sweep tiles (32 x 8 x 8) on every axis with ragged tails
    "ragged": dict(n=(40, 36, 52), band=(8, 6, 10), nt=5, seed=101, bound=13.0),
    # grid smaller than one tile: the halo wraps more than once
    "tiny": dict(n=(3, 5, 7), band=(2, 2, 4), nt=3, seed=202, bound=3.0),
    # a single time step: first and last sweep steps coincide
    "nt1": dict(n=(16, 12, 20), band=(4, 4, 4), nt=1, seed=303, bound=2.0, sigma=0.5),
    # more than 128 x2 rows: two x2 tiles in the fused tensor-core transforms, the
    # second one partly filled
    "twotile": dict(n=(6, 140, 20), band=(4, 6, 8), nt=3, seed=404, bound=7.0),
    # x3 tables of 192 columns and band 48 x 48 in (x2, x3): the mixed expand
    # fetches each band slab in two halves (the grid of the precision form)
    "slabhalves": dict(n=(10, 52, 192), band=(4, 48, 48), nt=3, seed=505, bound=18.0),
}


@pytest.fixture(scope="module", params=[(c, pr) for c in sorted(CASES) for pr in ("fp32", "mixed")],
                ids=lambda t: f"{t[0]}-{t[1]}")
def case(request, blr):
    name, precision = request.param
    return Case(blr, precision=precision, **CASES[name])


def test_expand_project_parity(case):
    v = case.field()
    case.plan.expand(case.dev(case.vtf), v)
    assert rel(v.cpu().numpy(), O.expand(case.vt, case.p.n)) <= case.tol["field"]
    f = np.random.default_rng(7).normal(size=(3,) + case.n).astype(np.float32)
    ft = case.coef()
    case.plan.project(case.dev(f), ft)
    assert rel(ft.cpu().numpy(), O.project(f.astype(np.float64), case.band)) <= case.tol["field"]


def test_state_and_adjoint_parity(case):
    m1 = case.field(1)
    e = torch.zeros(3, dtype=torch.float64, device="cuda")
    case.plan.state(case.dev(case.vtf), m1, e)
    b = case.field()
    lam0 = case.field(1)
    case.plan.adjoint(b, lam0)
    assert case.plan.status() == 0
    pt = O.Point(case.vt, case.I0, case.I1, case.p)
    _, b_ref, lam0_ref = pt.gradient()
    tol = case.tol["field"]
    assert rel(m1.cpu().numpy(), pt.m[-1]) <= tol
    E = e.cpu().numpy()
    assert abs(E[0] - pt.energy) <= tol * pt.energy
    assert abs(E[1] - pt.energy_reg) <= 1e-5 * pt.energy_reg
    assert rel(lam0.cpu().numpy(), lam0_ref) <= tol
    assert rel(b.cpu().numpy(), b_ref) <= tol


def test_gradient_and_hessvec_parity(case):
    g = case.coef()
    case.plan.gradient(case.dev(case.vtf), g)
    h = case.coef()
    case.plan.hessvec(case.dev(case.dvf), h)
    pt = O.Point(case.vt, case.I0, case.I1, case.p)
    assert rel(g.cpu().numpy(), pt.gradient()[0]) <= case.tol["grad"]
    assert rel(h.cpu().numpy(), pt.gn_hessvec(case.dv)[0]) <= case.tol["grad"]


def test_pcg_iterates_parity(case):
    g = case.coef()
    case.plan.gradient(case.dev(case.vtf), g)
    rhs = -g
    x = case.coef()
    its, relres = case.plan.pcg(rhs, x, 4, 0.0)
    pt = O.Point(case.vt, case.I0, case.I1, case.p)
    rhs_ref = rhs.cpu().numpy().astype(np.complex128)
    x_ref, its_ref, rel_ref = O.pcg(lambda v: pt.gn_hessvec(v)[0], rhs_ref, 1.0 / pt.A[None],
                                    0.0, 4)
    assert its == its_ref == 4
    assert rel(x.cpu().numpy(), x_ref) <= case.tol["pcg"]
    assert abs(relres - rel_ref) <= 10 * case.tol["pcg"] * rel_ref


def test_deterministic_bitwise(case):
    g1, g2 = case.coef(), case.coef()
    case.plan.gradient(case.dev(case.vtf), g1)
    case.plan.gradient(case.dev(case.vtf), g2)
    assert torch.equal(g1, g2)
    h1, h2 = case.coef(), case.coef()
    case.plan.hessvec(case.dev(case.dvf), h1)
    case.plan.hessvec(case.dev(case.dvf), h2)
    assert torch.equal(h1, h2)


# --- degenerate cases and errors ---------------------------------------------


def test_zero_velocity_leaves_template_exactly(blr):
    c = Case(blr, n=(20, 18, 34), band=(4, 4, 6), nt=4, seed=404, bound=1.0)
    m1 = c.field(1)
    c.plan.state(c.coef(), m1)
    assert np.array_equal(m1.cpu().numpy(), c.I0f)


def test_constant_image_stays_constant(blr):
    n = (24, 20, 36)
    plan = blr.Plan(n, (6, 4, 8), 6)
    I = torch.full(n, 0.37, dtype=torch.float32, device="cuda")
    plan.set_images(I, I)
    vt = torch.from_numpy(synth.random_coefficients((6, 4, 8), 5, 10.0).astype(np.complex64)).cuda()
    m1 = torch.zeros(n, dtype=torch.float32, device="cuda")
    plan.state(vt, m1)
    assert float((m1 - 0.37).abs().max()) <= 1e-6


def test_cfl_violation_is_latched(blr):
    c = Case(blr, n=(16, 16, 16), band=(4, 4, 4), nt=2, seed=505, bound=1.0)
    vt = torch.from_numpy(synth.random_coefficients((4, 4, 4), 9, 40.0).astype(np.complex64)).cuda()
    c.plan.state(vt)
    assert c.plan.status() == blr.BLR_ECFL
    assert c.plan.status() == blr.BLR_OK        # cleared after reading
    c.plan.state(c.dev(c.vtf))
    assert c.plan.status() == blr.BLR_OK


def test_hessvec_needs_a_forward_solve(blr):
    plan = blr.Plan((8, 8, 8), (4, 4, 4), 2)
    z = torch.zeros((3, 4, 4, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(blr.BlrError) as ei:
        plan.hessvec(z, z.clone())
    assert ei.value.code == blr.BLR_ESTATE


# --- full registration (the 32^3 blob workload) --------------------------------


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_newton_registration_matches_oracle(blr, precision):
    n, band, nt = (32, 32, 32), (8, 8, 8), 10
    I0, I1, _ = synth.blob_pair(n, 1001, max_disp=2.0)
    (I0f, I0d), (I1f, I1d) = synth.as_device_inputs(I0, I1)
    plan = blr.Plan(n, band, nt,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(torch.from_numpy(I0f).cuda(), torch.from_numpy(I1f).cuda())
    vt = torch.zeros((3,) + band, dtype=torch.complex64, device="cuda")
    rep = plan.newton(vt, 5, 10, 1e-6)
    ref = O.newton(np.zeros((3,) + band, complex), I0d, I1d, O.Params(n, band, nt),
                   max_newton=5, max_pcg=10, gtol=1e-6)
    assert rep.newton_iters == ref.iterations
    assert abs(rep.energy - ref.energies[-1]) <= 1e-3 * ref.energies[-1]
    assert abs(rep.energy0 - ref.energies[0]) <= 1e-5 * ref.energies[0]
    assert abs(rep.pcg_iters - sum(ref.pcg_iterations)) <= ref.iterations
    assert rep.energy < 0.5 * rep.energy0


# --- full size: 128^3, band 32^3, 10 steps (the benchmark configuration) -------


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_full_size_gradient_and_hessvec(blr, precision):
    c = Case(blr, n=(128, 128, 128), band=(32, 32, 32), nt=10, seed=2002, bound=120.0,
             pair="phantom", max_disp=6.0, precision=precision)
    g = c.coef()
    e = torch.zeros(3, dtype=torch.float64, device="cuda")
    c.plan.gradient(c.dev(c.vtf), g, e)
    h = c.coef()
    c.plan.hessvec(c.dev(c.dvf), h)
    assert c.plan.status() == 0
    pt = O.Point(c.vt, c.I0, c.I1, c.p)
    assert abs(float(e[0]) - pt.energy) <= c.tol["field"] * pt.energy
    assert rel(g.cpu().numpy(), pt.gradient()[0]) <= c.tol["grad"]
    assert rel(h.cpu().numpy(), pt.gn_hessvec(c.dv)[0]) <= c.tol["grad"]


# --- precision form: 192x224x192 (the paper's 180x210x180 brains padded), band
# 48^3, 10 steps, 8-voxel phantom warp --------------------------------------------

N3C, B3C, SEED3 = (192, 224, 192), (48, 48, 48), 3001


@pytest.fixture(scope="module")
def big_point():
    I0, I1, _ = synth.phantom_pair(N3C, SEED3, max_disp=8.0)
    vt = synth.random_coefficients(B3C, SEED3 + 1, bound=200.0)   # 0.63 voxel per step
    dvt = synth.random_direction(B3C, SEED3 + 2)
    (I0f, I0d), (I1f, I1d), (vtf, vtd), (dvf, dvd) = synth.as_device_inputs(I0, I1, vt, dvt)
    pt = O.Point(vtd, I0d, I1d, O.Params(N3C, B3C, 10))
    g_ref = pt.gradient()[0]
    h_ref = pt.gn_hessvec(dvd)[0]
    return dict(I0f=I0f, I1f=I1f, vtf=vtf, dvf=dvf, energy=pt.energy, g=g_ref, h=h_ref)


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_precision_form_gradient_and_hessvec(blr, big_point, precision):
    b = big_point
    plan = blr.Plan(N3C, B3C, 10,
                    precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(torch.from_numpy(b["I0f"]).cuda(), torch.from_numpy(b["I1f"]).cuda())
    g = torch.zeros((3,) + B3C, dtype=torch.complex64, device="cuda")
    e = torch.zeros(3, dtype=torch.float64, device="cuda")
    plan.gradient(torch.from_numpy(b["vtf"]).cuda(), g, e)
    h = torch.zeros_like(g)
    plan.hessvec(torch.from_numpy(b["dvf"]).cuda(), h)
    assert plan.status() == 0
    tol = TOL[precision]
    assert abs(float(e[0]) - b["energy"]) <= tol["field"] * b["energy"]
    assert rel(g.cpu().numpy(), b["g"]) <= tol["grad"]
    assert rel(h.cpu().numpy(), b["h"]) <= tol["grad"]


@pytest.mark.slow
def test_precision_form_registration_mixed_against_fp32(blr, big_point):
    """10 Newton x <= 20 PCG from zero: the mixed path's final energy within
    1e-3 of the plain FP32 path's, PCG totals within +-1 per Newton step."""
    b = big_point
    reps = {}
    for precision in ("fp32", "mixed"):
        plan = blr.Plan(N3C, B3C, 10,
                        precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
        plan.set_images(torch.from_numpy(b["I0f"]).cuda(), torch.from_numpy(b["I1f"]).cuda())
        vt = torch.zeros((3,) + B3C, dtype=torch.complex64, device="cuda")
        reps[precision] = plan.newton(vt, 10, 20, 0.0)
        plan.close()
    f, m = reps["fp32"], reps["mixed"]
    assert f.status == m.status == blr.BLR_OK, reps
    assert f.newton_iters == m.newton_iters == 10, reps
    assert m.energy < 0.5 * m.energy0
    assert abs(m.energy0 - f.energy0) <= 5e-5 * f.energy0
    assert abs(m.energy - f.energy) <= 1e-3 * f.energy
    assert abs(m.pcg_iters - f.pcg_iters) <= f.newton_iters, reps
