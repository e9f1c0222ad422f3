"""Registration-level parity at the benchmark configuration: the 128^3 phantom
pair (band 32^3, 10 time steps), 10 Gauss-Newton updates x 20 PCG iterations
(forcing 0, so every update does the same fixed work), Armijo line search
(Section 3.4, Eqs. 54-55), run through blr_newton in both precisions against the
FP64 oracle's Newton run on the same rounded inputs.

Bars: Newton counts equal; the initial energy within 1e-5 and the final energy
within 1e-3 (relative); PCG totals within +-1 per Newton step; the same number
of step-length halvings (the line search took the same decisions)."""

import math

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

from oracle import blr_oracle as O  # noqa: E402
from paper_1807_05117_gb300 import synth  # noqa: E402

N, BAND, NT = (128, 128, 128), (32, 32, 32), 10
NEWTON, PCG = 10, 20
SEED, MAX_DISP = 2000, 6.0      # the benchmark's pair


@pytest.fixture(scope="module")
def oracle_run():
    I0, I1, _ = synth.phantom_pair(N, SEED, max_disp=MAX_DISP)
    (I0f, I0d), (I1f, I1d) = synth.as_device_inputs(I0, I1)
    ref = O.newton(np.zeros((3,) + BAND, complex), I0d, I1d, O.Params(N, BAND, NT),
                   max_newton=NEWTON, max_pcg=PCG, gtol=0.0, forcing=0.0)
    return I0f, I1f, ref


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_benchmark_registration_matches_oracle(oracle_run, precision):
    from paper_1807_05117_gb300 import blr
    I0f, I1f, ref = oracle_run
    plan = blr.Plan(N, BAND, NT, precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(torch.from_numpy(I0f).cuda(), torch.from_numpy(I1f).cuda())
    vt = torch.zeros((3,) + BAND, dtype=torch.complex64, device="cuda")
    rep = plan.newton(vt, NEWTON, PCG, 0.0, 0.0)
    plan.close()
    assert rep.status == blr.BLR_OK
    assert rep.newton_iters == ref.iterations == NEWTON
    assert abs(rep.energy0 - ref.energies[0]) <= 1e-5 * ref.energies[0]
    assert abs(rep.energy - ref.energies[-1]) <= 1e-3 * ref.energies[-1], (rep.energy, ref.energies)
    assert abs(rep.pcg_iters - sum(ref.pcg_iterations)) <= ref.iterations
    assert rep.n_halvings == sum(round(-math.log2(e)) for e in ref.steps)
    assert rep.energy < 0.2 * rep.energy0
