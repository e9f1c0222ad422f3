"""Failure detection without a GPU fault.

* A non-finite value made on the host (a NaN in the reference image, or in the
  velocity coefficients) comes back as BLR_ENAN from blr_status and from
  blr_newton; the plan recovers on clean inputs.
* A bounded device wait that runs out comes back as BLR_ETIMEOUT.  The wait is
  the tensor-core kernel's test hook (blr_test_expire_waits): a wait on a
  barrier nothing arrives at, taken before the kernel issues any copy or MMA,
  so nothing is in flight when it expires.  The launch frees its tensor memory
  and writes nothing; afterwards the same plan computes the same product as
  before, bit for bit.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1807_05117_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def blr():
    from paper_1807_05117_gb300 import blr as _blr
    return _blr


def _inputs(n, band, seed):
    I0, I1, _ = synth.blob_pair(n, seed, max_disp=2.0)
    vt = synth.random_coefficients(band, seed + 1, bound=8.0)
    dvt = synth.random_direction(band, seed + 2)
    (I0f, _), (I1f, _), (vtf, _), (dvf, _) = synth.as_device_inputs(I0, I1, vt, dvt)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    return dev(I0f), dev(I1f), dev(vtf), dev(dvf)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_nan_in_the_reference_image_is_reported_and_cleared(blr, precision):
    n, band = (24, 20, 36), (6, 4, 8)
    I0, I1, vt, _ = _inputs(n, band, 41)
    plan = blr.Plan(n, band, 4, precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    bad = I1.clone()
    bad[3, 5, 7] = float("nan")
    plan.set_images(I0, bad)
    plan.state(vt)
    assert plan.status() == blr.BLR_ENAN
    assert plan.status() == blr.BLR_OK          # latched once, cleared by reading
    rep = plan.newton(torch.zeros_like(vt), 2, 3, 0.0, raise_on_error=False)
    assert rep.status == blr.BLR_ENAN and rep.newton_iters == 0
    plan.set_images(I0, I1)
    e = torch.zeros(3, dtype=torch.float64, device="cuda")
    plan.state(vt, energy=e)
    assert plan.status() == blr.BLR_OK
    assert np.isfinite(e.cpu().numpy()).all()
    plan.close()


def test_nan_in_the_velocity_is_reported(blr):
    n, band = (24, 20, 36), (6, 4, 8)
    I0, I1, vt, _ = _inputs(n, band, 43)
    plan = blr.Plan(n, band, 4)
    plan.set_images(I0, I1)
    bad = vt.clone()
    bad[1, 2, 1, 3] = complex(float("nan"), 0.0)
    plan.state(bad)
    assert plan.status() == blr.BLR_ENAN
    plan.state(vt)
    assert plan.status() == blr.BLR_OK
    plan.close()


def test_expired_tensor_core_wait_is_reported_and_the_plan_recovers(blr):
    n, band = (64, 64, 64), (16, 16, 16)
    I0, I1, vt, dv = _inputs(n, band, 47)
    plan = blr.Plan(n, band, 5, precision=blr.BLR_MIXED)
    plan.set_images(I0, I1)
    g = torch.zeros_like(vt)
    plan.gradient(vt, g)
    h_ref = torch.zeros_like(vt)
    plan.hessvec(dv, h_ref)
    assert plan.status() == blr.BLR_OK
    h = torch.full_like(vt, complex(7.0, 7.0))
    blr.blr_test_expire_waits(True)
    try:
        plan.hessvec(dv, h)
        assert plan.status() == blr.BLR_ETIMEOUT
    finally:
        blr.blr_test_expire_waits(False)
    assert plan.status() == blr.BLR_OK          # cleared by the read above
    plan.hessvec(dv, h)
    assert plan.status() == blr.BLR_OK
    assert torch.equal(h, h_ref)
    plan.close()
