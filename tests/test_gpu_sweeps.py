"""Sweep kernels chosen by the autotuner compute the same results bit for bit.

The adjoint sweep runs one time step per launch, or two (temporal blocking:
lambda^n kept in shared memory, the body force of both steps written once), or
is split (the steps transport lambda alone into kept adjoint states, one pass
then sums the body force of every step).  blr_plan_set_tuning forces each form
on the same plan; the gradient (Eq. 38),
the Gauss-Newton HVP (Eq. 46), and blr_adjoint's body force and lambda^0 must be
identical, for odd and even numbers of steps (an odd count ends with one
single step) and for ragged tiles.  The FP32 transforms' GEMM tiles likewise."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1807_05117_gb300 import synth  # noqa: E402

CASES = {
    "ragged-nt5": dict(n=(40, 36, 52), band=(8, 6, 10), nt=5, seed=611, bound=13.0),
    "nt2": dict(n=(24, 20, 36), band=(6, 4, 8), nt=2, seed=621, bound=4.0),
    "nt3": dict(n=(20, 44, 28), band=(4, 8, 6), nt=3, seed=631, bound=5.0),
    "nt1": dict(n=(16, 12, 20), band=(4, 4, 4), nt=1, seed=641, bound=2.0),
    "128cube": dict(n=(128, 128, 128), band=(32, 32, 32), nt=10, seed=651, bound=120.0),
}


def _run(plan, vt, dv, n, band, lambda0):
    g = torch.empty((3,) + band, dtype=torch.complex64, device="cuda")
    h = torch.empty_like(g)
    plan.gradient(vt, g)
    plan.hessvec(dv, h)
    b = torch.empty((3,) + n, dtype=torch.float32, device="cuda")
    lam0 = torch.empty(n, dtype=torch.float32, device="cuda") if lambda0 else None
    plan.adjoint(b, lam0)
    torch.cuda.synchronize()
    return g, h, b, lam0


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_adjoint_forms_are_bit_identical(name, precision):
    from paper_1807_05117_gb300 import blr
    c = CASES[name]
    n, band, nt = c["n"], c["band"], c["nt"]
    I0, I1, _ = synth.blob_pair(n, c["seed"], max_disp=2.0)
    vt = synth.random_coefficients(band, c["seed"] + 1, bound=c["bound"])
    dv = synth.random_direction(band, c["seed"] + 2)
    (I0f, _), (I1f, _), (vtf, _), (dvf, _) = synth.as_device_inputs(I0, I1, vt, dv)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    plan = blr.Plan(n, band, nt, precision=blr.BLR_MIXED if precision == "mixed" else blr.BLR_FP32)
    plan.set_images(dev(I0f), dev(I1f))
    assert plan.tuning()["grad_kept"] == 1
    out = {}
    for adj2, split in ((0, 0), (1, 0), (2, 0), (0, 1)):
        if (adj2 or split) and nt < 2:
            continue
        plan.set_tuning(adjoint_two_step=adj2, adjoint_split=split)
        tun = plan.tuning()
        assert (tun["adjoint_two_step"], tun["adjoint_split"]) == (adj2, split)
        for lambda0 in (False, True):
            out[(adj2, split, lambda0)] = _run(plan, dev(vtf), dev(dvf), n, band, lambda0)
    assert plan.status() == blr.BLR_OK
    for (adj2, split, lambda0), res in out.items():
        ref = out[(0, 0, lambda0)]
        for a, r in zip(res, ref):
            if r is not None:
                assert torch.equal(a, r), (adj2, split, lambda0)


GEMM_CASES = {
    "ragged-nt5": dict(n=(40, 36, 52), band=(8, 6, 10), nt=5, seed=661, bound=13.0, ns=False),
    "ragged-nonstationary": dict(n=(24, 20, 36), band=(6, 4, 8), nt=3, seed=671, bound=5.0, ns=True),
    "128cube": dict(n=(128, 128, 128), band=(32, 32, 32), nt=10, seed=681, bound=120.0, ns=False),
}


@pytest.mark.parametrize("name", sorted(GEMM_CASES))
def test_gemm_tiles_are_bit_identical(name):
    """The FP32 transforms' GEMM stages sum over k in order whatever the register
    tile and thread count, so every candidate (forced on all five stages at once)
    gives the gradient, the HVP and the body force bit for bit."""
    from paper_1807_05117_gb300 import blr
    c = GEMM_CASES[name]
    n, band, nt = c["n"], c["band"], c["nt"]
    I0, I1, _ = synth.blob_pair(n, c["seed"], max_disp=2.0)
    if c["ns"]:
        vt = np.stack([synth.random_coefficients(band, c["seed"] + 1 + k, bound=c["bound"])
                       for k in range(nt)])
        dv = np.stack([synth.random_direction(band, c["seed"] + 50 + k) for k in range(nt)])
        cshape = (nt, 3) + band
    else:
        vt = synth.random_coefficients(band, c["seed"] + 1, bound=c["bound"])
        dv = synth.random_direction(band, c["seed"] + 2)
        cshape = (3,) + band
    (I0f, _), (I1f, _), (vtf, _), (dvf, _) = synth.as_device_inputs(I0, I1, vt, dv)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    plan = blr.Plan(n, band, nt, precision=blr.BLR_FP32, nonstationary=c["ns"])
    plan.set_images(dev(I0f), dev(I1f))
    chosen = plan.tuning()["gemm_tiles"]
    assert all(1 <= (chosen >> (3 * st)) & 7 <= 6 for st in range(5)), chosen
    out = {}
    for cand in range(1, 7):
        plan.set_tuning(gemm_tiles=sum(cand << (3 * st) for st in range(5)))
        g = torch.empty(cshape, dtype=torch.complex64, device="cuda")
        h = torch.empty_like(g)
        plan.gradient(dev(vtf), g)
        plan.hessvec(dev(dvf), h)
        b = torch.empty(((nt,) if c["ns"] else ()) + (3,) + n, dtype=torch.float32, device="cuda")
        plan.adjoint(b)
        torch.cuda.synchronize()
        out[cand] = (g, h, b)
    assert plan.status() == blr.BLR_OK
    for cand, res in out.items():
        for a, r in zip(res, out[1]):
            assert torch.equal(a, r), cand
    plan.set_tuning(gemm_tiles=chosen)
    assert plan.tuning()["gemm_tiles"] == chosen


def test_set_tuning_rejects_shapes_the_plan_cannot_run():
    from paper_1807_05117_gb300 import blr
    plan = blr.Plan((16, 16, 16), (4, 4, 4), 4, ckpt_every=2)   # checkpoints: no kept gradients
    assert plan.tuning()["grad_kept"] == 0
    for bad in (dict(adjoint_two_step=1), dict(incremental_form=2), dict(adjoint_reads_grad=1),
                dict(march_chunk=0), dict(grad_kept=1), dict(adjoint_split=1),
                dict(gemm_tiles=7), dict(gemm_tiles=-1), dict(gemm_tiles=1 << 15)):
        with pytest.raises(blr.BlrError) as ei:
            plan.set_tuning(**bad)
        assert ei.value.code == blr.BLR_EINVAL
