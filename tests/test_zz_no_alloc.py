"""blr_expand_noalloc, the allocation-free expand for callers that cannot
allocate device memory (a host framework that owns every device allocation, or a
loop that cannot afford cudaMalloc's device synchronisation).  Its output must
match blr_expand of a plan within the expand tolerance of the parity tests
(relative L2 1e-5), on two calls in a row that share the library's one fixed
scratch array.  This file is collected last on purpose."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1807_05117_gb300 import synth  # noqa: E402


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _coefficients(band, seed):
    vt = synth.random_coefficients(band, seed, 10.0).astype(np.complex64)
    return torch.from_numpy(vt).cuda()


def test_expand_noalloc_matches_plan_expand_on_two_calls_in_a_row():
    from paper_1807_05117_gb300 import blr
    cases = [((40, 36, 52), (8, 6, 10), 11),        # ragged tiles on every axis
             ((128, 128, 128), (32, 32, 32), 12)]   # the largest size the array holds
    inputs, outs = [], []
    for n, band, seed in cases:
        inputs.append(_coefficients(band, seed))
        outs.append(torch.full((3,) + n, float("nan"), dtype=torch.float32, device="cuda"))
    # two calls in a row, back to back on one stream
    for (n, band, _), vt, out in zip(cases, inputs, outs):
        blr.blr_expand_noalloc(n, band, vt, out)
    torch.cuda.synchronize()
    for (n, band, _), vt, out in zip(cases, inputs, outs):
        ref = torch.zeros((3,) + n, dtype=torch.float32, device="cuda")
        with blr.Plan(n, band, 2) as plan:
            plan.expand(vt, ref)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) <= 1e-5


def test_expand_noalloc_rejects_sizes_beyond_the_array():
    """Correctly sized tensors, so that the library itself (not the binding's
    size check) rejects the problem: too large for the fixed array, or an odd band."""
    from paper_1807_05117_gb300 import blr
    for n, band in (((192, 224, 192), (48, 48, 48)), ((16, 16, 16), (5, 4, 4))):
        vt = torch.zeros((3,) + band, dtype=torch.complex64, device="cuda")
        v = torch.zeros((3,) + n, dtype=torch.float32, device="cuda")
        with pytest.raises(blr.BlrError) as ei:
            blr.blr_expand_noalloc(n, band, vt, v)
        assert ei.value.code == blr.BLR_EINVAL
    # a wrongly sized output is caught by the binding before any call
    vt = torch.zeros((3, 4, 4, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError):
        blr.blr_expand_noalloc((16, 16, 16), (4, 4, 4), vt,
                               torch.zeros(4, dtype=torch.float32, device="cuda"))
