"""Write oracle_regression.json: regression values of the FP64 oracle on small
seeded cases, one per variant (energy, gradient, Gauss-Newton and full Newton
products, a short Newton run).  Calls only oracle/ and the seeded input
generators; the values pin the oracle against unintended changes of its
arithmetic (its agreement with the paper and the mathematics is pinned by
tests/test_oracle_pins.py).  The paper prints no worked example to store here.

    python tests/golden/make_golden.py
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import blr_oracle as O  # noqa: E402
from paper_1807_05117_gb300 import synth  # noqa: E402

CASES = {
    "image_gn": dict(kw=dict(), hv="gn"),
    "image_full": dict(kw=dict(sigma=0.5), hv="full"),
    "incompressible_h1": dict(kw=dict(s=0.5, incompressible=True), hv="gn"),
    "nonstationary": dict(kw=dict(stationary=False), hv="gn"),
    "deformation": dict(kw=dict(state="deformation"), hv="gn"),
}
N, BAND, NT, SEED = (12, 10, 14), (4, 4, 6), 4, 3001


def summarise(z):
    z = np.asarray(z)
    return {"l2": float(np.linalg.norm(z)), "sum_re": float(np.sum(z.real)),
            "sum_im": float(np.sum(z.imag)), "first": [float(z.ravel()[0].real),
                                                       float(z.ravel()[0].imag)]}


def compute():
    out = {}
    I0, I1, _ = synth.blob_pair(N, SEED, max_disp=2.0)
    for name, c in CASES.items():
        p = O.Params(n=N, band=BAND, nt=NT, **c["kw"])
        steps = (NT,) if not p.stationary else ()
        vt = synth.random_coefficients(BAND, SEED + 1, bound=2.5)
        dvt = synth.random_direction(BAND, SEED + 2)
        if steps:
            vt = np.stack([synth.random_coefficients(BAND, SEED + 10 + n, bound=2.5)
                           for n in range(NT)])
            dvt = np.stack([synth.random_direction(BAND, SEED + 20 + n) for n in range(NT)])
        pt = O.make_point(vt, I0, I1, p)
        g = pt.gradient()[0]
        h = pt.full_hessvec(dvt)[0] if c["hv"] == "full" else pt.gn_hessvec(dvt)[0]
        rep = O.newton(np.zeros(steps + (3,) + BAND, complex), I0, I1, p, max_newton=2,
                       max_pcg=5, gtol=1e-8, hessian=c["hv"])
        out[name] = {"energy": pt.energy, "gradient": summarise(g), "hessvec": summarise(h),
                     "newton_energies": [float(e) for e in rep.energies],
                     "newton_pcg": [int(k) for k in rep.pcg_iterations]}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(compute(), f, indent=1, sort_keys=True)
        f.write("\n")
