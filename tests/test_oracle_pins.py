"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
brute-force sums, closed forms, library FFTs, exact shifts, finite differences,
dense linear algebra.  Each test names the plausible mistake it would catch.

These run on the CPU (not marked gpu)."""

import cmath
import itertools
import math

import numpy as np
import pytest

from oracle import blr_oracle as O
from paper_1807_05117_gb300 import synth


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


# ----------------------------------------------------------------------------
# iota / pi (Section 3.1, Eq. 33)
# ----------------------------------------------------------------------------

N_SMALL = (6, 5, 4)      # non-cubic so a transposed axis shows up
B_SMALL = (4, 2, 4)


def test_expand_brute_force_triple_sum():
    """iota against the definition summed term by term with cmath.exp
    (catches a wrong sign in the exponent, a transposed axis, an off-centre band)."""
    vt = synth.random_direction(B_SMALL, 1) * 10
    got = O.expand(vt, N_SMALL)
    ks = [np.arange(B) - B // 2 for B in B_SMALL]
    for c in range(3):
        for x in itertools.product(*[range(N) for N in N_SMALL]):
            acc = 0j
            for j in itertools.product(*[range(B) for B in B_SMALL]):
                ph = sum(ks[d][j[d]] * x[d] / N_SMALL[d] for d in range(3))
                acc += vt[(c,) + j] * cmath.exp(2j * math.pi * ph)
            assert abs(got[(c,) + x] - acc.real) < 1e-12


def test_expand_single_mode_is_cosine():
    """A unit coefficient at frequency k gives cos(2 pi k.x/N); i at k gives -sin."""
    n = (8, 6, 10)
    band = (4, 4, 6)
    x = np.indices(n)
    for c, j in [(0, (0, 0, 0)), (1, (3, 1, 5)), (2, (1, 2, 0))]:
        k = [j[d] - band[d] // 2 for d in range(3)]
        theta = sum(2 * np.pi * k[d] * x[d] / n[d] for d in range(3))
        for coef, want in [(1.0, np.cos(theta)), (1j, -np.sin(theta))]:
            vt = np.zeros((3,) + band, complex)
            vt[(c,) + j] = coef
            v = O.expand(vt, n)
            assert np.max(np.abs(v[c] - want)) < 1e-12
            others = [a for a in range(3) if a != c]
            assert np.max(np.abs(v[others])) == 0.0


def test_expand_matches_numpy_inverse_fft():
    """iota(v) = Re(V * ifftn(v embedded at k mod N)) -- a library routine with
    its own sign and normalisation conventions."""
    n = (12, 10, 8)
    band = (6, 4, 8)
    vt = synth.random_direction(band, 2)
    X = np.zeros((3,) + n, complex)
    ks = [np.arange(B) - B // 2 for B in band]
    for j in itertools.product(*[range(B) for B in band]):
        idx = tuple(ks[d][j[d]] % n[d] for d in range(3))
        X[(slice(None),) + idx] = vt[(slice(None),) + j]
    want = np.real(np.fft.ifftn(X, axes=(1, 2, 3))) * np.prod(n)
    assert rel(O.expand(vt, n), want) < 1e-13


def test_project_matches_numpy_fft():
    """pi(f)(k) = fftn(f)[k mod N] (numpy's forward FFT uses exp(-2 pi i k x/N))."""
    n = (12, 10, 8)
    band = (6, 4, 8)
    f = np.random.default_rng(3).normal(size=(3,) + n)
    F = np.fft.fftn(f, axes=(1, 2, 3))
    got = O.project(f, band)
    ks = [np.arange(B) - B // 2 for B in band]
    for j in itertools.product(*[range(B) for B in band]):
        idx = tuple(ks[d][j[d]] % n[d] for d in range(3))
        assert np.max(np.abs(got[(slice(None),) + j] - F[(slice(None),) + idx])) < 1e-10


def test_project_brute_force_triple_sum():
    f = np.random.default_rng(4).normal(size=(3,) + N_SMALL)
    got = O.project(f, B_SMALL)
    ks = [np.arange(B) - B // 2 for B in B_SMALL]
    for c in range(3):
        for j in itertools.product(*[range(B) for B in B_SMALL]):
            acc = 0j
            for x in itertools.product(*[range(N) for N in N_SMALL]):
                ph = sum(ks[d][j[d]] * x[d] / N_SMALL[d] for d in range(3))
                acc += f[(c,) + x] * cmath.exp(-2j * math.pi * ph)
            assert abs(got[(c,) + j] - acc) < 1e-11


def test_project_is_transpose_of_expand():
    """<iota v, f> = <v, pi f> under the real inner product of the parameters."""
    n = (16, 12, 10)
    band = (8, 6, 4)
    vt = synth.random_direction(band, 5)
    f = np.random.default_rng(6).normal(size=(3,) + n)
    lhs = float(np.sum(O.expand(vt, n) * f))
    rhs = O.inner(vt, O.project(f, band))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _band_projector(f, n, band):
    """P = iota o diag(c_k / V) o pi, c_k = 1 if -k is in the band, else 2."""
    V = np.prod(n)
    ks = [np.arange(B) - B // 2 for B in band]
    c = np.ones(band)
    for j in itertools.product(*[range(B) for B in band]):
        neg_in = all(-ks[d][j[d]] >= -(band[d] // 2) and -ks[d][j[d]] <= band[d] // 2 - 1
                     for d in range(3))
        c[j] = 1.0 if neg_in else 2.0
    return O.expand(c[None] * O.project(f, band) / V, n)


def test_band_projector_idempotent_symmetric_parseval():
    n = (12, 10, 14)
    band = (6, 4, 8)
    rng = np.random.default_rng(7)
    f = rng.normal(size=(3,) + n)
    g = rng.normal(size=(3,) + n)
    Pf = _band_projector(f, n, band)
    assert rel(_band_projector(Pf, n, band), Pf) < 1e-12                 # P^2 = P
    a, b = np.sum(Pf * g), np.sum(f * _band_projector(g, n, band))
    assert abs(a - b) < 1e-11 * abs(a)                                   # P = P^T
    # Parseval on a band-limited field: ||iota v||^2 = V^-1 sum_{band u -band} |F|^2
    vt = synth.random_direction(band, 8)
    v = O.expand(vt, n)
    F = np.fft.fftn(v, axes=(1, 2, 3))
    mask = np.zeros(n, bool)
    ks = [np.arange(B) - B // 2 for B in band]
    for j in itertools.product(*[range(B) for B in band]):
        mask[tuple(ks[d][j[d]] % n[d] for d in range(3))] = True
        mask[tuple(-ks[d][j[d]] % n[d] for d in range(3))] = True
    lhs = np.sum(v * v)
    rhs = np.sum(np.abs(F[:, mask]) ** 2) / np.prod(n)
    assert abs(lhs - rhs) < 1e-12 * lhs
    assert np.sum(np.abs(F[:, ~mask]) ** 2) < 1e-20 * lhs


# ----------------------------------------------------------------------------
# Regulariser symbol (Eq. 1 family; Section 3.1)
# ----------------------------------------------------------------------------


def _neg_laplacian(u):
    out = 6.0 * u
    for ax in range(3):
        out -= np.roll(u, 1, axis=ax) + np.roll(u, -1, axis=ax)
    return out


def test_regulariser_symbol_is_stencil_eigenvalue():
    """A(k) = eigenvalue of (alpha(-Lap_h) + gamma) applied 2s times to the Fourier
    mode k, with Lap_h the periodic 7-point stencil (catches a wrong exponent,
    a missing 2 pi or a cos/sin mix-up)."""
    for s in (2, 0.5):     # s = 1/2: the H^1 regulariser alpha(-Lap) + gamma
        p = O.Params(n=(10, 12, 8), band=(6, 8, 4), alpha=3.0, gamma=1.0, s=s)
        A = O.regulariser_weights(p)
        omega = O.laplacian_symbol(p.n, p.band)
        x = np.indices(p.n)
        for j in [(0, 0, 0), (1, 5, 2), (3, 4, 0), (5, 7, 3)]:
            k = [j[d] - p.band[d] // 2 for d in range(3)]
            mode = np.exp(2j * np.pi * sum(k[d] * x[d] / p.n[d] for d in range(3)))
            lap = _neg_laplacian(mode)
            assert np.max(np.abs(lap - omega[j] * mode)) < 1e-12
            u = mode
            for _ in range(int(2 * s)):
                u = p.alpha * _neg_laplacian(u) + p.gamma * u
            assert np.max(np.abs(u - A[j] * mode)) < 1e-9 * A[j]
    with pytest.raises(ValueError):
        O.regulariser_weights(O.Params(n=(8, 8, 8), band=(4, 4, 4), s=0.3))


# ----------------------------------------------------------------------------
# Transport (state equation, Eq. 36)
# ----------------------------------------------------------------------------


def test_zero_velocity_leaves_template_unchanged():
    p = O.Params(n=(9, 8, 7), band=(4, 4, 2), nt=5)
    I0, I1, _ = synth.blob_pair(p.n, 11)
    pt = O.Point(np.zeros((3,) + p.band, complex), I0, I1, p)
    assert np.array_equal(pt.m[-1], I0)


def test_constant_image_stays_constant():
    p = O.Params(n=(9, 8, 7), band=(4, 4, 2), nt=6)
    vt = synth.random_coefficients(p.band, 12, bound=3.0)
    I0 = np.full(p.n, 0.37)
    pt = O.Point(vt, I0, I0, p)
    assert np.max(np.abs(pt.m[-1] - 0.37)) < 1e-15


def test_integer_constant_velocity_is_exact_periodic_shift():
    """v~(0) = c gives the constant velocity Re c; with dt*c integer every step is
    an exact periodic shift m^{n+1}(x) = m^n(x - dt c)."""
    p = O.Params(n=(9, 8, 7), band=(4, 4, 2), nt=2)
    vt = np.zeros((3,) + p.band, complex)
    zero = tuple(B // 2 for B in p.band)
    vt[(slice(None),) + zero] = [2.0, -2.0, 4.0]          # d = -dt v = (-1, 1, -2)
    I0, _, _ = synth.blob_pair(p.n, 13)
    pt = O.Point(vt, I0, I0, p)
    want = I0
    for _ in range(p.nt):
        want = np.roll(want, shift=(1, -1, 2), axis=(0, 1, 2))   # m(x) <- m(x + d)
    assert np.array_equal(pt.m[-1], want)


def test_interpolation_reproduces_affine_field():
    """Trilinear interpolation is exact on affine fields and its gradient is the
    slope (interior voxels, away from the periodic seam)."""
    n = (12, 11, 10)
    rng = np.random.default_rng(14)
    a = rng.normal(size=3)
    x = np.indices(n).astype(float)
    m = 0.3 + sum(a[k] * x[k] for k in range(3))
    d = rng.uniform(-0.95, 0.95, size=(3,) + n)
    st = O.Stencil(d)
    val = st.apply(m)
    grad = st.gradient(m)
    inner_sl = (slice(1, -1),) * 3
    want = 0.3 + sum(a[k] * (x[k] + d[k]) for k in range(3))
    assert np.max(np.abs(val[inner_sl] - want[inner_sl])) < 1e-12
    for k in range(3):
        assert np.max(np.abs(grad[k][inner_sl] - a[k])) < 1e-12


def test_interpolation_separable_closed_form_with_wrap():
    """On m = g1(x1) g2(x2) g3(x3) the trilinear value is the product of 1-D
    periodic linear interpolants, and each partial derivative replaces one factor
    by its slope; displacements up to 2.5 voxels exercise the periodic wrap and
    the floor cell rule."""
    n = (7, 6, 5)
    rng = np.random.default_rng(15)
    g = [rng.normal(size=N) for N in n]
    m = g[0][:, None, None] * g[1][None, :, None] * g[2][None, None, :]
    d = rng.uniform(-2.5, 2.5, size=(3,) + n)
    st = O.Stencil(d)
    val, grad = st.apply(m), st.gradient(m)
    x = np.indices(n)
    L, dL = [], []
    for k in range(3):
        pos = x[k] + d[k]
        i = np.floor(pos).astype(int)
        f = pos - i
        g0, g1 = g[k][i % n[k]], g[k][(i + 1) % n[k]]
        L.append((1 - f) * g0 + f * g1)
        dL.append(g1 - g0)
    assert np.max(np.abs(val - L[0] * L[1] * L[2])) < 1e-12
    assert np.max(np.abs(grad[0] - dL[0] * L[1] * L[2])) < 1e-12
    assert np.max(np.abs(grad[1] - L[0] * dL[1] * L[2])) < 1e-12
    assert np.max(np.abs(grad[2] - L[0] * L[1] * dL[2])) < 1e-12


def test_adjoint_step_is_exact_transpose():
    """Dense S built column by column from the forward step, against the adjoint
    step applied to unit vectors; plus the dot-product identity at a larger size."""
    n = (3, 4, 5)
    V = int(np.prod(n))
    d = np.random.default_rng(16).uniform(-0.9, 0.9, size=(3,) + n)
    st = O.Stencil(d)
    S = np.zeros((V, V))
    ST = np.zeros((V, V))
    for j in range(V):
        e = np.zeros(V)
        e[j] = 1.0
        S[:, j] = st.apply(e.reshape(n)).ravel()
        ST[:, j] = st.apply_transpose(e.reshape(n)).ravel()
    assert np.max(np.abs(ST - S.T)) == 0.0
    assert np.allclose(S.sum(axis=1), 1.0, atol=1e-14)     # weights sum to one
    n2 = (14, 13, 12)
    rng = np.random.default_rng(17)
    st2 = O.Stencil(rng.uniform(-0.9, 0.9, size=(3,) + n2))
    a, b = rng.normal(size=n2), rng.normal(size=n2)
    lhs, rhs = np.sum(st2.apply(a) * b), np.sum(a * st2.apply_transpose(b))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ----------------------------------------------------------------------------
# Gradient (Eq. 38) against central finite differences of the energy (Eq. 35)
# ----------------------------------------------------------------------------


def _kink_free(vt, dvt, eps, p):
    """True when no voxel changes interpolation cell between v -+ eps dv."""
    lo = np.floor(O.displacement(vt - eps * dvt, p))
    hi = np.floor(O.displacement(vt + eps * dvt, p))
    return np.array_equal(lo, hi)


def test_gradient_matches_central_finite_differences():
    """32 random directions on a 16^3 grid, step 1e-6, relative error 1e-6."""
    p = O.Params(n=(16, 16, 16), band=(6, 6, 6), nt=10)
    I0, I1, _ = synth.blob_pair(p.n, 21, max_disp=2.0)
    vt = synth.random_coefficients(p.band, 22, bound=2.5)
    pt = O.Point(vt, I0, I1, p)
    g, _, _ = pt.gradient()
    eps = 1e-6
    checked = 0
    for s in range(48):
        dvt = synth.random_direction(p.band, 100 + s)
        if not _kink_free(vt, dvt, eps, p):
            continue
        fd = (O.energy(vt + eps * dvt, I0, I1, p) - O.energy(vt - eps * dvt, I0, I1, p)) / (2 * eps)
        dd = O.inner(g, dvt)
        assert abs(fd - dd) <= 1e-6 * abs(dd), (s, fd, dd)
        checked += 1
        if checked == 32:
            break
    assert checked == 32


def test_gradient_regulariser_part_only():
    """With I1 equal to the transported template the data term is zero and the
    gradient's data part vanishes: g = A v (catches a missing 1/2 or a square)."""
    p = O.Params(n=(10, 9, 8), band=(4, 4, 4), nt=4)
    I0, _, _ = synth.blob_pair(p.n, 23)
    vt = synth.random_coefficients(p.band, 24, bound=1.5)
    pt0 = O.Point(vt, I0, I0, p)
    pt = O.Point(vt, I0, pt0.m[-1], p)
    g, _, _ = pt.gradient()
    A = O.regulariser_weights(p)
    assert rel(g, A[None] * vt) < 1e-14
    assert abs(pt.energy - 0.5 * np.sum(A[None] * np.abs(vt) ** 2)) < 1e-12 * pt.energy


# ----------------------------------------------------------------------------
# Gauss-Newton Hessian (Eq. 46 with the Section 3.4 drops)
# ----------------------------------------------------------------------------


def _theta(z):
    return np.concatenate([z.real.ravel(), z.imag.ravel()])


def _from_theta(t, shape):
    h = t.size // 2
    return (t[:h] + 1j * t[h:]).reshape(shape)


def test_gn_hessian_symmetric_positive_16cube():
    p = O.Params(n=(16, 16, 16), band=(6, 6, 6), nt=10)
    I0, I1, _ = synth.blob_pair(p.n, 31, max_disp=2.0)
    vt = synth.random_coefficients(p.band, 32, bound=2.5)
    pt = O.Point(vt, I0, I1, p)
    for s in range(3):
        v = synth.random_direction(p.band, 300 + s)
        w = synth.random_direction(p.band, 400 + s)
        Hv, Hw = pt.gn_hessvec(v)[0], pt.gn_hessvec(w)[0]
        a, b = O.inner(Hv, w), O.inner(v, Hw)
        assert abs(a - b) <= 1e-10 * max(abs(a), abs(b))
        assert O.inner(Hv, v) > 0.0


def test_gn_hessian_equals_dense_jacobian_bruteforce():
    """8^3 grid, band 4^3 (384 real parameters): J = dm^nt/dtheta by central
    differences of the state, H = A + (2/sigma^2) J^T J, compared with the
    incremental state / incremental adjoint chain."""
    p = O.Params(n=(8, 8, 8), band=(4, 4, 4), nt=3, sigma=0.7)
    I0, I1, _ = synth.blob_pair(p.n, 41, max_disp=1.5)
    # first seeded point whose displacements keep >= 1e-4 voxel from every cell
    # boundary, so no per-parameter difference straddles a kink
    for seed in range(42, 80):
        vt = synth.random_coefficients(p.band, seed, bound=1.2)
        d = O.displacement(vt, p)
        if np.min(np.abs(d - np.round(d))) >= 1e-4:
            break
    else:
        raise AssertionError("no kink-free point")
    pt = O.Point(vt, I0, I1, p)
    P = 2 * 3 * 64
    eps = 1e-6
    J = np.zeros((int(np.prod(p.n)), P))
    for j in range(P):
        e = np.zeros(P)
        e[j] = eps
        de = _from_theta(e, vt.shape)
        mp = O.Point(vt + de, I0, I1, p).m[-1]
        mm = O.Point(vt - de, I0, I1, p).m[-1]
        J[:, j] = ((mp - mm) / (2 * eps)).ravel()
    A = O.regulariser_weights(p)
    Ad = np.concatenate([np.tile(A.ravel(), 3)] * 2)
    H = np.diag(Ad) + (2.0 / p.sigma**2) * J.T @ J
    for s in range(4):
        v = synth.random_direction(p.band, 500 + s)
        got = _theta(pt.gn_hessvec(v)[0])
        assert rel(got, H @ _theta(v)) < 1e-7


def test_gn_hessian_is_fd_of_gradient_at_zero_residual():
    """At zero residual (I1 = m^nt(v)) the terms the Gauss-Newton step drops are
    zero, so H_GN dv equals the central difference of the gradient."""
    p = O.Params(n=(12, 12, 12), band=(4, 6, 4), nt=5)
    I0, _, _ = synth.blob_pair(p.n, 51, max_disp=2.0)
    vt = synth.random_coefficients(p.band, 52, bound=2.0)
    I1 = O.Point(vt, I0, I0, p).m[-1]
    pt = O.Point(vt, I0, I1, p)
    eps = 1e-6
    for s in range(3):
        dvt = synth.random_direction(p.band, 600 + s)
        if not _kink_free(vt, dvt, eps, p):
            continue
        gp = O.Point(vt + eps * dvt, I0, I1, p).gradient()[0]
        gm = O.Point(vt - eps * dvt, I0, I1, p).gradient()[0]
        assert rel(pt.gn_hessvec(dvt)[0], (gp - gm) / (2 * eps)) < 1e-6


# ----------------------------------------------------------------------------
# PCG and Newton (Section 3.4)
# ----------------------------------------------------------------------------


def test_pcg_to_convergence_equals_dense_solve():
    p = O.Params(n=(8, 8, 8), band=(4, 4, 4), nt=3)
    I0, I1, _ = synth.blob_pair(p.n, 61, max_disp=1.5)
    vt = synth.random_coefficients(p.band, 62, bound=1.0)
    pt = O.Point(vt, I0, I1, p)
    P = 2 * 3 * 64
    H = np.zeros((P, P))
    for j in range(P):
        e = np.zeros(P)
        e[j] = 1.0
        H[:, j] = _theta(pt.gn_hessvec(_from_theta(e, vt.shape))[0])
    g, _, _ = pt.gradient()
    want = np.linalg.solve(H, -_theta(g))
    x, its, r = O.pcg(lambda v: pt.gn_hessvec(v)[0], -g, 1.0 / pt.A[None], 1e-13, 500)
    assert r <= 1e-13
    assert rel(_theta(x), want) < 1e-9


def test_newton_decreases_energy_and_gradient():
    p = O.Params(n=(16, 16, 16), band=(4, 4, 4), nt=5)
    I0, I1, _ = synth.blob_pair(p.n, 71, max_disp=2.0)
    rep = O.newton(np.zeros((3,) + p.band, complex), I0, I1, p, max_newton=4, max_pcg=8,
                   gtol=1e-6)
    assert rep.iterations >= 3
    assert all(b < a for a, b in zip(rep.energies, rep.energies[1:]))
    assert rep.grad_inf_rel < 0.5


# Closed-form objectives for the Newton iteration itself (Section 3.4, Eqs. 54-55
# read as v~ <- v~ + eps p with H p = -g).  The parameter space is complex arrays
# with <a, b> = Re sum a conj(b), i.e. the real vector (Re x, Im x).


class _DiagObjective:
    """E(x) = sum_i phi(Re x_i) + phi(Im x_i) for a scalar function phi with
    derivatives dphi, ddphi: gradient and Hessian are elementwise.  The
    preconditioner 1 / A is per frequency, shared by the three components: A is
    component 0's Hessian diagonal (exact where only component 0 moves) unless
    `A` is given."""

    def __init__(self, x, phi, dphi, ddphi, A=None):
        self.vt = x
        self.energy = float(np.sum(phi(x.real)) + np.sum(phi(x.imag)))
        self._g = dphi(x.real) + 1j * dphi(x.imag)
        self._hr, self._hi = ddphi(x.real), ddphi(x.imag)
        self.A = self._hr[0] if A is None else A
        self.cfl = 0.0

    def gradient(self):
        return self._g, None, None

    def gn_hessvec(self, v):
        return self._hr * v.real + 1j * (self._hi * v.imag), None


class _Quadratic:
    """E(x) = 1/2 <x, q x> - <c, x>, q > 0 real elementwise; the preconditioner
    is 1 / A (A per frequency: q[0] when q is the same for every component)."""

    def __init__(self, x, q, c, A):
        self.vt = x
        self.energy = 0.5 * O.inner(x, q * x) - O.inner(c, x)
        self._g = q * x - c
        self._q = q
        self.A = A
        self.cfl = 0.0

    def gradient(self):
        return self._g, None, None

    def gn_hessvec(self, v):
        return self._q * v, None


def _quadratic(q, c, A=None):
    return lambda x: _Quadratic(x, q, c, q[0] if A is None else A)


def test_newton_takes_the_exact_newton_step_on_a_quadratic():
    """With the exact preconditioner PCG solves H p = -g in one iteration, the
    full step eps = 1 passes Armijo and lands on the minimiser q^-1 c, where the
    gradient vanishes (catches v - eps p, a wrong PCG start, a missing step)."""
    rng = np.random.default_rng(3)
    shape = (3, 2, 2, 2)
    q = np.broadcast_to(rng.uniform(0.5, 4.0, size=shape[1:]), shape).copy()
    c = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    rep = O.newton(np.zeros(shape, complex), None, None, None, max_newton=3, max_pcg=5,
                   gtol=1e-12, point=_quadratic(q, c))
    assert rep.iterations == 1 and rep.steps == [1.0] and rep.pcg_iterations == [1]
    assert rel(rep.vt, c / q) < 1e-14
    assert abs(rep.energies[1] - (-0.5 * O.inner(c, c / q))) < 1e-12 * abs(rep.energies[1])


def _huber():
    return (lambda t: np.sqrt(1 + t * t), lambda t: t / np.sqrt(1 + t * t),
            lambda t: (1 + t * t) ** -1.5)


def test_newton_backtracking_halves_to_the_first_armijo_step():
    """phi(t) = sqrt(1 + t^2): the Newton step from t is -t(1 + t^2).  From t = 2
    it goes to -8 (eps = 1) and -3 (eps = 1/2), both uphill, and eps = 1/4 gives
    t = -1/2.  From there full steps are taken and t -> -t^3 (catches a missing
    halving, a wrong halving factor, a step that is not re-based on the accepted
    point)."""
    phi, dphi, ddphi = _huber()
    x0 = np.zeros((3, 2, 2, 2), complex)
    x0[0, 0, 1, 0] = 2.0
    rep = O.newton(x0, None, None, None, max_newton=3, max_pcg=5, gtol=0.0,
                   point=lambda x: _DiagObjective(x, phi, dphi, ddphi))
    assert rep.steps == [0.25, 1.0, 1.0]
    want = [2.0, -0.5, 0.125, -0.125 ** 3]
    E = [float(np.sum(phi(np.array([t])))) + (2 * x0.size - 1) for t in want]
    assert np.allclose(rep.energies, E, rtol=0, atol=1e-14)
    assert rep.vt.shape == x0.shape
    assert abs(rep.vt[0, 0, 1, 0] - want[-1]) < 1e-15


@pytest.mark.parametrize("ratio,eps", [(1.25e-4, 1.0), (0.8e-4, 0.5)])
def test_newton_armijo_constant_is_1e_4(ratio, eps):
    """From t0 = 1 - delta the full Newton step lands on -(1 - delta)^3, a small
    decrease.  delta is chosen (bisection on the closed form) so that the
    decrease is `ratio` times |eps <g, p>| at eps = 1: with c1 = 1e-4 the full step
    is accepted at ratio 1.25e-4 and rejected at 0.8e-4 (then eps = 1/2 passes).
    A constant outside [0.8e-4, 1.25e-4) fails one of the two cases."""
    phi, dphi, ddphi = _huber()

    def decrease_ratio(d):
        t0 = 1.0 - d
        p = -t0 * (1 + t0 * t0)
        return (phi(t0) - phi(t0 + p)) / abs(dphi(t0) * p)

    lo, hi = 1e-9, 1e-2          # decrease_ratio is increasing in delta on this range
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if decrease_ratio(mid) < ratio:
            lo = mid
        else:
            hi = mid
    t0 = 1.0 - 0.5 * (lo + hi)
    x0 = np.zeros((3, 2, 2, 2), complex)
    x0[0, 1, 1, 1] = t0   # component 0: the preconditioner is exact there
    rep = O.newton(x0, None, None, None, max_newton=1, max_pcg=5, gtol=0.0,
                   point=lambda x: _DiagObjective(x, phi, dphi, ddphi))
    assert rep.steps == [eps]


def test_newton_forcing_term_matches_scipy_cg_iteration_counts():
    """Without a preconditioner (A = 1) PCG is plain CG; per Newton step its
    iteration count must be that of scipy's CG on the same system with
    rtol = eta, eta = min(0.5, sqrt(||g|| / ||g0||)) (catches a forcing term in
    the inf-norm, without the square root, or measured against the wrong norm)."""
    from scipy.sparse.linalg import cg
    rng = np.random.default_rng(11)
    shape = (3, 4, 4, 4)
    q = rng.uniform(1.0, 300.0, size=shape)
    c = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    rep = O.newton(np.zeros(shape, complex), None, None, None, max_newton=3, max_pcg=200,
                   gtol=0.0, point=_quadratic(q, c, A=np.ones(shape[1:])))
    assert rep.steps == [1.0, 1.0, 1.0]   # CG iterates satisfy Armijo at eps = 1
    Q = np.concatenate([q.ravel(), q.ravel()])
    x = np.zeros(2 * q.size)
    b = np.concatenate([c.real.ravel(), c.imag.ravel()])
    g0 = np.linalg.norm(Q * x - b)
    for its in rep.pcg_iterations:
        g = Q * x - b
        eta = min(0.5, math.sqrt(np.linalg.norm(g) / g0))
        count = []
        p, _ = cg(np.diag(Q), -g, rtol=eta, atol=0.0, maxiter=200,
                  callback=lambda _x: count.append(1))
        assert its == len(count)
        x = x + p
    assert rel(np.concatenate([rep.vt.real.ravel(), rep.vt.imag.ravel()]), x) < 1e-10


def test_newton_line_search_log_on_a_registration():
    """On a registration: every accepted eps satisfies the Armijo inequality with
    c1 = 1e-4 against the base point's energy and slope <g, p>, and every trial
    before it (eps' = 2 eps, 4 eps, ... from 1) did not."""
    p = O.Params(n=(12, 12, 12), band=(4, 4, 4), nt=4)
    I0, I1, _ = synth.blob_pair(p.n, 72, max_disp=2.5)
    log = []

    def point(v):
        pt = O.make_point(v, I0, I1, p)
        log.append(pt)
        return pt

    rep = O.newton(np.zeros((3,) + p.band, complex), None, None, None, max_newton=4,
                   max_pcg=6, gtol=0.0, point=point)
    assert rep.iterations >= 3
    i = 0
    base = log[0]
    for eps in rep.steps:
        step = None
        trials = [1.0]
        while trials[-1] > eps:
            trials.append(trials[-1] * 0.5)
        g = base.gradient()[0]
        for k, e in enumerate(trials):
            i += 1
            t = log[i]
            if step is None:
                step = (t.vt - base.vt) / e
            assert rel(t.vt, base.vt + e * step) < 1e-13
            bound = base.energy + 1e-4 * e * O.inner(g, step)
            if k == len(trials) - 1:
                assert t.energy <= bound
            else:
                assert not (t.cfl < 1.0 and t.energy <= bound)
        base = log[i]


# ----------------------------------------------------------------------------
# Incompressible form (Eq. 4 with gamma = 1, constraint in the band)
# ----------------------------------------------------------------------------

N_INC = (12, 10, 8)      # anisotropic, so a wave vector without the 1/N_d shows up
B_INC = (6, 4, 6)


def _band_field(vt, n, pts):
    """The band-limited field Re sum_k v~(k) exp(2 pi i sum_d k_d x_d / N_d) at
    arbitrary real points (P, 3), summed directly (not through the oracle)."""
    B = vt.shape[1:]
    ks = np.stack(np.meshgrid(*[np.arange(b) - b // 2 for b in B], indexing="ij"),
                  axis=-1).reshape(-1, 3)
    phase = np.exp(2j * np.pi * (pts / np.asarray(n, float)) @ ks.T)     # (P, K)
    return (phase @ vt.reshape(3, -1).T).real                           # (P, 3)


def _fd_jacobian(vt, n, pts, h=1e-5):
    """(P, 3, 3): d f_c / d x_e by central differences of _band_field."""
    J = np.zeros((len(pts), 3, 3))
    for e in range(3):
        step = np.zeros(3)
        step[e] = h
        J[:, :, e] = (_band_field(vt, n, pts + step) - _band_field(vt, n, pts - step)) / (2 * h)
    return J


def test_leray_field_is_divergence_free():
    """The field of P v~ has zero divergence at off-grid points, by finite
    differences of the directly summed trigonometric polynomial, while the field
    of v~ does not (catches a wave vector without 1/N_d, a transposed axis, the
    projector applied to the wrong index)."""
    vt = synth.random_coefficients(B_INC, 81, bound=2.0)
    pts = np.random.default_rng(82).uniform(0, 1, (64, 3)) * np.asarray(N_INC)
    div_raw = np.trace(_fd_jacobian(vt, N_INC, pts), axis1=1, axis2=2)
    div_inc = np.trace(_fd_jacobian(O.leray(vt, N_INC), N_INC, pts), axis1=1, axis2=2)
    scale = np.max(np.abs(div_raw))
    assert scale > 0.1
    assert np.max(np.abs(div_inc)) < 1e-8 * scale


def test_leray_is_orthogonal_helmholtz_split():
    """v = P v + (v - P v): P is idempotent and self-adjoint in <.,.>, and the
    removed part is a gradient field (zero curl by finite differences), the
    L2-orthogonal complement of the divergence-free fields."""
    v = synth.random_coefficients(B_INC, 83, bound=2.0)
    w = synth.random_coefficients(B_INC, 84, bound=2.0)
    Pv, Pw = O.leray(v, N_INC), O.leray(w, N_INC)
    assert rel(O.leray(Pv, N_INC), Pv) < 1e-14
    assert abs(O.inner(Pv, w) - O.inner(v, Pw)) < 1e-12 * np.linalg.norm(v) * np.linalg.norm(w)
    assert abs(O.inner(v - Pv, Pw)) < 1e-12 * np.linalg.norm(v) * np.linalg.norm(w)
    pts = np.random.default_rng(85).uniform(0, 1, (48, 3)) * np.asarray(N_INC)
    J = _fd_jacobian(v - Pv, N_INC, pts)
    curl = np.stack([J[:, 2, 1] - J[:, 1, 2], J[:, 0, 2] - J[:, 2, 0], J[:, 1, 0] - J[:, 0, 1]])
    Jv = _fd_jacobian(v, N_INC, pts)
    assert np.max(np.abs(curl)) < 1e-8 * np.max(np.abs(Jv))
    # the zero frequency (a constant field) is divergence-free and kept
    c = np.zeros((3,) + B_INC, complex)
    c[(slice(None),) + tuple(b // 2 for b in B_INC)] = [1.0, -2.0, 0.5j]
    assert rel(O.leray(c, N_INC), c) < 1e-15


def test_incompressible_departure_jacobian_is_one_to_second_order():
    """With a divergence-free velocity, det(I + grad d) of the step map
    x -> x + d(x), d = -dt iota(P v~), differs from 1 only at second order in dt
    (halving dt divides the deviation by 4), while a compressible velocity
    deviates at first order (by 2): the Jacobians stay 1."""
    vt = synth.random_coefficients(B_INC, 86, bound=2.0)
    pts = np.random.default_rng(87).uniform(0, 1, (64, 3)) * np.asarray(N_INC)
    dev = {}
    for name, v in (("inc", O.leray(vt, N_INC)), ("comp", vt)):
        G = _fd_jacobian(v, N_INC, pts)
        for dt in (0.1, 0.05):
            det = np.linalg.det(np.eye(3)[None] - dt * G)
            dev[name, dt] = np.max(np.abs(det - 1.0))
    assert 3.5 < dev["inc", 0.1] / dev["inc", 0.05] < 4.5
    assert 1.5 < dev["comp", 0.1] / dev["comp", 0.05] < 2.5
    assert dev["inc", 0.1] < 0.2 * dev["comp", 0.1]


def _kink_free_inc(vt, dvt, eps, p):
    lo = np.floor(O.displacement(O.leray(vt - eps * dvt, p.n), p))
    hi = np.floor(O.displacement(O.leray(vt + eps * dvt, p.n), p))
    return np.array_equal(lo, hi)


def test_incompressible_gradient_matches_finite_differences():
    """E(P v~) with the H^1 regulariser (s = 1/2): the gradient P grad E(P v~)
    against central differences along unprojected random directions
    (catches a projection missing on the input, the output or the regulariser)."""
    p = O.Params(n=(12, 12, 10), band=(6, 4, 6), nt=6, s=0.5, incompressible=True)
    I0, I1, _ = synth.blob_pair(p.n, 88, max_disp=2.0)
    vt = synth.random_coefficients(p.band, 89, bound=2.5)
    g, _, _ = O.Point(vt, I0, I1, p).gradient()
    assert rel(O.leray(g, p.n), g) < 1e-14
    eps = 1e-6
    checked = 0
    for s in range(24):
        dvt = synth.random_direction(p.band, 900 + s)
        if not _kink_free_inc(vt, dvt, eps, p):
            continue
        fd = (O.energy(vt + eps * dvt, I0, I1, p) - O.energy(vt - eps * dvt, I0, I1, p)) / (2 * eps)
        dd = O.inner(g, dvt)
        assert abs(fd - dd) <= 1e-6 * abs(dd), (s, fd, dd)
        checked += 1
        if checked == 8:
            break
    assert checked == 8


def test_incompressible_gn_hessian():
    """P H P: symmetric, positive on divergence-free directions, zero on gradient
    fields, with range in the divergence-free fields; at zero residual it is the
    central difference of the incompressible gradient."""
    p = O.Params(n=(12, 10, 12), band=(4, 4, 6), nt=5, s=0.5, incompressible=True)
    I0, _, _ = synth.blob_pair(p.n, 91, max_disp=2.0)
    vt = synth.random_coefficients(p.band, 92, bound=2.0)
    I1 = O.Point(vt, I0, I0, p).m[-1]
    pt = O.Point(vt, I0, I1, p)
    v = synth.random_direction(p.band, 93)
    w = synth.random_direction(p.band, 94)
    Hv, Hw = pt.gn_hessvec(v)[0], pt.gn_hessvec(w)[0]
    a, b = O.inner(Hv, w), O.inner(v, Hw)
    assert abs(a - b) <= 1e-10 * max(abs(a), abs(b))
    assert O.inner(Hv, v) > 0.0
    assert rel(O.leray(Hv, p.n), Hv) < 1e-14
    grad_part = v - O.leray(v, p.n)
    assert np.linalg.norm(pt.gn_hessvec(grad_part)[0]) < 1e-12 * np.linalg.norm(Hv)
    eps = 1e-6
    checked = 0
    for s in range(6):
        dvt = synth.random_direction(p.band, 950 + s)
        if not _kink_free_inc(vt, dvt, eps, p):
            continue
        gp = O.Point(vt + eps * dvt, I0, I1, p).gradient()[0]
        gm = O.Point(vt - eps * dvt, I0, I1, p).gradient()[0]
        assert rel(pt.gn_hessvec(dvt)[0], (gp - gm) / (2 * eps)) < 1e-6
        checked += 1
    assert checked >= 2


def test_incompressible_newton_stays_divergence_free():
    p = O.Params(n=(16, 16, 16), band=(4, 4, 4), nt=5, s=0.5, incompressible=True)
    I0, I1, _ = synth.blob_pair(p.n, 95, max_disp=2.0)
    rep = O.newton(np.zeros((3,) + p.band, complex), I0, I1, p, max_newton=3, max_pcg=8,
                   gtol=1e-6)
    assert rep.iterations >= 2
    assert all(b < a for a, b in zip(rep.energies, rep.energies[1:]))
    assert rel(O.leray(rep.vt, p.n), rep.vt) < 1e-13


# ----------------------------------------------------------------------------
# Full Newton Hessian (Eqs. 44-46 without the drops of Section 3.4)
# ----------------------------------------------------------------------------


def test_full_hessian_is_fd_of_gradient():
    """Away from a minimum (sigma = 0.5, large residual) the full Hessian equals
    central differences of the gradient to 1e-7, while the Gauss-Newton one is
    off by more than 1e-3.  Dropping any one of the three terms that the
    Gauss-Newton step leaves out (pi(lambda grad dm), the variation of S^T, the
    move of the departure point inside its cell) changes the result by more
    than 1e-4, so each is checked."""
    p = O.Params(n=(12, 12, 12), band=(4, 6, 4), nt=5, sigma=0.5)
    I0, I1, _ = synth.blob_pair(p.n, 51, max_disp=2.0)
    vt = synth.random_coefficients(p.band, 52, bound=2.0)
    pt = O.Point(vt, I0, I1, p)
    eps = 1e-6
    checked = 0
    for s in range(8):
        dvt = synth.random_direction(p.band, 1600 + s)
        if not _kink_free(vt, dvt, eps, p):
            continue
        gp = O.Point(vt + eps * dvt, I0, I1, p).gradient()[0]
        gm = O.Point(vt - eps * dvt, I0, I1, p).gradient()[0]
        fd = (gp - gm) / (2 * eps)
        assert rel(pt.full_hessvec(dvt)[0], fd) < 1e-7
        assert rel(pt.gn_hessvec(dvt)[0], fd) > 1e-3
        checked += 1
        if checked == 4:
            break
    assert checked == 4


def test_full_hessian_symmetric_and_gauss_newton_at_zero_residual():
    p = O.Params(n=(16, 16, 16), band=(6, 6, 6), nt=6, sigma=0.5)
    I0, I1, _ = synth.blob_pair(p.n, 1611, max_disp=2.0)
    vt = synth.random_coefficients(p.band, 1612, bound=2.5)
    pt = O.Point(vt, I0, I1, p)
    v = synth.random_direction(p.band, 1613)
    w = synth.random_direction(p.band, 1614)
    a, b = O.inner(pt.full_hessvec(v)[0], w), O.inner(v, pt.full_hessvec(w)[0])
    assert abs(a - b) <= 1e-10 * max(abs(a), abs(b))
    # zero residual: lambda = 0, so the extra terms vanish
    pt0 = O.Point(vt, I0, pt.m[-1], p)
    assert rel(pt0.full_hessvec(v)[0], pt0.gn_hessvec(v)[0]) < 1e-13


def test_full_hessian_equals_dense_fd_hessian_bruteforce():
    """8^3 grid, band 4^3 (384 real parameters): the dense Hessian from central
    differences of the gradient, one parameter at a time, against the
    Hessian-vector product on random directions."""
    p = O.Params(n=(8, 8, 8), band=(4, 4, 4), nt=3, sigma=0.5)
    I0, I1, _ = synth.blob_pair(p.n, 1621, max_disp=1.5)
    for seed in range(1622, 1680):
        vt = synth.random_coefficients(p.band, seed, bound=1.2)
        d = O.displacement(vt, p)
        if np.min(np.abs(d - np.round(d))) >= 1e-4:
            break
    else:
        raise AssertionError("no kink-free point")
    pt = O.Point(vt, I0, I1, p)
    P = 2 * 3 * 64
    eps = 1e-6
    H = np.zeros((P, P))
    for j in range(P):
        e = np.zeros(P)
        e[j] = eps
        de = _from_theta(e, vt.shape)
        gp = O.Point(vt + de, I0, I1, p).gradient()[0]
        gm = O.Point(vt - de, I0, I1, p).gradient()[0]
        H[:, j] = _theta((gp - gm) / (2 * eps))
    assert np.max(np.abs(H - H.T)) < 1e-6 * np.max(np.abs(H))
    for s in range(4):
        v = synth.random_direction(p.band, 1690 + s)
        assert rel(_theta(pt.full_hessvec(v)[0]), H @ _theta(v)) < 1e-7


def test_truncated_pcg_on_an_indefinite_hessian():
    """With a weak regulariser the full Hessian is indefinite away from the
    minimum: plain PCG raises, truncated PCG stops at the non-positive curvature
    with a descent direction; with no update made it returns M^-1 rhs."""
    p = O.Params(n=(12, 12, 12), band=(4, 4, 4), nt=5, sigma=1.0, alpha=0.0, gamma=0.1, s=1)
    I0, I1, _ = synth.blob_pair(p.n, 51, max_disp=2.0)
    pt = O.Point(synth.random_coefficients(p.band, 52, bound=2.0), I0, I1, p)
    g = pt.gradient()[0]
    with pytest.raises(O.NegativeCurvature):
        O.pcg(lambda v: pt.full_hessvec(v)[0], -g, 1.0 / pt.A[None], 1e-10, 60)
    x, its, _ = O.pcg(lambda v: pt.full_hessvec(v)[0], -g, 1.0 / pt.A[None], 1e-10, 60,
                      truncate=True)
    assert 1 <= its < 60
    assert O.inner(g, x) < 0.0
    Minv = 1.0 / pt.A[None]
    x0, its0, _ = O.pcg(lambda v: -v, -g, Minv, 1e-10, 5, truncate=True)
    assert its0 == 0 and rel(x0, -Minv * g) == 0.0


def test_full_newton_decreases_energy():
    p = O.Params(n=(16, 16, 16), band=(4, 4, 4), nt=5)
    I0, I1, _ = synth.blob_pair(p.n, 71, max_disp=2.0)
    rep = O.newton(np.zeros((3,) + p.band, complex), I0, I1, p, max_newton=4, max_pcg=8,
                   gtol=1e-6, hessian="full")
    assert rep.iterations >= 3
    assert all(b < a for a, b in zip(rep.energies, rep.energies[1:]))
    assert rep.grad_inf_rel < 0.5


# ----------------------------------------------------------------------------
# Non-stationary velocity (one band-limited velocity per time step)
# ----------------------------------------------------------------------------


def test_nonstationary_constant_in_time_reduces_to_stationary():
    """With v~^n = v~ for every step the energy is the stationary one, and the
    per-step gradients and HVPs (constant direction) sum to the stationary
    gradient and HVP (catches a missing dt in the regulariser, a step index off
    by one in the body force or the incremental state)."""
    ps = O.Params(n=(12, 10, 14), band=(4, 4, 6), nt=5, sigma=0.7)
    pn = O.Params(n=ps.n, band=ps.band, nt=ps.nt, sigma=ps.sigma, stationary=False)
    I0, I1, _ = synth.blob_pair(ps.n, 1701, max_disp=2.0)
    vt = synth.random_coefficients(ps.band, 1702, bound=2.5)
    dvt = synth.random_direction(ps.band, 1703)
    a = O.Point(vt, I0, I1, ps)
    b = O.Point(np.stack([vt] * ps.nt), I0, I1, pn)
    assert abs(a.energy - b.energy) < 1e-12 * a.energy
    assert rel(b.gradient()[0].sum(axis=0), a.gradient()[0]) < 1e-12
    assert rel(b.gn_hessvec(np.stack([dvt] * ps.nt))[0].sum(axis=0), a.gn_hessvec(dvt)[0]) < 1e-12


def test_nonstationary_single_step_velocity_is_exact_shift():
    """Only step 1 moves, by a constant displacement of (1, -1, 0) voxels (a hair
    inside the cell): m^1 = I0, and m^2 = m^nt is I0 shifted by exactly that
    vector (catches steps taken in the wrong order or with another step's
    velocity)."""
    n, band, nt = (8, 6, 10), (4, 4, 4), 4
    p = O.Params(n=n, band=band, nt=nt, stationary=False)
    I0 = np.random.default_rng(1704).normal(size=n)
    vt = np.zeros((nt, 3) + band, complex)
    centre = tuple(b // 2 for b in band)
    shift = (1, -1, 0)
    for c in range(3):
        vt[(1, c) + centre] = -shift[c] / p.dt * 0.999999999999   # d = shift (just inside the cell)
    pt = O.Point(vt, I0, I0, p)
    want = np.roll(I0, shift=[-s for s in shift], axis=(0, 1, 2))
    assert np.max(np.abs(pt.m[1] - I0)) == 0.0
    assert np.max(np.abs(pt.m[2] - want)) < 1e-9
    assert np.max(np.abs(pt.m[-1] - want)) < 1e-9


def _kink_free_nst(vt, dvt, eps, p):
    lo = np.floor(O.per_step(lambda v: O.displacement(v, p), vt - eps * dvt, p))
    hi = np.floor(O.per_step(lambda v: O.displacement(v, p), vt + eps * dvt, p))
    return np.array_equal(lo, hi)


def test_nonstationary_gradient_matches_finite_differences():
    p = O.Params(n=(12, 12, 12), band=(4, 6, 4), nt=4, stationary=False)
    I0, I1, _ = synth.blob_pair(p.n, 1705, max_disp=2.0)
    vt = np.stack([synth.random_coefficients(p.band, 1710 + n, bound=2.5) for n in range(p.nt)])
    g = O.Point(vt, I0, I1, p).gradient()[0]
    eps = 1e-6
    checked = 0
    for s in range(24):
        dvt = np.stack([synth.random_direction(p.band, 1800 + 10 * s + n) for n in range(p.nt)])
        if not _kink_free_nst(vt, dvt, eps, p):
            continue
        fd = (O.energy(vt + eps * dvt, I0, I1, p) - O.energy(vt - eps * dvt, I0, I1, p)) / (2 * eps)
        dd = O.inner(g, dvt)
        assert abs(fd - dd) <= 1e-6 * abs(dd), (s, fd, dd)
        checked += 1
        if checked == 8:
            break
    assert checked == 8


def test_nonstationary_gn_hessian():
    """Symmetric, positive, and the FD of the gradient at zero residual."""
    p = O.Params(n=(12, 10, 12), band=(4, 4, 6), nt=4, stationary=False)
    I0, _, _ = synth.blob_pair(p.n, 1720, max_disp=2.0)
    vt = np.stack([synth.random_coefficients(p.band, 1721 + n, bound=2.0) for n in range(p.nt)])
    I1 = O.Point(vt, I0, I0, p).m[-1]
    pt = O.Point(vt, I0, I1, p)
    v = np.stack([synth.random_direction(p.band, 1730 + n) for n in range(p.nt)])
    w = np.stack([synth.random_direction(p.band, 1740 + n) for n in range(p.nt)])
    Hv, Hw = pt.gn_hessvec(v)[0], pt.gn_hessvec(w)[0]
    a, b = O.inner(Hv, w), O.inner(v, Hw)
    assert abs(a - b) <= 1e-10 * max(abs(a), abs(b))
    assert O.inner(Hv, v) > 0.0
    eps = 1e-6
    checked = 0
    for s in range(6):
        dvt = np.stack([synth.random_direction(p.band, 1750 + 10 * s + n) for n in range(p.nt)])
        if not _kink_free_nst(vt, dvt, eps, p):
            continue
        gp = O.Point(vt + eps * dvt, I0, I1, p).gradient()[0]
        gm = O.Point(vt - eps * dvt, I0, I1, p).gradient()[0]
        assert rel(pt.gn_hessvec(dvt)[0], (gp - gm) / (2 * eps)) < 1e-6
        checked += 1
    assert checked >= 2


def test_nonstationary_newton_decreases_energy():
    p = O.Params(n=(16, 16, 16), band=(4, 4, 4), nt=4, stationary=False)
    I0, I1, _ = synth.blob_pair(p.n, 71, max_disp=2.0)
    rep = O.newton(np.zeros((p.nt, 3) + p.band, complex), I0, I1, p, max_newton=4,
                   max_pcg=8, gtol=1e-6)
    assert rep.iterations >= 3
    assert all(b < a for a, b in zip(rep.energies, rep.energies[1:]))
    assert rep.grad_inf_rel < 0.5


# ----------------------------------------------------------------------------
# Deformation-state-equation variant (Section 2.3, Eqs. 16-18)
# ----------------------------------------------------------------------------


def _kink_free_def(vt, dvt, eps, p):
    """No cell change in the step stencil nor in the final warp between v -+ eps dv."""
    a = O.DeformationPoint(vt - eps * dvt, np.zeros(p.n), np.zeros(p.n), p)
    b = O.DeformationPoint(vt + eps * dvt, np.zeros(p.n), np.zeros(p.n), p)
    return (np.array_equal(np.floor(a.d), np.floor(b.d)) and
            np.array_equal(np.floor(a.u[-1]), np.floor(b.u[-1])))


def test_deformation_constant_velocity_is_exact_shift():
    """A constant velocity moving 1 voxel per step (a hair less) along axes 0
    and 2: u^nt = nt d, and m(1) is I0 shifted by nt voxels on those axes,
    as in the image variant (catches a missing + d in the deformation step or a
    wrong warp)."""
    n, band, nt = (10, 8, 12), (4, 4, 4), 3
    I0 = np.random.default_rng(1901).normal(size=n)
    vt = np.zeros((3,) + band, complex)
    centre = tuple(b // 2 for b in band)
    vt[(0,) + centre] = -0.999999999999 * nt     # d_0 = 0.999999999999
    vt[(2,) + centre] = 0.999999999999 * nt      # d_2 = -0.999999999999
    for state in ("deformation", "image"):
        p = O.Params(n=n, band=band, nt=nt, state=state)
        pt = O.make_point(vt, I0, I0, p)
        m1 = pt.m1 if state == "deformation" else pt.m[-1]
        want = np.roll(I0, shift=(-nt, 0, nt), axis=(0, 1, 2))
        assert np.max(np.abs(m1 - want)) < 1e-9, state
    assert np.max(np.abs(pt.energy_reg)) > 0


def test_deformation_gradient_matches_finite_differences():
    p = O.Params(n=(12, 12, 12), band=(4, 6, 4), nt=5, state="deformation")
    I0, I1, _ = synth.blob_pair(p.n, 1911, max_disp=2.0)
    vt = synth.random_coefficients(p.band, 1912, bound=2.5)
    g = O.DeformationPoint(vt, I0, I1, p).gradient()[0]
    eps = 1e-6
    checked = 0
    for s in range(24):
        dvt = synth.random_direction(p.band, 1920 + s)
        if not _kink_free_def(vt, dvt, eps, p):
            continue
        fd = (O.energy(vt + eps * dvt, I0, I1, p) - O.energy(vt - eps * dvt, I0, I1, p)) / (2 * eps)
        dd = O.inner(g, dvt)
        assert abs(fd - dd) <= 1e-6 * abs(dd), (s, fd, dd)
        checked += 1
        if checked == 8:
            break
    assert checked == 8


def test_deformation_gn_hessian():
    """Symmetric, positive, the FD of the gradient at zero residual, and A +
    (2/sigma^2) J^T J with J = dm(1)/dtheta from central differences (8^3, 384
    parameters)."""
    p = O.Params(n=(12, 10, 12), band=(4, 4, 6), nt=4, state="deformation")
    I0, _, _ = synth.blob_pair(p.n, 1931, max_disp=2.0)
    vt = synth.random_coefficients(p.band, 1932, bound=2.0)
    I1 = O.DeformationPoint(vt, I0, I0, p).m1
    pt = O.DeformationPoint(vt, I0, I1, p)
    v = synth.random_direction(p.band, 1933)
    w = synth.random_direction(p.band, 1934)
    Hv, Hw = pt.gn_hessvec(v)[0], pt.gn_hessvec(w)[0]
    a, b = O.inner(Hv, w), O.inner(v, Hw)
    assert abs(a - b) <= 1e-10 * max(abs(a), abs(b))
    assert O.inner(Hv, v) > 0.0
    eps = 1e-6
    checked = 0
    for s in range(6):
        dvt = synth.random_direction(p.band, 1940 + s)
        if not _kink_free_def(vt, dvt, eps, p):
            continue
        gp = O.DeformationPoint(vt + eps * dvt, I0, I1, p).gradient()[0]
        gm = O.DeformationPoint(vt - eps * dvt, I0, I1, p).gradient()[0]
        assert rel(pt.gn_hessvec(dvt)[0], (gp - gm) / (2 * eps)) < 1e-6
        checked += 1
    assert checked >= 2

    q = O.Params(n=(8, 8, 8), band=(4, 4, 4), nt=3, sigma=0.7, state="deformation")
    J0, J1, _ = synth.blob_pair(q.n, 1951, max_disp=1.5)
    # a point whose step and final displacements keep >= 1e-5 voxel from every
    # cell boundary: a 1e-6 change of one coefficient moves them by less
    for seed in range(1952, 2300):
        vq = synth.random_coefficients(q.band, seed, bound=1.2)
        dq = O.DeformationPoint(vq, J0, J1, q)
        if (np.min(np.abs(dq.d - np.round(dq.d))) >= 1e-5 and
                np.min(np.abs(dq.u[-1] - np.round(dq.u[-1]))) >= 1e-5):
            break
    else:
        raise AssertionError("no kink-free point")
    P = 2 * 3 * 64
    J = np.zeros((int(np.prod(q.n)), P))
    for j in range(P):
        e = np.zeros(P)
        e[j] = 1e-6
        de = _from_theta(e, vq.shape)
        J[:, j] = ((O.DeformationPoint(vq + de, J0, J1, q).m1 -
                    O.DeformationPoint(vq - de, J0, J1, q).m1) / 2e-6).ravel()
    A = O.regulariser_weights(q)
    H = np.diag(np.concatenate([np.tile(A.ravel(), 3)] * 2)) + (2.0 / q.sigma**2) * J.T @ J
    for s in range(3):
        v = synth.random_direction(q.band, 2020 + s)
        assert rel(_theta(dq.gn_hessvec(v)[0]), H @ _theta(v)) < 1e-7


def test_deformation_newton_decreases_energy():
    p = O.Params(n=(16, 16, 16), band=(4, 4, 4), nt=5, state="deformation")
    I0, I1, _ = synth.blob_pair(p.n, 71, max_disp=2.0)
    rep = O.newton(np.zeros((3,) + p.band, complex), I0, I1, p, max_newton=4, max_pcg=8,
                   gtol=1e-6)
    assert rep.iterations >= 3
    assert all(b < a for a, b in zip(rep.energies, rep.energies[1:]))
    assert rep.grad_inf_rel < 0.5


def test_form_combinations_match_finite_differences():
    """The forms compose: the incompressible H^1 form with non-stationary
    velocities and with the deformation state equation, each gradient against
    central differences of its own energy (4 directions)."""
    cases = [
        O.Params(n=(12, 10, 12), band=(4, 4, 6), nt=3, s=0.5, incompressible=True,
                 stationary=False),
        O.Params(n=(12, 10, 12), band=(4, 4, 6), nt=4, s=0.5, incompressible=True,
                 state="deformation"),
    ]
    for k, p in enumerate(cases):
        I0, I1, _ = synth.blob_pair(p.n, 2101 + k, max_disp=2.0)
        shape = ((p.nt,) if not p.stationary else ()) + (3,) + p.band
        rng = np.random.default_rng(2110 + k)
        vt = (rng.normal(size=shape) + 1j * rng.normal(size=shape)) * 0.3
        g = O.make_point(vt, I0, I1, p).gradient()[0]
        eps = 1e-6
        checked = 0
        for s in range(12):
            dvt = rng.normal(size=shape) + 1j * rng.normal(size=shape)
            a = O.make_point(vt - eps * dvt, I0, I1, p)
            b = O.make_point(vt + eps * dvt, I0, I1, p)
            cells = [(np.floor(a.d), np.floor(b.d))]
            if p.state == "deformation":
                cells.append((np.floor(a.u[-1]), np.floor(b.u[-1])))
            if not all(np.array_equal(x, y) for x, y in cells):
                continue
            fd = (b.energy - a.energy) / (2 * eps)
            dd = O.inner(g, dvt)
            assert abs(fd - dd) <= 1e-6 * abs(dd), (k, s, fd, dd)
            checked += 1
            if checked == 4:
                break
        assert checked == 4, k


def test_nonstationary_gn_hessian_equals_dense_jacobian_bruteforce():
    """8^3 grid, band 4^3, two steps (768 real parameters): H = dt A (per step) +
    (2/sigma^2) J^T J with J = dm^nt/dtheta from central differences of the
    state, against the per-step incremental state / adjoint chain."""
    p = O.Params(n=(8, 8, 8), band=(4, 4, 4), nt=2, sigma=0.7, stationary=False)
    I0, I1, _ = synth.blob_pair(p.n, 2201, max_disp=1.5)
    for seed in range(2202, 2400):
        vt = np.stack([synth.random_coefficients(p.band, seed + 500 * n, bound=1.2)
                       for n in range(p.nt)])
        d = O.per_step(lambda v: O.displacement(v, p), vt, p)
        if np.min(np.abs(d - np.round(d))) >= 1e-5:
            break
    else:
        raise AssertionError("no kink-free point")
    pt = O.Point(vt, I0, I1, p)
    P = 2 * p.nt * 3 * 64
    J = np.zeros((int(np.prod(p.n)), P))
    for j in range(P):
        e = np.zeros(P)
        e[j] = 1e-6
        de = _from_theta(e, vt.shape)
        J[:, j] = ((O.Point(vt + de, I0, I1, p).m[-1] - O.Point(vt - de, I0, I1, p).m[-1])
                   / 2e-6).ravel()
    A = O.regulariser_weights(p)
    Ad = np.concatenate([np.tile(p.dt * A.ravel(), 3 * p.nt)] * 2)
    H = np.diag(Ad) + (2.0 / p.sigma**2) * J.T @ J
    for s in range(3):
        v = np.stack([synth.random_direction(p.band, 2450 + 10 * s + n) for n in range(p.nt)])
        assert rel(_theta(pt.gn_hessvec(v)[0]), H @ _theta(v)) < 1e-7


def test_deformation_full_hessian():
    """The deformation variant's full Newton Hessian: central differences of the
    gradient to 1e-7 away from a minimum (Gauss-Newton off by more than 1e-3),
    symmetric, equal to Gauss-Newton at zero residual, and a full Newton run
    decreases the energy."""
    p = O.Params(n=(12, 12, 12), band=(4, 6, 4), nt=5, sigma=0.5, state="deformation")
    I0, I1, _ = synth.blob_pair(p.n, 2301, max_disp=2.0)
    vt = synth.random_coefficients(p.band, 2302, bound=2.0)
    pt = O.DeformationPoint(vt, I0, I1, p)
    eps = 1e-6
    checked = 0
    for s in range(12):
        dvt = synth.random_direction(p.band, 2310 + s)
        if not _kink_free_def(vt, dvt, eps, p):
            continue
        gp = O.DeformationPoint(vt + eps * dvt, I0, I1, p).gradient()[0]
        gm = O.DeformationPoint(vt - eps * dvt, I0, I1, p).gradient()[0]
        fd = (gp - gm) / (2 * eps)
        assert rel(pt.full_hessvec(dvt)[0], fd) < 1e-7
        assert rel(pt.gn_hessvec(dvt)[0], fd) > 1e-3
        checked += 1
        if checked == 3:
            break
    assert checked == 3
    v = synth.random_direction(p.band, 2330)
    w = synth.random_direction(p.band, 2331)
    a, b = O.inner(pt.full_hessvec(v)[0], w), O.inner(v, pt.full_hessvec(w)[0])
    assert abs(a - b) <= 1e-10 * max(abs(a), abs(b))
    pt0 = O.DeformationPoint(vt, I0, pt.m1, p)
    assert rel(pt0.full_hessvec(v)[0], pt0.gn_hessvec(v)[0]) < 1e-13
    q = O.Params(n=(16, 16, 16), band=(4, 4, 4), nt=5, state="deformation")
    J0, J1, _ = synth.blob_pair(q.n, 71, max_disp=2.0)
    rep = O.newton(np.zeros((3,) + q.band, complex), J0, J1, q, max_newton=3, max_pcg=8,
                   gtol=1e-6, hessian="full")
    assert rep.iterations >= 2
    assert all(y < x for x, y in zip(rep.energies, rep.energies[1:]))
