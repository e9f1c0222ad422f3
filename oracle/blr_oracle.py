"""Plain FP64 CPU oracle for band-limited PDE-LDDMM (state-equation variant) with
Gauss-Newton-Krylov optimisation.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct reference
that the CUDA library is compared against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import it.  The product path (``paper_1807_05117_gb300``) never imports it, and
this module imports nothing from the product.

What is computed (Hernandez, "Newton-Krylov optimization in PDE-constrained
diffeomorphic registration parameterized in the space of band-limited vector
fields", arXiv 1807.05117):

* band-limited space: inclusion iota and projection pi (Section 3.1, Eq. 33);
* regulariser / preconditioner diagonal in the band (Section 3.1, Eq. 34, with
  Eq. 1's operator family): A(k) = (alpha*omega(k) + gamma)^(2s), K~ = 1/A;
* energy E(v~) = 1/2 <L~v~, v~> + sigma^-2 ||m(1) - I1||^2 (Section 3.2, Eq. 35)
  subject to the state equation d_t m + grad m . iota(v~) = 0, m(0) = I0
  (Eq. 36, Section 2.2 Eq. 5);
* gradient  g~ = L~v~ + pi(lambda grad m)  (Section 3.2, Eq. 38; adjoint
  equation Eq. 8 and its final condition lambda(1) = -(2/sigma^2)(m(1)-I1),
  Section 2.2);
* Gauss-Newton Hessian-vector product H~dv~ = L~dv~ + pi(dlambda grad m) with
  the Gauss-Newton drops of Section 3.4 applied to Eq. 46;
* the full Newton Hessian-vector product (Eqs. 44-46 without those drops):
  the exact second derivative of the discrete energy;
* PCG with preconditioner K~ and the reduced-space Newton update with a step
  length (Section 3.4, Eqs. 54-55; Section 2.4, Eqs. 31-32);
* the non-stationary parameterisation (one band-limited velocity v~^n per time
  step, the time-varying v~_t of Section 3.2 and of the NSt. experiments): the
  regulariser is the time integral 1/2 dt sum_n <L~ v~^n, v~^n>, and the
  gradient and Hessian are taken per step;
* the deformation-state-equation variant (Section 2.3, Eqs. 16-18; its
  band-limited form in Section 3.3): the deformation phi = id + u is transported,
  u^0 = 0, u^{n+1} = S u^n + d, and the template is warped once,
  m(1) = T[I0](x + u^nt); the adjoint rho (a vector field) starts from
  rho^nt = lambda(1) grad T[I0](x + u^nt) and runs backwards with S^T; the body
  force is dt sum_n (rho^{n+1} + D u^n^T rho^{n+1}); Gauss-Newton and full
  Newton Hessians;
* the incompressible form (Eq. 4 with gamma = 1, imposed in the band as in
  Section 3.2): the velocity is restricted to divergence-free band fields by the
  Fourier-diagonal Leray projector P(k) = I - kappa kappa^T / |kappa|^2,
  kappa_d = 2 pi k_d / N_d; the energy is E(P v~), so the gradient is
  P grad E(P v~) and the Hessian P H P.

The paper states the continuous equations only (optimise-then-discretise).  The
oracle fixes one discretisation and differentiates it exactly
(discretise-then-optimise), so that finite differences and Hessian symmetry hold
to rounding:

* time: nt stationary steps, dt = 1/nt, semi-Lagrangian first-order departure
  point x + d(x) with d = -dt * iota(v~) (voxel units, h = 1);
* space: trilinear interpolation with periodic wrap; the interpolation cell of
  voxel x on axis a is x_a + floor(d_a(x)), so the cell depends on the
  displacement only;
* the transport step is the sparse linear map S (8 weights per row), its exact
  transpose S^T gives the adjoint step, and D_a holds the exact partial
  derivatives of the trilinear polynomial inside the chosen cell;
* frequencies are centred: k_d in {-B_d/2, ..., B_d/2 - 1}; iota takes the real
  part of the sum; pi = iota^T under <a, b> = Re sum(a * conj(b));
* omega(k) is the symbol of the periodic 7-point Laplacian with h = 1;
* a Newton trial point whose displacement reaches one voxel per step on some
  axis (the CFL bound of Section 2.4) is rejected by the line search.

Every function works in float64 / complex128.  Parity status: every function
here is pinned by ``tests/test_oracle_pins.py`` (brute force, closed forms,
adjoint identities, finite differences, dense solves).
"""

from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------------------
# Problem parameters
# ----------------------------------------------------------------------------


@dataclass(frozen=True)
class Params:
    """Grid, band and model constants.

    n      -- grid (N1, N2, N3); array layout [N1][N2][N3], N3 fastest
    band   -- (B1, B2, B3), each even; centred frequencies -B/2 .. B/2-1
    nt     -- number of time steps (dt = 1/nt)
    alpha, gamma, s -- L = (-alpha*Laplacian + gamma)^s, regulariser L^T L;
              s may be a half-integer (2s integer): s = 1/2 gives the H^1
              regulariser alpha*omega + gamma of the incompressible experiments
    sigma  -- weight of the image term sigma^-2 ||m(1) - I1||^2 (Eq. 35)
    incompressible -- restrict v~ to divergence-free band fields (Eq. 4, gamma = 1)
    stationary -- one velocity for all steps, coefficients (3, B1, B2, B3); else one
              per step, (nt, 3, B1, B2, B3), step n transported by v~^n
    state  -- "image" (the state equation) or "deformation" (the deformation state
              equation: u = phi - id is transported, I0 warped once at the end)
    """

    n: tuple
    band: tuple
    nt: int = 10
    alpha: float = 3.0
    gamma: float = 1.0
    s: float = 2
    sigma: float = 1.0
    incompressible: bool = False
    stationary: bool = True
    state: str = "image"

    @property
    def dt(self) -> float:
        return 1.0 / self.nt


# ----------------------------------------------------------------------------
# Band-limited space (Section 3.1, Eq. 33)
# ----------------------------------------------------------------------------


def band_frequencies(B: int) -> np.ndarray:
    """Centred integer frequencies -B/2 .. B/2-1 of one axis of the band."""
    return np.arange(B) - B // 2


def dft_matrix(N: int, B: int) -> np.ndarray:
    """E[x, j] = exp(2 pi i k_j x / N) for voxel x and band frequency k_j."""
    x = np.arange(N)
    k = band_frequencies(B)
    phase = np.outer(x, k) % N  # exact integer phase, reduced mod N
    return np.exp(2j * np.pi * phase / N)


def expand(vt: np.ndarray, n) -> np.ndarray:
    """iota: band coefficients (3, B1, B2, B3) complex -> real field (3, N1, N2, N3).

    iota(v~)_c(x) = Re sum_k v~_c(k) exp(2 pi i sum_d k_d x_d / N_d)   (Eq. 33)
    The exponential factorises over the axes; einsum evaluates the sum.
    """
    E1, E2, E3 = (dft_matrix(n[d], vt.shape[1 + d]) for d in range(3))
    return np.einsum("cabk,xa,yb,zk->cxyz", vt, E1, E2, E3, optimize=True).real


def project(f: np.ndarray, band) -> np.ndarray:
    """pi: real field (3, N1, N2, N3) -> band coefficients (3, B1, B2, B3).

    pi(f)_c(k) = sum_x f_c(x) exp(-2 pi i sum_d k_d x_d / N_d), which is the
    transpose of iota under <a, b> = Re sum a conj(b) (Section 3.1).
    """
    E1, E2, E3 = (dft_matrix(f.shape[1 + d], band[d]).conj() for d in range(3))
    return np.einsum("cxyz,xa,yb,zk->cabk", f, E1, E2, E3, optimize=True)


def inner(a: np.ndarray, b: np.ndarray) -> float:
    """Real inner product of the parameter space R^(2*3*B1*B2*B3)."""
    return float(np.real(np.vdot(b, a)))


# ----------------------------------------------------------------------------
# Regulariser (Eq. 1 operator family, Section 3.1 Eq. 34)
# ----------------------------------------------------------------------------


def laplacian_symbol(n, band) -> np.ndarray:
    """omega(k) = sum_d 2 (1 - cos(2 pi k_d / N_d)): eigenvalue of the periodic
    7-point negative Laplacian (h = 1) on the Fourier mode k."""
    parts = [2.0 * (1.0 - np.cos(2.0 * np.pi * band_frequencies(band[d]) / n[d]))
             for d in range(3)]
    return parts[0][:, None, None] + parts[1][None, :, None] + parts[2][None, None, :]


def regulariser_weights(p: Params) -> np.ndarray:
    """A(k) = (alpha omega(k) + gamma)^(2s): symbol of L^T L, L = (-alpha Lap + gamma)^s.
    The preconditioner K~ = (L^T L)^-1 is 1/A.  2s must be an integer."""
    q = int(round(2 * p.s))
    if q != 2 * p.s or q < 0:
        raise ValueError("2s must be a non-negative integer")
    return (p.alpha * laplacian_symbol(p.n, p.band) + p.gamma) ** q


def regulariser_energy(vt: np.ndarray, A: np.ndarray) -> float:
    """1/2 <L~ v~, v~>_{l2} for a stationary velocity (time integral over [0, 1])."""
    return 0.5 * float(np.sum(A[None] * np.abs(vt) ** 2))


# ----------------------------------------------------------------------------
# Incompressible form (Eq. 4 with gamma = 1, constraint taken in the band)
# ----------------------------------------------------------------------------


def leray_matrices(n, band) -> np.ndarray:
    """(B1, B2, B3, 3, 3) real: P(k) = I - kappa kappa^T / |kappa|^2 with
    kappa_d = 2 pi k_d / N_d, the wave vector of the Fourier mode k on the voxel
    grid (h = 1); P(0) = I.  The divergence of the mode v~(k) e^{i kappa.x} is
    i kappa.v~(k) e^{i kappa.x}, so P(k) v~(k) is the divergence-free part."""
    kap = [2.0 * np.pi * band_frequencies(band[d]) / n[d] for d in range(3)]
    K = np.stack(np.meshgrid(*kap, indexing="ij"), axis=-1)          # (B1, B2, B3, 3)
    k2 = np.sum(K * K, axis=-1)
    outer = K[..., :, None] * K[..., None, :]
    safe = np.where(k2 > 0.0, k2, 1.0)
    return np.eye(3) - np.where(k2[..., None, None] > 0.0, outer / safe[..., None, None], 0.0)


def leray(vt: np.ndarray, n) -> np.ndarray:
    """Apply P(k) to the three components of every band coefficient."""
    Pk = leray_matrices(n, vt.shape[1:])
    return np.einsum("abkcd,dabk->cabk", Pk, vt)


# ----------------------------------------------------------------------------
# Semi-Lagrangian transport operator (state equation, Eq. 36 / Eq. 5)
# ----------------------------------------------------------------------------


def displacement(vt: np.ndarray, p: Params) -> np.ndarray:
    """Per-step displacement d = -dt * iota(v~) in voxels; departure point x + d(x)."""
    return -p.dt * expand(vt, p.n)


def cfl_number(d: np.ndarray) -> float:
    """Largest per-axis displacement per step, in voxels."""
    return float(np.max(np.abs(d))) if d.size else 0.0


class Stencil:
    """Trilinear interpolation at x + d(x) with periodic wrap, as sparse matrices.

    S   -- (S m)(x) = trilinear value of m at x + d(x)
    D_a -- (D_a m)(x) = partial derivative along axis a of the trilinear
           polynomial of the cell used at x (right derivative on a node)
    D2[(a, b)], a < b -- the mixed second partial d_a d_b of that polynomial
           (its pure second partials are zero: it is linear along each axis)
    The cell on axis a is x_a + floor(d_a(x)) and the local coordinate is
    f_a = d_a - floor(d_a); corner o in {0,1}^3 has weight
    prod_a (f_a if o_a else 1 - f_a).
    """

    def __init__(self, d: np.ndarray):
        shape = d.shape[1:]
        V = int(np.prod(shape))
        fl = np.floor(d)
        f = d - fl
        fl = fl.astype(np.int64)
        grid = np.indices(shape)
        rows = np.arange(V)
        w = [[1.0 - f[a], f[a]] for a in range(3)]       # weight of corner bit o_a
        dw = [-1.0, 1.0]                                   # its derivative in p_a
        pairs = ((0, 1), (0, 2), (1, 2))
        cols, vals, dvals = [], [], [[], [], []]
        d2vals = {ab: [] for ab in pairs}
        for o in itertools.product((0, 1), repeat=3):
            idx = [(grid[a] + fl[a] + o[a]) % shape[a] for a in range(3)]
            cols.append(np.ravel_multi_index(idx, shape).ravel())
            vals.append((w[0][o[0]] * w[1][o[1]] * w[2][o[2]]).ravel())
            dvals[0].append((dw[o[0]] * w[1][o[1]] * w[2][o[2]]).ravel())
            dvals[1].append((w[0][o[0]] * dw[o[1]] * w[2][o[2]]).ravel())
            dvals[2].append((w[0][o[0]] * w[1][o[1]] * dw[o[2]]).ravel())
            for a, b in pairs:
                c3 = 3 - a - b
                d2vals[a, b].append((dw[o[a]] * dw[o[b]] * w[c3][o[c3]]).ravel())
        r = np.tile(rows, 8)
        c = np.concatenate(cols)
        self.shape = shape
        self.S = sp.csr_matrix((np.concatenate(vals), (r, c)), shape=(V, V))
        self.D = [sp.csr_matrix((np.concatenate(dv), (r, c)), shape=(V, V))
                  for dv in dvals]
        self.D2 = {ab: sp.csr_matrix((np.concatenate(d2vals[ab]), (r, c)), shape=(V, V))
                   for ab in pairs}

    def apply(self, m: np.ndarray) -> np.ndarray:
        return (self.S @ m.ravel()).reshape(self.shape)

    def apply_transpose(self, lam: np.ndarray) -> np.ndarray:
        return (self.S.T @ lam.ravel()).reshape(self.shape)

    def gradient(self, m: np.ndarray) -> np.ndarray:
        """(3, N1, N2, N3): exact gradient of the interpolant of m at x + d(x)."""
        mf = m.ravel()
        return np.stack([(Da @ mf).reshape(self.shape) for Da in self.D])

    def hessian_times(self, m: np.ndarray, u: np.ndarray) -> np.ndarray:
        """(3, ...): (Hess T[m](x + d(x))) u(x), the second derivatives of the
        cell polynomial of m at the departure point applied to the vector field u."""
        mf = m.ravel()
        out = np.zeros((3,) + self.shape)
        for (a, b), Dab in self.D2.items():
            h = (Dab @ mf).reshape(self.shape)
            out[a] += h * u[b]
            out[b] += h * u[a]
        return out

    def gradient_transpose(self, q: np.ndarray) -> np.ndarray:
        """sum_a D_a^T q_a for a vector field q: the transpose of m -> D m . q."""
        return sum((self.D[a].T @ q[a].ravel()) for a in range(3)).reshape(self.shape)


def state(I0: np.ndarray, st: Stencil, nt: int) -> list:
    """m^0 = I0, m^{n+1} = S m^n, n = 0 .. nt-1.  Returns [m^0, ..., m^nt]."""
    return state_steps(I0, [st] * nt)


def state_steps(I0: np.ndarray, stencils: list) -> list:
    """m^0 = I0, m^{n+1} = S^n m^n with the step's own stencil.  Returns [m^0, ..., m^nt]."""
    m = [np.asarray(I0, dtype=np.float64)]
    for st in stencils:
        m.append(st.apply(m[-1]))
    return m


def per_step(f, x: np.ndarray, p: Params) -> np.ndarray:
    """f applied to the coefficients of each step (the whole array when stationary)."""
    return f(x) if p.stationary else np.stack([f(x[n]) for n in range(p.nt)])


def data_energy(m1: np.ndarray, I1: np.ndarray, p: Params) -> float:
    """sigma^-2 ||m(1) - I1||^2 with the voxel sum as the L2 integral (h = 1)."""
    r = m1 - I1
    return float(np.sum(r * r)) / p.sigma**2


# ----------------------------------------------------------------------------
# Energy, gradient and Gauss-Newton Hessian-vector product (Eqs. 35-38, 44-46)
# ----------------------------------------------------------------------------


class Point:
    """Everything the gradient and the Hessian need at one velocity v~."""

    def __init__(self, vt: np.ndarray, I0: np.ndarray, I1: np.ndarray, p: Params):
        self.p = p
        self.vt = np.asarray(vt, dtype=np.complex128)
        want = (3,) + tuple(p.band) if p.stationary else (p.nt, 3) + tuple(p.band)
        if self.vt.shape != want:
            raise ValueError(f"coefficients of shape {self.vt.shape}, expected {want}")
        if p.incompressible:      # the energy is evaluated at P v~
            self.vt = per_step(lambda v: leray(v, p.n), self.vt, p)
        self.I1 = np.asarray(I1, dtype=np.float64)
        self.A = regulariser_weights(p)
        self.d = per_step(lambda v: displacement(v, p), self.vt, p)
        self.cfl = cfl_number(self.d)
        if p.stationary:
            self.stencils = [Stencil(self.d)] * p.nt
        else:
            self.stencils = [Stencil(self.d[n]) for n in range(p.nt)]
        self.stencil = self.stencils[0]
        self.m = state_steps(I0, self.stencils)
        # 1/2 int_0^1 <L~ v~_t, v~_t> dt: dt sum over the steps when v~ varies
        self.energy_reg = regulariser_energy(self.vt, self.A) * (1.0 if p.stationary else p.dt)
        self.energy_data = data_energy(self.m[-1], self.I1, p)
        self.energy = self.energy_reg + self.energy_data
        self._G = None

    def grad_m(self, n: int) -> np.ndarray:
        """G^n = gradient of the interpolant of m^n at the departure points of step n."""
        if self._G is None:
            self._G = [None] * self.p.nt
        if self._G[n] is None:
            self._G[n] = self.stencils[n].gradient(self.m[n])
        return self._G[n]

    def _assemble(self, v: np.ndarray, b: np.ndarray) -> np.ndarray:
        """A v~ + pi(b) (stationary), or dt A v~^n + pi(b^n) per step; then P."""
        p = self.p
        if p.stationary:
            out = self.A[None] * v + project(b, p.band)
        else:
            out = np.stack([p.dt * self.A[None] * v[n] + project(b[n], p.band)
                            for n in range(p.nt)])
        if p.incompressible:
            out = per_step(lambda x: leray(x, p.n), out, p)
        return out

    def adjoint_states(self) -> list:
        """[lambda^0, ..., lambda^nt] of the gradient's adjoint solve at this point."""
        if getattr(self, "_lams", None) is None:
            lam = -(2.0 / self.p.sigma**2) * (self.m[-1] - self.I1)
            lams = [lam]
            for n in range(self.p.nt - 1, -1, -1):
                lam = self.stencils[n].apply_transpose(lam)
                lams.append(lam)
            self._lams = lams[::-1]
        return self._lams

    def adjoint_chain(self, lam_final: np.ndarray):
        """lambda^n = S^T lambda^{n+1} (discrete adjoint equation, Eq. 8) and the
        body force b = dt sum_{n<nt} lambda^{n+1} G^n (the lambda grad m of Eq. 38);
        non-stationary: one body force per step, b^n = dt lambda^{n+1} G^n.
        Returns (b, lambda^0)."""
        p = self.p
        lam = lam_final
        b = np.zeros((3,) + tuple(p.n)) if p.stationary else np.zeros((p.nt, 3) + tuple(p.n))
        for n in range(p.nt - 1, -1, -1):
            if p.stationary:
                b += p.dt * lam[None] * self.grad_m(n)
            else:
                b[n] = p.dt * lam[None] * self.grad_m(n)
            lam = self.stencils[n].apply_transpose(lam)
        return b, lam

    def gradient(self):
        """g~ = A v~ + pi(b), final condition lambda^nt = -(2/sigma^2)(m^nt - I1);
        non-stationary: g~^n = dt A v~^n + pi(b^n), the derivative in each step's
        coefficients; incompressible: P applied to that.  Returns (g~, b, lambda^0)."""
        lam_final = -(2.0 / self.p.sigma**2) * (self.m[-1] - self.I1)
        b, lam0 = self.adjoint_chain(lam_final)
        return self._assemble(self.vt, b), b, lam0

    def incremental_state(self, dvt: np.ndarray) -> np.ndarray:
        """dm^0 = 0, dm^{n+1} = S dm^n - dt G^n . iota(dv~^n)  (linearised Eq. 36).
        Returns dm^nt."""
        p = self.p
        dv = per_step(lambda v: expand(v, p.n), dvt, p)
        dm = np.zeros(tuple(p.n))
        for n in range(p.nt):
            dvn = dv if p.stationary else dv[n]
            dm = self.stencils[n].apply(dm) - p.dt * np.sum(self.grad_m(n) * dvn, axis=0)
        return dm

    def gn_hessvec(self, dvt: np.ndarray):
        """H~ dv~ = A dv~ + pi(db): incremental adjoint with dlambda^nt =
        -(2/sigma^2) dm^nt, dlambda^n = S^T dlambda^{n+1},
        db = dt sum dlambda^{n+1} G^n.  The Gauss-Newton drops of Section 3.4 remove
        the pi(lambda grad dm) term and the dJ term (all second derivatives of
        the transport).  Incompressible: P H P.  Returns (H dv~, dm^nt, db)."""
        p = self.p
        dvt = np.asarray(dvt, dtype=np.complex128)
        if p.incompressible:
            dvt = per_step(lambda v: leray(v, p.n), dvt, p)
        dm1 = self.incremental_state(dvt)
        dlam_final = -(2.0 / p.sigma**2) * dm1
        db, _ = self.adjoint_chain(dlam_final)
        return self._assemble(dvt, db), dm1, db


    def full_hessvec(self, dvt: np.ndarray):
        """Exact Hessian of the discrete energy (Newton: Eqs. 44-46 without the
        drops of Section 3.4), with dd = -dt iota(dv~):
          dm^0 = 0, dm^{n+1} = S dm^n + G^n . dd             (incremental state)
          dlambda^nt = -(2/sigma^2) dm^nt,
          dlambda^n = S^T dlambda^{n+1} + sum_a D_a^T(dd_a lambda^{n+1})
                      (the variation of S^T: the dJ term of the incremental adjoint)
          db = dt sum_n [dlambda^{n+1} G^n
                         + lambda^{n+1} (D dm^n + Hess T[m^n] dd)]
                      (pi(lambda grad dm), and the move of the departure point
                       inside its cell)
          H dv~ = A dv~ + pi(db);  incompressible: P H P.
        Stationary velocities only.  Returns (H dv~, dm^nt, db)."""
        p, st = self.p, self.stencil
        if not p.stationary:
            raise NotImplementedError("the full Hessian is built for stationary velocities")
        dvt = np.asarray(dvt, dtype=np.complex128)
        if p.incompressible:
            dvt = leray(dvt, p.n)
        dd = -p.dt * expand(dvt, p.n)
        dms = [np.zeros(tuple(p.n))]
        for n in range(p.nt):
            dms.append(st.apply(dms[-1]) + np.sum(self.grad_m(n) * dd, axis=0))
        lams = self.adjoint_states()
        dlam = -(2.0 / p.sigma**2) * dms[-1]
        db = np.zeros((3,) + tuple(p.n))
        for n in range(p.nt - 1, -1, -1):
            lam1 = lams[n + 1]
            dG = st.gradient(dms[n]) + st.hessian_times(self.m[n], dd)
            db += p.dt * (dlam[None] * self.grad_m(n) + lam1[None] * dG)
            dlam = st.apply_transpose(dlam) + st.gradient_transpose(dd * lam1[None])
        h = self.A[None] * dvt + project(db, p.band)
        if p.incompressible:
            h = leray(h, p.n)
        return h, dms[-1], db


class DeformationPoint:
    """The deformation-state-equation variant at one velocity (Section 2.3,
    Eqs. 16-18, with the band-limited velocity of Section 3.3), discretised on
    the same semi-Lagrangian step S as the image variant:
      u^0 = 0, u^{n+1} = S u^n + d            (phi^{n+1}(x) = phi^n(x + d(x)))
      m(1) = T[I0](x + u^nt)                  (trilinear, any displacement, periodic)
      E = 1/2 <A v~, v~> + sigma^-2 ||m(1) - I1||^2.
    Stationary velocity; Gauss-Newton and full Newton Hessians."""

    def __init__(self, vt: np.ndarray, I0: np.ndarray, I1: np.ndarray, p: Params,
                 displacement_factor=None):
        """displacement_factor: None, or an array multiplying the displacement
        elementwise (the tests' probes of how the results respond to a small
        relative change of d)."""
        if not p.stationary:
            raise NotImplementedError("the deformation variant takes a stationary velocity")
        self.p = p
        self.vt = np.asarray(vt, dtype=np.complex128)
        if p.incompressible:
            self.vt = leray(self.vt, p.n)
        self.I0 = np.asarray(I0, dtype=np.float64)
        self.I1 = np.asarray(I1, dtype=np.float64)
        self.A = regulariser_weights(p)
        self.d = displacement(self.vt, p)
        if displacement_factor is not None:
            self.d = self.d * displacement_factor
        self.cfl = cfl_number(self.d)
        self.stencil = Stencil(self.d)
        u = [np.zeros((3,) + tuple(p.n))]
        for _ in range(p.nt):
            u.append(np.stack([self.stencil.apply(u[-1][c]) for c in range(3)]) + self.d)
        self.u = u
        self.warp = Stencil(u[-1])              # T[.](x + u^nt): general displacement
        self.m1 = self.warp.apply(self.I0)
        self.grad_warp = self.warp.gradient(self.I0)   # grad T[I0](x + u^nt)
        self.energy_reg = regulariser_energy(self.vt, self.A)
        self.energy_data = data_energy(self.m1, self.I1, p)
        self.energy = self.energy_reg + self.energy_data
        self._Du = {}

    def grad_u(self, n: int) -> np.ndarray:
        """(3 components c, 3 axes a, ...): D_a u_c^n at the departure points."""
        if n not in self._Du:
            self._Du[n] = np.stack([self.stencil.gradient(self.u[n][c]) for c in range(3)])
        return self._Du[n]

    def _body_force(self, rho_final: np.ndarray) -> np.ndarray:
        """rho^n = S^T rho^{n+1} per component and b_a = dt sum_n (rho_a^{n+1} +
        sum_c rho_c^{n+1} D_a u_c^n), the derivative of u^{n+1} = S u^n + d in d."""
        p = self.p
        rho = rho_final
        b = np.zeros((3,) + tuple(p.n))
        for n in range(p.nt - 1, -1, -1):
            b += p.dt * (rho + np.einsum("c...,ca...->a...", rho, self.grad_u(n)))
            rho = np.stack([self.stencil.apply_transpose(rho[c]) for c in range(3)])
        return b

    def gradient(self):
        """g~ = A v~ + pi(b) with rho^nt = lambda(1) grad T[I0](x + u^nt),
        lambda(1) = -(2/sigma^2)(m(1) - I1).  Returns (g~, b)."""
        lam = -(2.0 / self.p.sigma**2) * (self.m1 - self.I1)
        b = self._body_force(lam[None] * self.grad_warp)
        g = self.A[None] * self.vt + project(b, self.p.band)
        if self.p.incompressible:
            g = leray(g, self.p.n)
        return g, b

    def incremental_state(self, dvt: np.ndarray) -> np.ndarray:
        """du^0 = 0, du^{n+1} = S du^n + (D u^n) dd + dd, dd = -dt iota(dv~);
        returns dm(1) = grad T[I0](x + u^nt) . du^nt."""
        p = self.p
        dd = -p.dt * expand(dvt, p.n)
        du = np.zeros((3,) + tuple(p.n))
        for n in range(p.nt):
            Sdu = np.stack([self.stencil.apply(du[c]) for c in range(3)])
            du = Sdu + np.einsum("ca...,a...->c...", self.grad_u(n), dd) + dd
        return np.sum(self.grad_warp * du, axis=0)

    def gn_hessvec(self, dvt: np.ndarray):
        """A dv~ + pi(db): drho^nt = dlambda(1) grad T[I0](x + u^nt) with
        dlambda(1) = -(2/sigma^2) dm(1); the Gauss-Newton drops of Section 3.4
        remove lambda(1) d(grad m(1)), the D du^T rho term and the variation of
        S^T.  Returns (H dv~, dm(1))."""
        dvt = np.asarray(dvt, dtype=np.complex128)
        if self.p.incompressible:
            dvt = leray(dvt, self.p.n)
        dm1 = self.incremental_state(dvt)
        dlam = -(2.0 / self.p.sigma**2) * dm1
        db = self._body_force(dlam[None] * self.grad_warp)
        h = self.A[None] * dvt + project(db, self.p.band)
        if self.p.incompressible:
            h = leray(h, self.p.n)
        return h, dm1


    def full_hessvec(self, dvt: np.ndarray):
        """Exact Hessian of the discrete energy of this variant (Eqs. 19-21 of
        Section 2.3 without the drops of Section 3.4), with dd = -dt iota(dv~):
          du as in incremental_state;
          drho^nt = dlambda(1) Gw + lambda(1) Hess T[I0](x + u^nt) du^nt,
          drho^n_c = S^T drho^{n+1}_c + sum_a D_a^T (dd_a rho^{n+1}_c),
          db_a = dt sum_n (drho_a^{n+1} + sum_c [drho_c^{n+1} D_a u_c^n
                 + rho_c^{n+1} (D_a du_c^n + (Hess T[u_c^n] dd)_a)]).
        Incompressible: P H P.  Returns (H dv~, dm(1))."""
        p, st = self.p, self.stencil
        dvt = np.asarray(dvt, dtype=np.complex128)
        if p.incompressible:
            dvt = leray(dvt, p.n)
        dd = -p.dt * expand(dvt, p.n)
        dus = [np.zeros((3,) + tuple(p.n))]
        for n in range(p.nt):
            Sdu = np.stack([st.apply(dus[-1][c]) for c in range(3)])
            dus.append(Sdu + np.einsum("ca...,a...->c...", self.grad_u(n), dd) + dd)
        lam = -(2.0 / p.sigma**2) * (self.m1 - self.I1)
        dm1 = np.sum(self.grad_warp * dus[-1], axis=0)
        dlam = -(2.0 / p.sigma**2) * dm1
        rho = lam[None] * self.grad_warp
        drho = dlam[None] * self.grad_warp + lam[None] * self.warp.hessian_times(self.I0, dus[-1])
        rhos = [rho]
        for n in range(p.nt - 1, 0, -1):      # rho^n for n = nt-1 .. 1
            rho = np.stack([st.apply_transpose(rho[c]) for c in range(3)])
            rhos.append(rho)
        rhos = rhos[::-1]                     # rhos[n - 1] = rho^n, n = 1 .. nt
        db = np.zeros((3,) + tuple(p.n))
        for n in range(p.nt - 1, -1, -1):
            rho1 = rhos[n]
            Du = self.grad_u(n)
            dDu = np.stack([st.gradient(dus[n][c]) + st.hessian_times(self.u[n][c], dd)
                            for c in range(3)])
            db += p.dt * (drho + np.einsum("c...,ca...->a...", drho, Du)
                          + np.einsum("c...,ca...->a...", rho1, dDu))
            drho = np.stack([st.apply_transpose(drho[c]) + st.gradient_transpose(dd * rho1[c][None])
                             for c in range(3)])
        h = self.A[None] * dvt + project(db, p.band)
        if p.incompressible:
            h = leray(h, p.n)
        return h, dm1


def make_point(vt, I0, I1, p: Params):
    """The point of the chosen state equation (Point or DeformationPoint)."""
    return DeformationPoint(vt, I0, I1, p) if p.state == "deformation" else Point(vt, I0, I1, p)


def energy(vt, I0, I1, p: Params) -> float:
    return make_point(vt, I0, I1, p).energy


# ----------------------------------------------------------------------------
# Krylov solver and reduced-space Newton (Section 3.4, Eqs. 54-55)
# ----------------------------------------------------------------------------


class NegativeCurvature(RuntimeError):
    pass


def pcg(apply_H, rhs: np.ndarray, Minv: np.ndarray, eta: float, maxit: int,
        truncate: bool = False):
    """Preconditioned CG on H x = rhs from x = 0 with M^-1 = K~ (elementwise Minv).
    Stops when ||r_j|| <= eta ||r_0|| or after maxit iterations.
    <p, Hp> <= 0 raises NegativeCurvature, or with truncate (the full Newton
    Hessian, which can be indefinite away from a minimum, Section 3.4) ends the
    solve: the iterate so far, or the first direction M^-1 rhs when no update
    was made (truncated Newton-CG; both are descent directions for rhs = -g).
    Returns (x, iterations, ||r|| / ||r_0||)."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    r0 = np.sqrt(inner(r, r))
    if r0 == 0.0:
        return x, 0, 0.0
    z = Minv * r
    p = z.copy()
    rz = inner(r, z)
    it = 0
    rel = 1.0
    while it < maxit:
        q = apply_H(p)
        pq = inner(p, q)
        if pq <= 0.0:
            if not truncate:
                raise NegativeCurvature(f"<p, Hp> = {pq}")
            return (p.copy() if it == 0 else x), it, rel
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rel = np.sqrt(inner(r, r)) / r0
        if rel <= eta:
            break
        z = Minv * r
        rz_new = inner(r, z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it, rel


def max_abs(g: np.ndarray) -> float:
    """Infinity norm of the real parameter vector (real and imaginary parts)."""
    return float(max(np.max(np.abs(g.real)), np.max(np.abs(g.imag))))


@dataclass
class NewtonReport:
    iterations: int
    pcg_iterations: list
    energies: list
    steps: list
    grad_inf_rel: float
    vt: np.ndarray


def newton(vt0, I0, I1, p: Params, max_newton=5, max_pcg=10, gtol=1e-2,
           forcing=None, c1=1e-4, max_halvings=10, hessian="gn",
           point=None) -> NewtonReport:
    """Gauss-Newton-Krylov (hessian="gn") or Newton-Krylov (hessian="full",
    truncated PCG): p from PCG on H p = -g (preconditioner K~), then
    v~ <- v~ + eps p with Armijo backtracking from eps = 1 (halving).

    The paper writes the update as v - eps dv with H dv = -g (Eqs. 54-55); read
    literally that is an ascent step, so the descent direction p = dv is added.
    forcing=None uses eta = min(0.5, sqrt(||g|| / ||g0||)); a number fixes eta.
    Stops when ||g||_inf / ||g0||_inf < gtol, after max_newton updates, or when
    the line search fails.

    point: the objective, a callable vt -> an object with .vt, .energy, .cfl,
    .A (the preconditioner is 1 / A), .gradient() and .gn_hessvec(v) /
    .full_hessvec(v) (first element of each result used).  None is the
    registration energy of the chosen state equation (make_point); the pins
    pass closed-form objectives to check the iteration itself."""
    if point is None:
        point = lambda v: make_point(v, I0, I1, p)  # noqa: E731
    pt = point(vt0)
    g = pt.gradient()[0]
    g0_inf = max_abs(g)
    g0_2 = np.sqrt(inner(g, g))
    energies = [pt.energy]
    pcg_its, steps = [], []
    rel = 1.0
    for _ in range(max_newton):
        rel = max_abs(g) / g0_inf if g0_inf > 0 else 0.0
        if rel < gtol:
            break
        eta = (min(0.5, np.sqrt(np.sqrt(inner(g, g)) / g0_2)) if forcing is None
               else forcing)
        cur = pt
        hv = cur.full_hessvec if hessian == "full" else cur.gn_hessvec
        step, its, _ = pcg(lambda v: hv(v)[0], -g, 1.0 / cur.A[None], eta, max_pcg,
                           truncate=(hessian == "full"))
        pcg_its.append(its)
        slope = inner(g, step)
        eps = 1.0
        accepted = None
        for _ in range(max_halvings + 1):
            trial = point(pt.vt + eps * step)
            if trial.cfl < 1.0 and trial.energy <= pt.energy + c1 * eps * slope:
                accepted = trial
                break
            eps *= 0.5
        if accepted is None:
            break
        steps.append(eps)
        pt = accepted
        g = pt.gradient()[0]
        energies.append(pt.energy)
    rel = max_abs(g) / g0_inf if g0_inf > 0 else 0.0
    return NewtonReport(len(steps), pcg_its, energies, steps, rel, pt.vt)
