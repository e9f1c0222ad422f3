/*
 * blr.h -- C-ABI of the band-limited PDE-LDDMM Gauss-Newton-Krylov library
 * (libblr.so, CUDA kernels for sm_103a).
 *
 * Method: Hernandez, "Newton-Krylov optimization in PDE-constrained
 * diffeomorphic registration parameterized in the space of band-limited vector
 * fields" (arXiv 1807.05117): the state-equation variant (stationary or
 * non-stationary velocity, Gauss-Newton or full Newton Hessian) and the
 * deformation-state-equation variant (stationary, Gauss-Newton or full
 * Newton Hessian); compressible or incompressible velocities.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid      N = (N1, N2, N3), V = N1*N2*N3 voxels, voxel spacing 1.
 * Fields    float32, C order [N1][N2][N3] (N3 fastest).  Vector fields are
 *           [3][N1][N2][N3] (component-major).
 * Band      B = (B1, B2, B3), each even, 2 <= B_d <= N_d.  Centred integer
 *           frequencies k_d = -B_d/2 ... B_d/2-1 (Section 3.1, Eq. 33 read as a
 *           centred truncation).  Coefficient arrays are complex64 stored as
 *           interleaved float pairs (re, im), layout [3][B1][B2][B3]:
 *           2*3*B1*B2*B3 floats.
 * iota      iota(v~)_c(x) = Re sum_k v~_c(k) exp(2 pi i sum_d k_d x_d / N_d).
 * pi        pi(f)_c(k) = sum_x f_c(x) exp(-2 pi i sum_d k_d x_d / N_d) = iota^T
 *           under <a, b> = Re sum a conj(b).
 * A(k)      (alpha*omega(k) + gamma)^(2s), omega(k) = sum_d 2(1 - cos(2 pi k_d/N_d))
 *           (2s an integer);
 *           the regulariser L~ of Eq. 34 with L = (-alpha Lap + gamma)^s, and
 *           the preconditioner K~ = 1/A (Sections 3.1, 3.4).
 * Transport nt steps, dt = 1/nt; d = -dt * iota(v~) is the per-step
 *           displacement in voxels; m^{n+1}(x) = trilinear value of m^n at
 *           x + d(x) with periodic wrap (semi-Lagrangian solve of the state
 *           equation, Eq. 36).  The discrete adjoint uses the exact transpose
 *           of that step, which the kernels evaluate as a gather; it requires
 *           |d_a(x)| < 1 voxel on every axis (the CFL bound of Section 2.4).
 *
 * Pointers  "device" = memory the GPU can read (cudaMalloc / torch CUDA
 *           tensors).  "host or device" = either; the library copies it with
 *           cudaMemcpyDefault (pinned host memory gives asynchronous copies).
 *           All caller pointers are borrowed for the duration of the call only;
 *           the plan never keeps them.
 * Streams   Every call is ordered on `stream` (NULL = legacy default stream)
 *           and is asynchronous unless stated otherwise.  A plan may be used
 *           by one stream at a time; plans are independent of each other.
 * Errors    Functions return BLR_OK (0) or a negative code; nothing throws
 *           across the ABI.  Conditions detected on the device (a displacement
 *           that breaks the CFL bound, a non-finite energy) are latched in the
 *           plan and returned by blr_status(), which synchronises the stream.
 */
#ifndef BLR_H
#define BLR_H

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define BLR_OK        0
#define BLR_EINVAL   (-1)  /* bad argument, shape or call order            */
#define BLR_ENOMEM   (-2)  /* device allocation failed                     */
#define BLR_ECUDA    (-3)  /* CUDA runtime error                           */
#define BLR_ECFL     (-4)  /* |d_a(x)| >= 1 voxel per step somewhere        */
#define BLR_ENAN     (-5)  /* non-finite energy or residual                */
#define BLR_ESTATE   (-6)  /* needs a prior blr_state / blr_gradient        */
#define BLR_ECURV    (-7)  /* PCG met <p, Hp> <= 0                          */
#define BLR_ETIMEOUT (-8)  /* a bounded device wait expired (tensor cores)  */

/* Hessian used by blr_hessvec, blr_pcg and blr_newton. */
#define BLR_GAUSS_NEWTON 0 /* Eq. 46 with the Gauss-Newton drops of Section 3.4 */
#define BLR_NEWTON       1 /* the full Hessian of the discrete energy (Eqs. 44-46, */
                           /* no drops); may be indefinite away from a minimum  */

/* State equation of the constraint (Section 2.2 or 2.3). */
#define BLR_STATE_IMAGE       0 /* d_t m + grad m . v = 0, m(0) = I0 (Eq. 5)     */
#define BLR_STATE_DEFORMATION 1 /* d_t phi + D phi . v = 0, phi(0) = id, and    */
                                /* m(1) = I0 o phi(1) (Eqs. 16-18)             */

/* Precision of the truncated-DFT contractions (the transport is always FP32). */
#define BLR_FP32   0       /* FP32 FMA contractions                         */
#define BLR_MIXED  1       /* BF16 hi+lo split operands on tensor cores,     */
                           /* FP32 accumulation                             */

typedef struct CUstream_st *blr_stream_t;   /* identical to cudaStream_t */
typedef struct blr_plan *blr_plan_t;

/* Problem description (Section 3.2, Eq. 35 and the constants of L). */
typedef struct blr_params {
    int n[3];        /* grid N1, N2, N3 (each >= 1; N1 <= 65535; V <= 2^31) */
    int band[3];     /* B1, B2, B3 (each even, 2 <= B_d <= N_d)             */
    int nt;          /* number of time steps, >= 1                          */
    double alpha;    /* L = (-alpha Lap + gamma)^s, alpha >= 0              */
    double gamma;    /* gamma > 0                                           */
    double s;        /* s >= 0 with 2s an integer <= 64 (A = symbol^(2s)).  */
                     /* s = 0.5 is the H^1 regulariser alpha(-Lap) + gamma   */
                     /* of the incompressible experiments (Section 4)       */
    double sigma;    /* image term weight 1/sigma^2, sigma > 0              */
    int precision;   /* BLR_FP32 or BLR_MIXED                               */
    int ckpt_every;  /* 0: keep all nt+1 states.  k in 1..nt-1: keep only   */
                     /* m^0, m^k, m^2k, ... and m^nt; adjoint and HVP sweeps */
                     /* recompute each segment's states from its checkpoint  */
                     /* (same FP32 arithmetic, so results are bit-identical) */
    int incompressible; /* 0: compressible velocities (Eq. 4, gamma = 0).    */
                     /* 1: v~ restricted to divergence-free band fields      */
                     /* (Eq. 4, gamma = 1, imposed in the band): every call  */
                     /* that takes a velocity evaluates the energy at P v~,  */
                     /* P the Leray projector P(k) = I - kappa kappa^T /     */
                     /* |kappa|^2, kappa_d = 2 pi k_d / N_d (P(0) = I); the  */
                     /* gradient is then P grad E(P v~) and the Hessian      */
                     /* P H P.  blr_expand / blr_project / blr_adjoint stay  */
                     /* the plain operators.  Batches reject it.             */
    int hessian;     /* BLR_GAUSS_NEWTON or BLR_NEWTON.  BLR_NEWTON keeps   */
                     /* every adjoint and incremental state (2 nt V floats  */
                     /* more; 6 nt V for the deformation state equation),   */
                     /* so it takes no checkpoints; batches reject it       */
    int nonstationary; /* 0: one velocity v~ for all steps.  1: one per time */
                     /* step, v~^n transporting step n (the time-varying    */
                     /* v~_t of Section 3.2): every velocity, gradient, HVP, */
                     /* PCG and Newton array is then [nt][3][B1][B2][B3]    */
                     /* (nt times 2*3*B1*B2*B3 floats), the regulariser is  */
                     /* 1/2 dt sum_n <A v~^n, v~^n> and the gradient is     */
                     /* g^n = dt A v~^n + pi(b^n), b^n = dt lambda^{n+1}    */
                     /* grad m^n(x + d^n).  blr_adjoint then writes nt * 3V */
                     /* floats (b^n per step).  Gauss-Newton only; batches  */
                     /* reject it.                                          */
    int state_equation; /* BLR_STATE_IMAGE, or BLR_STATE_DEFORMATION: the    */
                     /* deformation u = phi - id is transported on the same  */
                     /* step, u^{n+1} = S u^n + d, and I0 is warped once,    */
                     /* m(1) = T[I0](x + u^nt) (trilinear, any displacement, */
                     /* periodic).  The adjoint is the vector rho, from       */
                     /* rho^nt = lambda(1) grad T[I0](x + u^nt); the body     */
                     /* force is dt sum_n (rho^{n+1} + sum_c rho_c^{n+1}      */
                     /* grad u^n_c(x + d)).  Stationary velocity, no         */
                     /* checkpoints; either Hessian; blr_adjoint takes no    */
                     /* lambda0; batches reject it.  Keeps 3 (nt + 1) V      */
                     /* floats of u^n.                                      */
} blr_params;

/* Result of blr_newton (host struct filled by the library). */
typedef struct blr_report {
    int newton_iters;      /* accepted Newton updates                       */
    int pcg_iters;         /* PCG iterations summed over the run            */
    int n_state;           /* forward solves (gradients + line-search trials) */
    int n_hessvec;         /* Gauss-Newton Hessian-vector products          */
    int n_halvings;        /* step-length halvings in the line search       */
    int status;            /* BLR_OK, or why the run stopped early          */
    double energy0;        /* E at the initial velocity                     */
    double energy;         /* E at the returned velocity                    */
    double grad_inf_rel;   /* ||g||_inf / ||g_0||_inf at the returned velocity */
} blr_report;

/* Create a plan: validates `p`, allocates every device buffer the hot path
 * needs for this grid/band/nt (state stack: nt+1 fields, or ceil(nt/k) + k with
 * checkpoints every k steps; adjoint and
 * incremental fields, DFT tables and intermediates, PCG vectors, reduction
 * scratch) and builds the DFT tables on the current device.
 * `p` is host memory, read once.  On success *out owns the allocations.
 * Returns BLR_EINVAL for an invalid `p`, BLR_ENOMEM / BLR_ECUDA otherwise. */
int blr_plan_create(const blr_params *p, blr_plan_t *out);

/* Release every allocation of the plan (synchronises the device first).
 * NULL is accepted. */
int blr_plan_destroy(blr_plan_t plan);

/* Template I0 and reference I1 of the registration (Section 2.2: m(0) = I0,
 * the image term compares m(1) with I1).  Host or device, V floats each; the
 * plan keeps its own copies.  Invalidates any stored state. */
int blr_set_images(blr_plan_t plan, const float *I0, const float *I1,
                   blr_stream_t stream);

/* iota (Section 3.1, Eq. 33): band coefficients -> spatial vector field.
 * vt: device, 2*3*B1*B2*B3 floats (interleaved complex).
 * v : device, 3*V floats, written. */
int blr_expand(blr_plan_t plan, const float *vt, float *v, blr_stream_t stream);

/* pi = iota^T (Section 3.1): spatial vector field -> band coefficients.
 * f : device, 3*V floats.   ft: device, 2*3*B1*B2*B3 floats, written. */
int blr_project(blr_plan_t plan, const float *f, float *ft, blr_stream_t stream);

/* Forward solve of the state equation (Section 3.2, Eq. 36, m(0) = I0) at the
 * velocity vt and the energy of Eq. 35.  Stores vt, the displacement and all
 * states m^0..m^nt in the plan (the "current point" used by blr_adjoint,
 * blr_hessvec and blr_pcg).
 * vt    : device, 2*3*B1*B2*B3 floats.
 * m1    : device, V floats, receives m^nt; may be NULL.
 * energy: device, 3 doubles {E, regulariser part, image part}; may be NULL.
 * A displacement with |d| >= 1 latches BLR_ECFL (see blr_status). */
int blr_state(blr_plan_t plan, const float *vt, float *m1, double *energy,
              blr_stream_t stream);

/* Adjoint solve (Eq. 8 with lambda(1) = -(2/sigma^2)(m(1) - I1)) at the current
 * point, and the body force b = dt sum_n lambda^{n+1} grad m^n(x + d), the
 * discrete lambda grad m of Eq. 38.  Needs a prior blr_state (BLR_ESTATE).
 * Repeatable: the plan keeps lambda^nt of the current point apart from the
 * buffers that blr_hessvec uses.
 * b      : device, 3*V floats, written (non-stationary plans: nt * 3V, b^n).
 * lambda0: device, V floats, receives lambda^0; may be NULL (must be NULL for
 *          the deformation state equation, whose adjoint is a vector). */
int blr_adjoint(blr_plan_t plan, float *b, float *lambda0, blr_stream_t stream);

/* Reduced gradient (Section 3.2, Eq. 38): g~ = A v~ + pi(b), i.e. blr_state +
 * blr_adjoint + blr_project + the regulariser term, at vt.
 * vt: device (input), g: device, 2*3*B1*B2*B3 floats (written),
 * energy: device, 3 doubles, may be NULL. */
int blr_gradient(blr_plan_t plan, const float *vt, float *g, double *energy,
                 blr_stream_t stream);

/* Reduced gradient (Eq. 38) at the current point, i.e. the velocity of the last
 * blr_state / blr_gradient, without a new forward solve: the adjoint solve (with
 * segment recomputation when checkpointing), pi(b) and A v~.  This is the
 * backward of the energy returned by blr_state.
 * g: device, 2*3*B1*B2*B3 floats (written).  Needs a prior blr_state (BLR_ESTATE). */
int blr_gradient_at_state(blr_plan_t plan, float *g, blr_stream_t stream);

/* Hessian-vector product at the current point (Section 3.2, Eqs. 44-46).
 * BLR_GAUSS_NEWTON (the drops of Section 3.4):
 *   H~ dv~ = A dv~ + pi(db), incremental state dm^0 = 0,
 *   dm^{n+1} = S dm^n - dt grad m^n(x+d) . iota(dv~), dlambda^nt =
 *   -(2/sigma^2) dm^nt, dlambda^n = S^T dlambda^{n+1},
 *   db = dt sum_n dlambda^{n+1} grad m^n(x + d).
 * BLR_NEWTON (the exact Hessian of the discrete energy), with dd = -dt iota(dv~)
 * and lambda^n the gradient's adjoint states at the current point:
 *   dlambda^n = S^T dlambda^{n+1} + sum_a D_a^T (dd_a lambda^{n+1}),
 *   db = dt sum_n [dlambda^{n+1} grad m^n(x+d)
 *                  + lambda^{n+1} (grad dm^n(x+d) + Hess m^n(x+d) dd)],
 *   D_a and Hess the first and second derivatives of the trilinear cell
 *   polynomial at the departure point (the adjoint states are computed on the
 *   first call after a forward solve when blr_gradient has not done so).
 * BLR_NEWTON with BLR_STATE_DEFORMATION (Eqs. 19-21 without the drops), with the
 *   gradient's adjoint states rho^n and du^n the incremental deformation:
 *   drho^nt = dlambda(1) grad T[I0](x+u^nt) + lambda(1) Hess T[I0](x+u^nt) du^nt,
 *   drho^n_c = S^T drho^{n+1}_c + sum_a D_a^T (dd_a rho^{n+1}_c),
 *   db_a = dt sum_n (drho_a^{n+1} + sum_c [drho_c^{n+1} D_a u_c^n
 *          + rho_c^{n+1} (D_a du_c^n + (Hess T[u_c^n] dd)_a)]).
 * dvt: device input, hdv: device output, 2*3*B1*B2*B3 floats each.
 * Needs a prior blr_state / blr_gradient (BLR_ESTATE). */
int blr_hessvec(blr_plan_t plan, const float *dvt, float *hdv,
                blr_stream_t stream);

/* Preconditioned CG (Section 3.4, Eq. 55) on H~ x = rhs from x = 0 with the
 * preconditioner K~ = 1/A, at the current point.  Inner products and step
 * scalars are FP64 on the device.  Stops when ||r|| <= eta ||r_0|| or after
 * maxit iterations.  Synchronises the stream once per iteration.
 * rhs, x: device, 2*3*B1*B2*B3 floats (x written).
 * iters, relres: host, may be NULL (iterations run, final ||r||/||r_0||).
 * Returns BLR_ECURV if <p, Hp> <= 0 (x then holds the iterate before that
 * direction). */
int blr_pcg(blr_plan_t plan, const float *rhs, float *x, int maxit, double eta,
            int *iters, double *relres, blr_stream_t stream);

/* Gauss-Newton-Krylov registration (Section 3.4, Eqs. 54-55): from vt, up to
 * max_newton updates v~ <- v~ + eps p with H~ p = -g~ solved by blr_pcg
 * (<= max_pcg iterations) and eps from Armijo backtracking (c1 = 1e-4,
 * eps = 1, 1/2, ..., at most 10 halvings; a trial breaking the CFL bound is
 * rejected).  The paper's "v - eps dv" is read as this descent step.
 * PCG tolerance: eta = forcing if forcing >= 0, else
 * min(0.5, sqrt(||g|| / ||g_0||)).  Stops when ||g||_inf / ||g_0||_inf < gtol.
 * With BLR_NEWTON the solve is truncated at non-positive curvature: p is the
 * PCG iterate before that direction, or K~(-g) when it is the first (truncated
 * Newton-CG; both are descent directions).
 * vt : host or device, 2*3*B1*B2*B3 floats, in: initial velocity, out: result.
 * rep: host, may be NULL.  Synchronous. */
int blr_newton(blr_plan_t plan, float *vt, int max_newton, int max_pcg,
               double gtol, double forcing, blr_report *rep,
               blr_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batching form.  The paper registers one pair at a time; this is a library
 * facility for many independent pairs (each with its own grid, band, sigma and
 * images; all with the same nt, FP32, no checkpointing) advanced together:
 * every sweep time step of all pairs is one persistent kernel launch over a
 * (pair, tile) work queue, the per-pair truncated DFTs run concurrently on side
 * streams, and one PCG iteration of all pairs is a CUDA graph that is captured
 * once and replayed.  The x1 tile length is autotuned at creation by timing
 * candidate shapes on the batch.  Each pair's arithmetic is that of a single
 * plan, so results are bit-identical to per-pair blr_* calls.
 * All calls below synchronise `stream` first and are synchronous.
 * --------------------------------------------------------------------------- */
typedef struct blr_batch *blr_batch_t;

/* params: host array of npairs descriptions.  BLR_EINVAL if they differ in nt,
 * request BLR_MIXED, checkpoints, the incompressible form, the full Hessian,
 * non-stationary velocities or the deformation state equation, or one is
 * invalid. */
int blr_batch_create(const blr_params *params, int npairs, blr_batch_t *out);
int blr_batch_destroy(blr_batch_t batch);

/* Diagnostic (no counterpart in the paper): the batch's sweep choices into
 * vals[0 .. min(n, 7) - 1]: [0] 1 if every pair keeps its state gradients
 * grad m^n(x + d(x)) (3 nt V floats per pair, allocated when they fit),
 * [1] 1 if the batched sweeps use them (the state sweep writes them, the
 * adjoint and incremental-state sweeps read them), [2] the x1 tile length of
 * the adjoint sweep's work items and [3] that of the state and
 * incremental-state sweeps (0: each pair's own one-wave length, else planes for
 * every pair, capped at its N1), [4] the grid size in voxels from which a pair
 * runs "solo" (0: no pair does), [5] the number of solo pairs, [6] 1 if the
 * queued incremental-state steps use the gather form (with [1]).  A solo pair
 * skips the work queue and runs its own plan's autotuned kernels, solo pairs on
 * three concurrent lanes.  [1] to [3] and [6] are chosen at creation by timing
 * the batch.  BLR_EINVAL for a NULL batch or vals. */
int blr_batch_tuning(blr_batch_t batch, int *vals, int n);

/* Diagnostic: force the choices [0] to [4] (and, when n >= 7, [6]; [5] is
 * ignored) of blr_batch_tuning (n >= 5; vals[0] must be the batch's own,
 * vals[1] <= vals[0], vals[2..3] 0 or 2..1024, vals[4] >= 0, vals[6] <= vals[1]).
 * Every choice computes the same results bit for bit.
 * A change of vals[1] or of the set of solo pairs drops every pair's current
 * point (the next call must be blr_batch_gradient or blr_batch_newton).
 * Synchronises the device. */
int blr_batch_set_tuning(blr_batch_t batch, const int *vals, int n);

/* Images of pair `pair` (host or device pointers, as blr_set_images). */
int blr_batch_set_images(blr_batch_t batch, int pair, const float *I0, const float *I1,
                         blr_stream_t stream);

/* Gradients (Eq. 38) of all pairs: vt[p] device input, g[p] device output
 * (host arrays of npairs pointers); sets every pair's current point. */
int blr_batch_gradient(blr_batch_t batch, const float *const *vt, float *const *g,
                       blr_stream_t stream);

/* Gauss-Newton HVPs (Eq. 46, Section 3.4) of all pairs at their current points. */
int blr_batch_hessvec(blr_batch_t batch, const float *const *dvt, float *const *hdv,
                      blr_stream_t stream);

/* Gauss-Newton-Krylov registration of all pairs (the algorithm of blr_newton,
 * per pair); vt[p] host or device, in/out; reps: host array of npairs (may be
 * NULL).  A pair that fails (CFL, non-positive curvature) stops with its status
 * in its report while the others continue. */
int blr_batch_newton(blr_batch_t batch, float *const *vt, int max_newton, int max_pcg,
                     double gtol, double forcing, blr_report *reps, blr_stream_t stream);

/* Synchronise `stream`, return the first latched device condition
 * (BLR_ECFL, BLR_ENAN) or BLR_OK, and clear it. */
int blr_status(blr_plan_t plan, blr_stream_t stream);

/* Allocation-free iota.  The paper has no counterpart: this is a convenience of
 * the library for callers that cannot allocate device memory, such as a host
 * framework that owns every device allocation through its own pool (nothing else
 * may call cudaMalloc, so its accounting stays exact) or a latency-critical loop
 * that cannot accept cudaMalloc / cudaFree, which may synchronise the device.
 * Result: the same field as blr_expand for the same grid and band.
 * n, band: host arrays of 3 ints with the rules of blr_params (band even,
 *          2 <= band[d] <= n[d], band[2] <= 64).
 * vt     : device, 2*3*B1*B2*B3 floats;  v: device, 3*N1*N2*N3 floats, written.
 * Storage: no plan and no allocation.  The DFT tables and intermediates live in
 *   one fixed device array of BLR_NOALLOC_SCRATCH_BYTES that the library keeps
 *   in every GPU that loads it until the process exits.  A call needs
 *   4 * (2 B1 N1 + 2 B2 N2 + 2 B3 N3 + B1 B2 B3 + 6 B1 B2 N3 + 6 B1 N2 N3) bytes
 *   (each term rounded up to 256 bytes); larger problems are rejected with
 *   BLR_EINVAL before anything runs (a 128^3 grid with a 32^3 band fits).
 * Set-up: the first call on each device, with that device current, looks up
 *   the array's device address (cudaGetSymbolAddress); make that first call
 *   before any stream capture.  The look-up is repeated when the device's
 *   context has changed since (after cudaDeviceReset the library's device code
 *   is loaded again and the array may have moved), so make the first call after
 *   a reset before any capture too.
 * Sharing: every call on a device uses the same array.  Calls whose work
 *   overlaps on the GPU (other streams, other host threads) race and corrupt
 *   each other's results: order them on one stream.  Each call writes every
 *   scratch element before reading it, so nothing carries over between calls.
 * Never calls cudaMalloc, cudaFree or any allocating routine. */
#define BLR_NOALLOC_SCRATCH_BYTES (16u << 20)
int blr_expand_noalloc(const int n[3], const int band[3], const float *vt, float *v,
                       blr_stream_t stream);

/* Diagnostic (no counterpart in the paper): number of kernels this library
 * has launched since it was loaded, over all plans and threads. */
unsigned long long blr_kernel_launches(void);

/* Diagnostic (no counterpart in the paper): the sweep shapes the plan's
 * autotuner chose at creation.  vals: host, n ints; the first min(n, 13) are
 * written, in this order: wide-copy sweeps (0/1), state gradients kept (0/1),
 * adjoint blocks per SM, adjoint reads the kept gradient (0/1), incremental
 * state form (0 wide-copy, 1 wide-copy reading the kept gradient, 2 gather),
 * its blocks per SM, march-kernel blocks per SM (0: chunked grid), march x1
 * chunk, adjoint march x1 chunk, displacement copy kept in persisting L2
 * lines (0/1; when 1, plan creation raised the context's persisting-L2
 * set-aside to hold it), two adjoint steps per launch (blocks per SM of that
 * kernel's grid, or 0 for one step per launch), split adjoint solve (0/1: the
 * steps transport lambda alone into kept adjoint states, (nt - 1) V floats,
 * and one pass sums the body force of all steps, bit-identical to the per-step
 * sums), the FP32 transforms' GEMM tiles (3 bits per stage, stage s at bits
 * 3s..3s+2, stages 0 axis 2 and 1 axis 1 of the expand, 2 axis 1 and 3 axis 2
 * of the project, 4 axis 3 of the expand; each 1..6 a register tile and thread
 * count timed at creation, 0 the modelled choice; every tile gives the same
 * results bit for bit).  Returns BLR_EINVAL for a NULL plan or vals. */
int blr_plan_tuning(blr_plan_t plan, int *vals, int n);

/* Test hook (no counterpart in the paper): while `on` is non-zero, every launch
 * of the pipelined tensor-core DFT kernel (BLR_MIXED plans) first waits about
 * 1 ms on a barrier that nothing arrives at, before it issues any copy or MMA.
 * The wait expires, the launch frees its tensor memory, writes no output and
 * latches BLR_ETIMEOUT (returned by blr_status / blr_newton), exactly as when a
 * real bounded wait of the kernel runs out.  It exists so that the timeout path
 * can be tested without a fault; the waits that guard copies or MMAs in flight
 * are never shortened.  Process-wide; returns BLR_OK. */
int blr_test_expire_waits(int on);

/* Diagnostic (no counterpart in the paper): set the sweep shapes, in the order
 * and meaning of blr_plan_tuning (n >= 11 values, a 12th sets the split
 * adjoint solve, a 13th the GEMM tiles; the first two must be the plan's own), instead of the
 * autotuner's choice, e.g. to reproduce a
 * configuration.  Every shape computes the same results bit for bit.
 * Synchronises the device.  BLR_EINVAL for a value out of range or a shape the
 * plan's buffers do not support (a kept-gradient form without kept gradients,
 * the persisting-L2 window where the device has none, the split adjoint
 * without its kept adjoint states or together with two steps per launch). */
int blr_plan_set_tuning(blr_plan_t plan, const int *vals, int n);

/* Human-readable text for a status code (static storage). */
const char *blr_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* BLR_H */
