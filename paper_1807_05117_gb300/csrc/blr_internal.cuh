// Internal definitions shared by the libblr translation units.
//
// Notation: fields are [N1][N2][N3] with N3 fastest; (i, j, k) index (x1, x2, x3).
// Vector component c displaces along array axis c (component 0 along x1).
// Band coefficients are interleaved complex [3][B1][B2][B3].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/blr.h"

#define BLR_CK(call)                                   \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return BLR_ECUDA;       \
    } while (0)

// Every kernel launch of the library is counted (blr_kernel_launches()).
extern unsigned long long g_blr_launches;
#define BLR_CK_LAUNCH()                                                   \
    do {                                                                  \
        __atomic_fetch_add(&g_blr_launches, 1ULL, __ATOMIC_RELAXED);      \
        BLR_CK(cudaGetLastError());                                       \
    } while (0)

// Programmatic dependent launch.  launch_pdl lets the kernel start while the
// previous kernel in the stream drains (block launch and any prologue that
// reads nothing the previous kernel writes overlap its tail); every kernel
// launched this way calls pdl_wait() before it touches such data, which returns
// once the previous grid has completed and its writes are visible.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel of the stream launch before this one has finished (it
// still waits for this grid's completion in its pdl_wait).  The next grid
// launches only once every block of this grid has executed the trigger or
// exited, so no block of this grid is still waiting for room on an SM.
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// launch_pdl with an L2 access-policy window (win may be nullptr: plain launch_pdl).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_l2(const cudaAccessPolicyWindow *win, void (*kernel)(KArgs...),
                                 dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                 Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (win) {
        attr[1].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[1].val.accessPolicyWindow = *win;
        cfg.numAttrs = 2;
    }
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Device-latched conditions (bit flags in blr_plan::dstatus).
enum { BLR_FLAG_CFL = 1, BLR_FLAG_NAN = 2, BLR_FLAG_TIMEOUT = 4 };

// Slots of the device scalar block blr_plan::dsc (doubles).
enum {
    SC_E = 0, SC_EREG = 1, SC_EDATA = 2,       // energy of blr_state
    SC_RZ = 3, SC_PQ = 4, SC_RR = 5, SC_BETA = 6, SC_RR0 = 7,
    SC_GINF = 8, SC_DOT = 9, SC_ALPHA = 10,
    SC_REL = 11,                               // ||r|| / ||r0|| after the last PCG update
    SC_COUNT = 16
};

struct Grid3 {
    int N1, N2, N3;
    long long V;
};

// Operands of one pair in a batched sweep launch (see k_sweep_batch).
struct SweepPair {
    Grid3 g;
    int chunk, tk, tj, ti;   // x1 chunk; tiles along x3, x2, x1 (for this kind)
    const float *in0;        // state: m^n | adjoint: lambda^{n+1} | incremental: dm^n
    const float *m;          // adjoint / incremental: m^n
    const float *d;          // displacement
    const float4 *d4;        // its float4 copy (wide-copy tiles)
    const float *aux;        // state: I1 (last step) | incremental: dv
    float *out0;             // state: m^{n+1} | adjoint: lambda^n | incremental: dm^{n+1}
    float *out1;             // state: lambda^nt (last step) | adjoint: body force
    double *partials;        // state (last step): image-term sums per 32-voxel row segment
    float dt, scale;         // time step; lambda scale -2/sigma^2
    const int *active;       // nullptr or a device flag: 0 skips the pair
    const float *G;          // adjoint / incremental (kept gradients): grad m^n(x + d(x))
    float *Gout;             // state (kept gradients): where grad m^n(x + d(x)) is written
};

struct blr_plan {
    blr_params p;
    int N1, N2, N3, B1, B2, B3;
    long long V;       // voxels
    long long nb;      // B1*B2*B3
    long long nf1;     // floats in one velocity's coefficients: 2*3*nb
    int nvel;          // velocities in the parameter vector: 1, or nt (non-stationary)
    long long nfloat;  // floats in one parameter vector: nvel * nf1
    float dt;
    int device;
    int chunk;          // x1 planes per state / incremental-state sweep block
    int chunk_adj;      // x1 planes per adjoint sweep block (both set by sweep_setup)
    int bal_sweep;      // state / incremental-state sweeps: balanced grid of bal_sweep
                        // blocks per SM, or 0 for the chunked grid
    int bal_adj;        // the same for the adjoint sweep (both chosen by sweep_autotune)
    int sms;            // multiprocessors of the plan's device
    int l2_persist;     // the wide sweeps keep d4 in persisting L2 lines (sweep_autotune)
    size_t l2_win_bytes;  // access-policy window over d4 (0: not available on this device)
    int l2_counted;     // counted among the plans that rely on the raised persisting-L2 limit
    float l2_hit;       // its hit ratio (set-aside / window)
    Grid3 grid;

    float *I0, *I1;
    float *vt;          // current point (nfloat)
    float *d;           // 3V displacement -dt*iota(vt), clamped to [-1, 1) (non-stationary:
                        // the step that use_step selected)
    float4 *d4;         // V (d0, d1, d2, 0) copy of d for the wide-copy sweeps, or nullptr
    float *d_base;      // [nvel][3V] every step's displacement
    float4 *d4_base;    // [nvel][V] their float4 copies, or nullptr
    bool sweep_wide;    // adjoint and incremental state use the wide-copy kernels (N3 % 4 == 0)
    bool use_gm;        // Gm is kept (see Gm)
    int bal_inc;        // blocks per SM of the wide-copy incremental-state grid (sweep_autotune)
    int adj_useg;       // the adjoint reads Gm (1) or interpolates it (0)      (sweep_autotune)
    int adj_split;      // adjoint solve as transport steps + one body-force pass (sweep_autotune)
    int bal_tr;         // blocks per SM of the transport-only grid (0: ADJ_BLOCKS)
    float *lam_keep;    // lambda^1 .. lambda^{nt-1} of the split adjoint solve, or nullptr
    float *rho_keep;    // rho^1 .. rho^{nt-1} ([3][V] each) of the deformation variant's split solve
    float *dv_all;      // non-stationary (fused or FP32 transforms): every step's direction [nt][3][V]
    float *b_all;       // non-stationary (fused or FP32 transforms): every step's body force [nt][3][V]
    int adj2;           // two adjoint steps per launch on a balanced grid of adj2 blocks
                        // per SM (plans that keep Gm), or 0: one step per launch
                        //                                                      (sweep_autotune)
    int inc_mode;       // incremental state: 0 wide-copy, 1 wide-copy reading Gm,
                        // 2 gather reading Gm                                  (sweep_autotune)
    float *m;           // state slots (see state_slot): checkpoints, segment, final
    int ck;             // checkpoint interval k (nt when every state is kept)
    int nseg;           // segments ceil(nt / k)
    int seg_valid;      // segment whose interior states the segment buffer holds
    bool have_state;
    bool have_lams;     // lam_all holds the adjoint states of the current point
    float *lam[2];      // V each (adjoint / incremental adjoint ping-pong)
    float *lam_nt;      // V: lambda^nt of the current point (written by the state sweep)
    float *lam_all;     // full Newton Hessian: [nt][V], slot k-1 = lambda^k (k = 1..nt; the
                        // last slot is lam_nt), else nullptr
    float *dm_all;      // full Newton Hessian: [nt-1][V], slot k-1 = dm^k of the last
                        // incremental state (k = 1..nt-1), else nullptr
    // deformation state equation (else nullptr)
    float *U;           // [nt+1][3][V] u^n = phi^n - id (u^0 = 0)
    float *rho_nt;      // 3V rho^nt of the current point
    float *rho[2];      // 3V each: adjoint / incremental adjoint ping-pong
    float *du[2];       // 3V each: incremental deformation ping-pong
    float *Gw;          // 3V grad T[I0](x + u^nt)
    float *rho_all;     // full Newton Hessian: [nt][3][V], slot k-1 = rho^k (k = 1..nt; the
                        // last slot is rho_nt), else nullptr
    float *du_all;      // full Newton Hessian: [nt-1][3][V], slot k-1 = du^k of the last
                        // incremental state (k = 1..nt-1), else nullptr
    float *nt_kap;      // full Newton Hessian: [27][V] stencil of the variation of S^T for
                        // the current direction (newton.cu), else nullptr
    float *Gm;          // [nt][3][V] grad of the trilinear cell of m^n at x + d(x) (written by
                        // the state sweep, read by the adjoint and incremental sweeps), or
                        // nullptr (checkpointed plans and batch members compute it on the fly)
    float *b;           // 3V body force
    float *dv;          // 3V iota(dv~)
    float *dm[2];       // V each (incremental state ping-pong)

    // truncated-DFT tables and intermediates
    float *W1;          // [2*B1][N1]: row 2j = cos, row 2j+1 = -sin (2 pi k_j x / N1)
    float *T2c, *T2s;   // [B2][N2]
    float *W1t;         // FP32 project axis-1 stage: W1 transposed, [N1][2 B1] (or nullptr)
    int gemm_tile[5];   // FP32 GEMM stages' tile candidate (0: modelled choice; dft_autotune)
    float *T3e;         // FP32 expand axis-3 stage's B operand [2 B3][2 N3] (or nullptr)
    float *T2e, *T2p;   // FP32 axis-2 stages as real GEMMs, A operand [k][m] (or nullptr):
                        // expand [2 B2][2 N2] = [[C, S], [-S, C]]^T-ordered, project [2 N2][2 B2]
    float *T3c, *T3s;   // [B3][N3]
    float *A;           // [B1][B2][B3] regulariser weights
    float *dft_big;     // 3*B1*N2*N3*2 floats
    float *dft_small;   // 3*B1*B2*N3*2 floats
    uint8_t *tc_tab_expand;    // BLR_MIXED: swizzled BF16 hi/lo table tiles (dft_tc.cu)
    uint8_t *tc_tab_project;
    uint8_t *tc_tab2_expand;   // BLR_MIXED axis-2 stages, or nullptr (SIMT axis 2)
    uint8_t *tc_tab2_project;
    uint8_t *fz_tab[4];        // BLR_MIXED fused transforms (dft_fused.cu), or nullptr:
                               // then the stages above are not used
    float *fz_buf;             // their band-sized intermediate

    // Krylov / Newton vectors (nfloat each)
    float *g, *r, *pv, *q, *x, *trial, *step, *vtmp;
    float *vproj;       // incompressible plans: the projected HVP direction (else nullptr)

    double *dsc;        // device scalars (SC_COUNT)
    double *hsc;        // pinned host mirror
    int *hlive;         // pinned: two mirrors of pcg_live (4 ints each) and its start value
    int *dstatus;
    int *pcg_live;      // device PCG control [running, stop code, updates] (single plans)
    double *partials;   // per-block partial sums
    double *partials2;  // second-level partials (energy)
    const int *active;  // batch member: device flag, 0 freezes PCG updates (else nullptr)
    unsigned int *ticket;
    int npart;
};

__host__ __device__ inline long long ceil_div_ll(long long a, long long b) { return (a + b - 1) / b; }

// Storage of m^n.  Slots: checkpoints C_j = m^{j k} (j < nseg), then the k-1
// interior states of one segment, then m^nt.  With k = nt this is m^n in slot n.
inline float *def_u(const blr_plan *P, int n, int c) {   // u^n_c (deformation variant)
    return P->U + ((size_t)3 * n + c) * P->V;
}

inline float *state_slot(const blr_plan *P, int n) {
    const int k = P->ck;
    long long slot;
    if (n == P->p.nt) slot = P->nseg + k - 1;
    else if (n % k == 0) slot = n / k;
    else slot = P->nseg + (n % k) - 1;
    return P->m + slot * P->V;
}

// Point d / d4 at the displacement of step n (a no-op for stationary plans: every
// step has the one displacement).  The launchers read P->d / P->d4 when they
// launch, so each step's kernels see their own step's field.
inline void use_step(blr_plan *P, int n) {
    if (P->nvel <= 1) return;
    P->d = P->d_base + (size_t)3 * n * P->V;
    if (P->d4_base) P->d4 = P->d4_base + (size_t)n * P->V;
}

// Plan creation (api.cu); grad_cache: keep the per-step state gradients Gm
// when every state is stored (batch members run their own sweeps and skip it).
int plan_create(const blr_params *p, bool grad_cache, blr_plan **out);

// ---- launchers implemented in the .cu files (return BLR_OK / BLR_ECUDA) ----

// dft.cu
int dft_init_tables(blr_plan *P, cudaStream_t s);
constexpr int SG_CANDS = 6;   // tile candidates of the FP32 GEMM stages (1 .. SG_CANDS)
int dft_autotune(blr_plan *P, cudaStream_t s);
// nc fields (3 per velocity; every step of a non-stationary plan) in one transform
// (fused mixed-precision kernels or the FP32 GEMM stages; BLR_EINVAL otherwise).
int dft_expand_nc(blr_plan *P, const float *vt, float *out, int mode, cudaStream_t s, int nc);
int dft_project_nc(blr_plan *P, const float *f, float *ft, const float *vadd, cudaStream_t s,
                   float areg, int nc);
// iota into out (3V). mode 0: out = v; mode 1: out = clamp(-dt*v) + CFL/NaN flags.
int dft_expand(blr_plan *P, const float *vt, float *out, int mode, cudaStream_t s);
// pi(f) (+ areg A * vadd when vadd != nullptr) into ft.
int dft_project(blr_plan *P, const float *f, float *ft, const float *vadd, cudaStream_t s,
                float areg = 1.0f);

// dft_tc.cu (BLR_MIXED)
// stage kinds: 0 / 1 axis-1 expand / project, 2 / 3 axis-2 expand / project
size_t tc_table_bytes(const blr_plan *P, int kind);
bool tc_supported(const blr_plan *P);          // axis-1 stages (required by BLR_MIXED)
bool tc_axis2_supported(const blr_plan *P);    // axis-2 stages as well
int tc_init_tables(blr_plan *P, cudaStream_t s);
int tc_axis1(blr_plan *P, int project, const float *X, float *D, float scale, int mode,
             cudaStream_t s);
int tc_axis2(blr_plan *P, int project, const float *X, float *D, cudaStream_t s);

// dft_fused.cu (BLR_MIXED): iota and pi as a band-sized axis-1 stage plus one
// tensor-core kernel over (component, x1 plane, x2 tile) units
bool fz_supported(const blr_plan *P);
size_t fz_table_bytes(const blr_plan *P, int kind);
size_t fz_buffer_floats(const blr_plan *P);
int fz_init_tables(blr_plan *P, cudaStream_t s);
int fz_expand(blr_plan *P, const float *vt, float *out, float scale, int mode, cudaStream_t s,
              int nc = 3);
int fz_project(blr_plan *P, const float *f, float *ft, const float *vadd, float areg,
               cudaStream_t s, int nc = 3);

// sweeps.cu
int sweep_setup(blr_plan *P);
long long sweep_blocks(const blr_plan *P);
int sweep_state(blr_plan *P, cudaStream_t s);                  // m^1..m^nt, lambda^nt, partials
// Adjoint sweep from lambda^nt = lam_final: b = dt sum_n lambda^{n+1} grad m^n,
// lambda^0 into lambda0 (nullable).  The gradient's solve (lam_final == P->lam_nt)
// also keeps every lambda^n in lam_all when the plan has it.
int sweep_adjoint(blr_plan *P, float *b, float *lambda0, const float *lam_final, cudaStream_t s);
// The full Newton incremental adjoint: as sweep_adjoint from dlambda^nt in lam[0], with
// the second-order terms of newton.cu after every step (needs lam_all and dm_all).
int sweep_adjoint_newton(blr_plan *P, float *b, cudaStream_t s);
// dm -> dlambda^nt in lam[0]; dvt_steps (non-stationary plans): the direction's
// coefficients, expanded into P->dv before each step.
int sweep_incremental(blr_plan *P, cudaStream_t s, const float *dvt_steps = nullptr);
// Non-stationary adjoint: per step n, b^n = dt lambda^{n+1} grad m^n (into b_steps +
// 3nV when given, else P->b) and, when gout is given, gout^n = pi(b^n) + dt A vadd^n.
int sweep_adjoint_steps(blr_plan *P, const float *lam_final, float *gout, const float *vadd,
                        float *b_steps, float *lambda0, cudaStream_t s);
// wide: the adjoint and incremental-state items use the wide-copy tiles (every
// pair has N3 % 4 == 0); the incremental-state tiles are then AJ rows high.
int sweep_batch_launch(int kind, bool f1, bool f2, bool wide, bool useg, const SweepPair *pairs,
                       const long long *starts, int npairs, unsigned long long *counter, int grid,
                       cudaStream_t s);
// kind: 0 state, 1 adjoint, 2 incremental state
void sweep_tiles(const blr_plan *P, int kind, bool wide, int *tk, int *tj, int *ti);
int sweep_chunk(const blr_plan *P, int kind);
int sweep_blocks_per_sm(int kind, bool wide = false);
void sweep_set_chunk(blr_plan *P, int kind, int chunk);
float *grad_slot(const blr_plan *P, int n);   // kept grad m^n, or nullptr
float *def_grad_slot(const blr_plan *P, int n, int c);   // kept grad u^n_c, or nullptr
int sweep_autotune(blr_plan *P, cudaStream_t s);
int sweep_pack_d4(blr_plan *P, cudaStream_t s);               // d4 from d (when P->d4)

// newton.cu: step n's second-order terms of the full Newton Hessian (b += ..., and
// dlam += the variation of S^T when transpose_term); dmn = dm^n or nullptr (n = 0).
int newton_terms(blr_plan *P, bool transpose_term, const float *lam1, const float *mn,
                 const float *dmn, float *dlam, float *b, cudaStream_t s);
// newton.cu: the step-invariant weights of those terms for the direction in P->dv.
int newton_prep(blr_plan *P, cudaStream_t s);

// deform.cu: y = a + alpha x over n floats; the final warp (mode 0: m(1) into the
// last state slot, Gw, rho^nt = lambda(1) Gw and the energy partials; mode 1:
// drho^nt from du^nt) and its fixed block count.
int field_axpy(blr_plan *P, float *y, const float *a, const float *x, float alpha, long long n,
               cudaStream_t s);
int def_final(blr_plan *P, int mode, const float *u, const float *du, float *rho, cudaStream_t s);
// deform.cu: the full Newton Hessian's start of the incremental adjoint,
// drho^nt = dlambda(1) grad T[I0](x + u^nt) + lambda(1) Hess T[I0](x + u^nt) du^nt.
int def_final_newton(blr_plan *P, const float *du, float *rho, cudaStream_t s);
int def_final_blocks(const blr_plan *P);
// sweeps.cu: the deformation variant's forward solve (u^1..u^nt, m(1), rho^nt,
// energy partials), incremental state (du^nt and drho^nt into rho[0]) and adjoint
// (body force b from rho_final).
int sweep_state_def(blr_plan *P, cudaStream_t s);
int sweep_incremental_def(blr_plan *P, cudaStream_t s);
int sweep_adjoint_def(blr_plan *P, const float *rho_final, float *b, cudaStream_t s);
// The deformation variant's full Newton incremental adjoint: as sweep_adjoint_def from
// drho^nt in rho[0], with the second-order terms of newton.cu per component after every
// step (needs rho_all, du_all and newton_prep's weights).
int sweep_adjoint_def_newton(blr_plan *P, float *b, cudaStream_t s);

// reduce.cu
int energy_finalize(blr_plan *P, const float *vt, double *energy_out, int nblocks, cudaStream_t s);
// A plan's forward solve at vt (device), gradient and Gauss-Newton / full HVP at
// its current point, on stream s (api.cu; the batch runs its solo pairs through them).
int state_at(blr_plan *P, const float *vt, double *energy_out, cudaStream_t s);
int gradient_here(blr_plan *P, float *g, cudaStream_t s);
int hessvec_here(blr_plan *P, const float *dvt, float *hdv, cudaStream_t s);
int vec_dot(blr_plan *P, const float *a, const float *b, const float *w, double *out, cudaStream_t s);
int vec_maxabs(blr_plan *P, const float *a, double *out, cudaStream_t s);
int pcg_init(blr_plan *P, const float *rhs, float *x, cudaStream_t s);
// live: nullptr (batch members; the host decides) or P->pcg_live, in which case
// the update itself decides to stop (curvature, NaN, ||r|| / ||r0|| <= eta) and
// both kernels do nothing once it has.
int pcg_update(blr_plan *P, float *x, cudaStream_t s, int *live = nullptr, double eta = 0.0);
int pcg_direction(blr_plan *P, cudaStream_t s, const int *live = nullptr);
// PCG stop codes in pcg_live[1]
enum { PCG_RUN = 0, PCG_CURV = 1, PCG_NAN_PQ = 2, PCG_NAN_REL = 3 };
// y = a + alpha * x
int vec_axpy(blr_plan *P, float *y, const float *a, const float *x, double alpha, cudaStream_t s);
// out = P in, the Leray projector of the incompressible form (out may alias in)
int vec_leray(blr_plan *P, float *out, const float *in, cudaStream_t s);
int reduce_partials_needed();
