// Semi-Lagrangian sweeps of the state, adjoint and incremental equations
// (Section 3.2, Eqs. 36, 38, 44-46 with the Gauss-Newton drops of Section 3.4),
// discretised as: m^{n+1}(x) = trilinear value of m^n at x + d(x), periodic,
// d = -dt iota(v~) clamped to [-1, 1) (the plan latches BLR_ECFL otherwise).
//
// Per axis a the displacement d_a selects the cell {x_a - 1, x_a} when d_a < 0
// (weights -d_a, 1 + d_a) and {x_a, x_a + 1} otherwise (weights 1 - d_a, d_a):
// the floor-of-displacement cell rule.  The same weights written as the hat
// function h(t) = max(0, 1 - |t|) at t = d_a - e_a (e_a = y_a - x_a in {-1,0,1})
// give the exact transpose S^T as a 27-neighbour gather, so the adjoint needs
// no atomics and is deterministic.
//
// Every kernel stages the fields it interpolates in shared memory as a tile of
// TI x TJ x TK voxels plus a one-voxel halo (periodic wrap on load); the
// per-voxel inputs (d, dv) and outputs stream through registers.
#include "blr_internal.cuh"

namespace {

__device__ __forceinline__ int wrapi(int i, int N) {
    int r = i % N;
    return r < 0 ? r + N : r;
}

// Offsets (within one x1-plane) of the halo positions p and p + SWEEP_THREADS.
struct PlaneSlots {
    long long off0, off1;
    bool ok1;
};

__device__ __forceinline__ PlaneSlots plane_slots(const Grid3 &g, int k0, int j0) {
    PlaneSlots ps;
    int p = threadIdx.x;
    int hj = p / HK, hk = p - hj * HK;
    ps.off0 = (long long)wrapi(j0 + hj - 1, g.N2) * g.N3 + wrapi(k0 + hk - 1, g.N3);
    p += SWEEP_THREADS;
    ps.ok1 = p < HJK;
    hj = p / HK;
    hk = p - hj * HK;
    ps.off1 = ps.ok1 ? (long long)wrapi(j0 + hj - 1, g.N2) * g.N3 + wrapi(k0 + hk - 1, g.N3) : 0;
    return ps;
}

__device__ __forceinline__ void load_scalar_halo(float *s, const float *__restrict__ f,
                                                 const Grid3 &g, const PlaneSlots &ps, int i0) {
    const long long plane = (long long)g.N2 * g.N3;
    for (int hi = 0; hi < HI; ++hi) {
        const float *fp = f + (long long)wrapi(i0 + hi - 1, g.N1) * plane;
        s[hi * HJK + threadIdx.x] = __ldg(fp + ps.off0);
        if (ps.ok1) s[hi * HJK + threadIdx.x + SWEEP_THREADS] = __ldg(fp + ps.off1);
    }
}

// (d0, d1, d2, lambda) per halo voxel.
__device__ __forceinline__ void load_dlam_halo(float4 *s, const float *__restrict__ d,
                                               const float *__restrict__ lam, const Grid3 &g,
                                               const PlaneSlots &ps, int i0) {
    const long long plane = (long long)g.N2 * g.N3;
    for (int hi = 0; hi < HI; ++hi) {
        long long base = (long long)wrapi(i0 + hi - 1, g.N1) * plane;
        long long o = base + ps.off0;
        s[hi * HJK + threadIdx.x] =
            make_float4(__ldg(d + o), __ldg(d + g.V + o), __ldg(d + 2 * g.V + o), __ldg(lam + o));
        if (ps.ok1) {
            o = base + ps.off1;
            s[hi * HJK + threadIdx.x + SWEEP_THREADS] = make_float4(
                __ldg(d + o), __ldg(d + g.V + o), __ldg(d + 2 * g.V + o), __ldg(lam + o));
        }
    }
}

struct AxisW {
    int lo;
    float wl, wh;
};

// Cell and weights of one axis for a displacement in [-1, 1).
__device__ __forceinline__ AxisW axis_weights(float d) {
    AxisW a;
    if (d < 0.f) {
        a.lo = -1;
        a.wl = -d;
        a.wh = 1.f + d;
    } else {
        a.lo = 0;
        a.wl = 1.f - d;
        a.wh = d;
    }
    return a;
}

// Weight that a neighbour with displacement d gives to the voxel at offset e
// (e = target - neighbour): the hat function at d - e, for |d| < 1.
template <int E>
__device__ __forceinline__ float hat(float d) {
    if (E == 0) return 1.f - fabsf(d);
    if (E == 1) return fmaxf(d, 0.f);
    return fmaxf(-d, 0.f);
}

// Trilinear value (and optionally the exact gradient of the cell's trilinear
// polynomial) of the halo tile s at halo coordinates (hi, hj, hk) + cell.
template <bool GRAD>
__device__ __forceinline__ float trilinear(const float *s, int hi, int hj, int hk, AxisW a0,
                                           AxisW a1, AxisW a2, float *G) {
    const int b = (hi + a0.lo) * HJK + (hj + a1.lo) * HK + (hk + a2.lo);
    const float c000 = s[b], c001 = s[b + 1], c010 = s[b + HK], c011 = s[b + HK + 1];
    const float c100 = s[b + HJK], c101 = s[b + HJK + 1], c110 = s[b + HJK + HK],
                c111 = s[b + HJK + HK + 1];
    const float l00 = fmaf(a2.wl, c000, a2.wh * c001), l01 = fmaf(a2.wl, c010, a2.wh * c011);
    const float l10 = fmaf(a2.wl, c100, a2.wh * c101), l11 = fmaf(a2.wl, c110, a2.wh * c111);
    const float m0 = fmaf(a1.wl, l00, a1.wh * l01), m1 = fmaf(a1.wl, l10, a1.wh * l11);
    if (GRAD) {
        G[0] = m1 - m0;
        G[1] = fmaf(a0.wl, l01 - l00, a0.wh * (l11 - l10));
        const float e0 = fmaf(a1.wl, c001 - c000, a1.wh * (c011 - c010));
        const float e1 = fmaf(a1.wl, c101 - c100, a1.wh * (c111 - c110));
        G[2] = fmaf(a0.wl, e0, a0.wh * e1);
    }
    return fmaf(a0.wl, m0, a0.wh * m1);
}

__device__ __forceinline__ double block_sum_256(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < SWEEP_THREADS / 32; ++w) t += red[w];
    return t;
}

__device__ __forceinline__ long long block_linear() {
    return ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
}

// ---------------------------------------------------------------------------
// State step m^{n+1} = S m^n.  LAST also writes lambda^nt = lam_scale (m^nt - I1)
// and the block's sum of (m^nt - I1)^2 (FP32 terms, FP64 block sum).
template <bool LAST>
__global__ void __launch_bounds__(SWEEP_THREADS)
k_state_step(const float *__restrict__ m_in, const float *__restrict__ d,
             float *__restrict__ m_out, Grid3 g, const float *__restrict__ I1,
             float *__restrict__ lam_out, float lam_scale, double *__restrict__ partials) {
    __shared__ float s[HI * HJK];
    __shared__ double red[SWEEP_THREADS / 32];
    const int k0 = blockIdx.x * TK, j0 = blockIdx.y * TJ, i0 = blockIdx.z * TI;
    const PlaneSlots ps = plane_slots(g, k0, j0);
    load_scalar_halo(s, m_in, g, ps, i0);
    __syncthreads();
    const int tk = threadIdx.x & 31, tj = threadIdx.x >> 5;
    const int k = k0 + tk, j = j0 + tj;
    float e2 = 0.f;
    if (k < g.N3 && j < g.N2) {
        for (int t = 0; t < TI; ++t) {
            const int i = i0 + t;
            if (i >= g.N1) break;
            const long long idx = ((long long)i * g.N2 + j) * g.N3 + k;
            const AxisW a0 = axis_weights(__ldg(d + idx));
            const AxisW a1 = axis_weights(__ldg(d + g.V + idx));
            const AxisW a2 = axis_weights(__ldg(d + 2 * g.V + idx));
            const float val = trilinear<false>(s, t + 1, tj + 1, tk + 1, a0, a1, a2, nullptr);
            m_out[idx] = val;
            if (LAST) {
                const float r = val - __ldg(I1 + idx);
                e2 = fmaf(r, r, e2);
                lam_out[idx] = lam_scale * r;
            }
        }
    }
    if (LAST) {
        const double t = block_sum_256((double)e2, red);
        if (threadIdx.x == 0) partials[block_linear()] = t;
    }
}

// ---------------------------------------------------------------------------
// Adjoint step at time n (also the Gauss-Newton incremental adjoint):
//   b(x) (+)= dt lambda^{n+1}(x) grad m^n(x + d(x))     (body force)
//   lambda^n(y) = sum_{e in {-1,0,1}^3} lambda^{n+1}(y-e) prod_a hat(d_a(y-e) - e_a)
template <bool FIRST, bool WRITE_LAM>
__global__ void __launch_bounds__(SWEEP_THREADS, 3)
k_adjoint_step(const float *__restrict__ lam_in, const float *__restrict__ m_n,
               const float *__restrict__ d, float *__restrict__ lam_out,
               float *__restrict__ b, float dt, Grid3 g) {
    extern __shared__ float4 smem4[];
    float4 *sq = smem4;
    float *sm = reinterpret_cast<float *>(smem4 + HI * HJK);
    const int k0 = blockIdx.x * TK, j0 = blockIdx.y * TJ, i0 = blockIdx.z * TI;
    const PlaneSlots ps = plane_slots(g, k0, j0);
    load_dlam_halo(sq, d, lam_in, g, ps, i0);
    load_scalar_halo(sm, m_n, g, ps, i0);
    __syncthreads();
    const int tk = threadIdx.x & 31, tj = threadIdx.x >> 5;
    const int k = k0 + tk, j = j0 + tj;
    if (k >= g.N3 || j >= g.N2) return;
    for (int t = 0; t < TI; ++t) {
        const int i = i0 + t;
        if (i >= g.N1) break;
        const long long idx = ((long long)i * g.N2 + j) * g.N3 + k;
        const int c = (t + 1) * HJK + (tj + 1) * HK + (tk + 1);
        const float4 q = sq[c];
        float G[3];
        trilinear<true>(sm, t + 1, tj + 1, tk + 1, axis_weights(q.x), axis_weights(q.y),
                        axis_weights(q.z), G);
        const float sl = dt * q.w;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float *bp = b + a * g.V + idx;
            *bp = FIRST ? sl * G[a] : fmaf(sl, G[a], *bp);
        }
        if (WRITE_LAM) {
            float acc = 0.f;
#define BLR_NB(E0, E1, E2)                                                           \
    {                                                                                \
        const float4 n = sq[c - (E0) * HJK - (E1) * HK - (E2)];                     \
        acc = fmaf(hat<E0>(n.x) * hat<E1>(n.y) * hat<E2>(n.z), n.w, acc);           \
    }
#define BLR_NB3(E0, E1) BLR_NB(E0, E1, -1) BLR_NB(E0, E1, 0) BLR_NB(E0, E1, 1)
#define BLR_NB9(E0) BLR_NB3(E0, -1) BLR_NB3(E0, 0) BLR_NB3(E0, 1)
            BLR_NB9(-1) BLR_NB9(0) BLR_NB9(1)
#undef BLR_NB9
#undef BLR_NB3
#undef BLR_NB
            lam_out[idx] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Incremental state step (linearised Eq. 36):
//   dm^{n+1}(x) = (S dm^n)(x) - dt grad m^n(x + d(x)) . dv(x),   dm^0 = 0.
// LAST writes dlambda^nt = lam_scale dm^nt instead of dm^nt.
template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(SWEEP_THREADS)
k_incstate_step(const float *__restrict__ dm_in, const float *__restrict__ m_n,
                const float *__restrict__ d, const float *__restrict__ dv,
                float *__restrict__ dm_out, float dt, float lam_scale, Grid3 g) {
    __shared__ float sm[HI * HJK];
    __shared__ float sdm[FIRST ? 1 : HI * HJK];
    const int k0 = blockIdx.x * TK, j0 = blockIdx.y * TJ, i0 = blockIdx.z * TI;
    const PlaneSlots ps = plane_slots(g, k0, j0);
    load_scalar_halo(sm, m_n, g, ps, i0);
    if (!FIRST) load_scalar_halo(sdm, dm_in, g, ps, i0);
    __syncthreads();
    const int tk = threadIdx.x & 31, tj = threadIdx.x >> 5;
    const int k = k0 + tk, j = j0 + tj;
    if (k >= g.N3 || j >= g.N2) return;
    for (int t = 0; t < TI; ++t) {
        const int i = i0 + t;
        if (i >= g.N1) break;
        const long long idx = ((long long)i * g.N2 + j) * g.N3 + k;
        const AxisW a0 = axis_weights(__ldg(d + idx));
        const AxisW a1 = axis_weights(__ldg(d + g.V + idx));
        const AxisW a2 = axis_weights(__ldg(d + 2 * g.V + idx));
        float G[3];
        trilinear<true>(sm, t + 1, tj + 1, tk + 1, a0, a1, a2, G);
        float out = FIRST ? 0.f : trilinear<false>(sdm, t + 1, tj + 1, tk + 1, a0, a1, a2, nullptr);
        const float gdv = fmaf(G[0], __ldg(dv + idx),
                               fmaf(G[1], __ldg(dv + g.V + idx), G[2] * __ldg(dv + 2 * g.V + idx)));
        out = fmaf(-dt, gdv, out);
        dm_out[idx] = LAST ? lam_scale * out : out;
    }
}

constexpr size_t ADJ_SMEM = HI * HJK * (sizeof(float4) + sizeof(float));

dim3 sweep_grid(const blr_plan *P) {
    return dim3((unsigned)ceil_div_ll(P->N3, TK), (unsigned)ceil_div_ll(P->N2, TJ),
                (unsigned)ceil_div_ll(P->N1, TI));
}

template <bool F, bool W>
int launch_adjoint(dim3 grid, cudaStream_t s, const float *lin, const float *mn, const float *d,
                   float *lout, float *b, float dt, Grid3 g) {
    k_adjoint_step<F, W><<<grid, SWEEP_THREADS, ADJ_SMEM, s>>>(lin, mn, d, lout, b, dt, g);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

}  // namespace

// Opt the adjoint kernels into their dynamic shared memory on the current device.
int sweep_setup() {
    BLR_CK(cudaFuncSetAttribute(k_adjoint_step<true, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ADJ_SMEM));
    BLR_CK(cudaFuncSetAttribute(k_adjoint_step<true, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ADJ_SMEM));
    BLR_CK(cudaFuncSetAttribute(k_adjoint_step<false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ADJ_SMEM));
    BLR_CK(cudaFuncSetAttribute(k_adjoint_step<false, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ADJ_SMEM));
    return BLR_OK;
}

long long sweep_blocks(const blr_plan *P) {
    dim3 gr = sweep_grid(P);
    return (long long)gr.x * gr.y * gr.z;
}

int sweep_state(blr_plan *P, cudaStream_t s) {
    const dim3 grid = sweep_grid(P);
    const int nt = P->p.nt;
    const float lam_scale = (float)(-2.0 / (P->p.sigma * P->p.sigma));
    for (int n = 0; n < nt; ++n) {
        const float *min_ = P->m + (long long)n * P->V;
        float *mout = P->m + (long long)(n + 1) * P->V;
        if (n == nt - 1)
            k_state_step<true><<<grid, SWEEP_THREADS, 0, s>>>(min_, P->d, mout, P->grid, P->I1,
                                                              P->lam[0], lam_scale, P->partials);
        else
            k_state_step<false><<<grid, SWEEP_THREADS, 0, s>>>(min_, P->d, mout, P->grid, nullptr,
                                                               nullptr, 0.f, nullptr);
        BLR_CK_LAUNCH();
    }
    return BLR_OK;
}

// lambda^nt must be in lam[0].  Writes the body force into b (3V) and, when
// lambda0 != nullptr, lambda^0 into lambda0.
int sweep_adjoint(blr_plan *P, float *b, float *lambda0, cudaStream_t s) {
    const dim3 grid = sweep_grid(P);
    const int nt = P->p.nt;
    int cur = 0;
    for (int n = nt - 1; n >= 0; --n) {
        const float *lin = P->lam[cur];
        float *lout = (n == 0 && lambda0) ? lambda0 : P->lam[1 - cur];
        const float *mn = P->m + (long long)n * P->V;
        const bool first = (n == nt - 1);
        const bool wlam = (n > 0) || (lambda0 != nullptr);
        int rc;
        if (first && wlam) rc = launch_adjoint<true, true>(grid, s, lin, mn, P->d, lout, b, P->dt, P->grid);
        else if (first) rc = launch_adjoint<true, false>(grid, s, lin, mn, P->d, lout, b, P->dt, P->grid);
        else if (wlam) rc = launch_adjoint<false, true>(grid, s, lin, mn, P->d, lout, b, P->dt, P->grid);
        else rc = launch_adjoint<false, false>(grid, s, lin, mn, P->d, lout, b, P->dt, P->grid);
        if (rc != BLR_OK) return rc;
        cur = 1 - cur;
    }
    return BLR_OK;
}

// Incremental state from dv = iota(dv~) (in P->dv); leaves dlambda^nt in lam[0].
int sweep_incremental(blr_plan *P, cudaStream_t s) {
    const dim3 grid = sweep_grid(P);
    const int nt = P->p.nt;
    const float lam_scale = (float)(-2.0 / (P->p.sigma * P->p.sigma));
    int cur = 0;
    for (int n = 0; n < nt; ++n) {
        const float *din = P->dm[cur];
        float *dout = (n == nt - 1) ? P->lam[0] : P->dm[1 - cur];
        const float *mn = P->m + (long long)n * P->V;
        const bool first = n == 0, last = n == nt - 1;
        if (first && last)
            k_incstate_step<true, true><<<grid, SWEEP_THREADS, 0, s>>>(din, mn, P->d, P->dv, dout, P->dt, lam_scale, P->grid);
        else if (first)
            k_incstate_step<true, false><<<grid, SWEEP_THREADS, 0, s>>>(din, mn, P->d, P->dv, dout, P->dt, lam_scale, P->grid);
        else if (last)
            k_incstate_step<false, true><<<grid, SWEEP_THREADS, 0, s>>>(din, mn, P->d, P->dv, dout, P->dt, lam_scale, P->grid);
        else
            k_incstate_step<false, false><<<grid, SWEEP_THREADS, 0, s>>>(din, mn, P->d, P->dv, dout, P->dt, lam_scale, P->grid);
        BLR_CK_LAUNCH();
        cur = 1 - cur;
    }
    return BLR_OK;
}
