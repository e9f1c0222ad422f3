// Second-order terms of the full Newton Hessian (Eqs. 44-46 without the drops
// of Section 3.4), applied once per time step inside the incremental adjoint
// sweep (sweep_adjoint_newton in sweeps.cu).
//
// With dd = -dt iota(dv~) and lambda^{n+1} the gradient's adjoint state, step n adds
//   b(y)         += dt lambda^{n+1}(y) [D dm^n(y) + Hess T[m^n](y + d(y)) dd(y)]
//   dlambda^n(y) += sum_x lambda^{n+1}(x) sum_a dd_a(x) d_a w(x -> y)
// to what the Gauss-Newton step computes (b += dt dlambda^{n+1} grad m^n and
// dlambda^n = S^T dlambda^{n+1}).  The first line is pi(lambda grad dm) of Eq. 46
// together with the move of the departure point inside its cell (the second
// derivatives of the trilinear polynomial of m^n: only the mixed ones are
// non-zero); the second is the variation of S^T, the dJ term of the
// incremental adjoint (Eq. 45).  w(x -> y) is the trilinear weight that voxel x
// gives corner y of its cell and d_a w its derivative in the departure point.
//
// The variation of S^T is a transpose whose weights, kappa_o(x) = sum_a dd_a(x)
// d_a w_o(x) for the 8 corners o of the cell of x, do not change from step to
// step.  k_newton_prep scatters them once per product into a 27-point stencil
// K_e(y) = kappa_o(x) for y = x + e the corner o of the cell of x (zero where y
// is no corner of its neighbour's cell; every (y, e) is written by at most one
// x, so the scatter needs no atomics), and each step applies
// dlambda^n(y) += sum_e K_e(y) lambda^{n+1}(y - e) over the 27 offsets in a fixed
// order: dense, coalesced loads instead of a dependent load per neighbour, and
// the sum of the earlier per-neighbour gather (which skipped the zero terms) bit
// for bit.  One thread per voxel; the cell rule is the sweeps': on each axis the
// cell starts at -1 for d < 0 and at 0 otherwise.
#include "blr_internal.cuh"

namespace {

constexpr int NK = 32, NJ = 8;   // block: 32 voxels along x3 x 8 rows along x2

struct Cell1 {
    int lo;         // cell start offset (-1 or 0)
    float wl, wh;   // weights of the low and high corner
};

__device__ __forceinline__ Cell1 cell_of(float d) {
    Cell1 c;
    if (d < 0.f) {
        c.lo = -1;
        c.wl = -d;
        c.wh = 1.f + d;
    } else {
        c.lo = 0;
        c.wl = 1.f - d;
        c.wh = d;
    }
    return c;
}

__device__ __forceinline__ int wrap(int s, int N) { return s < 0 ? s + N : (s >= N ? s - N : s); }

// The 8 corner values of f around cell (i + c0.lo, j + c1.lo, k + c2.lo), c[o0][o1][o2].
__device__ __forceinline__ void corners(const float *__restrict__ f, int i, int j, int k,
                                        const Cell1 &c0, const Cell1 &c1, const Cell1 &c2,
                                        const Grid3 &g, float c[2][2][2]) {
    const long long plane = (long long)g.N2 * g.N3;
    const long long p[2] = {(long long)wrap(i + c0.lo, g.N1) * plane,
                            (long long)wrap(i + c0.lo + 1, g.N1) * plane};
    const long long r[2] = {(long long)wrap(j + c1.lo, g.N2) * g.N3,
                            (long long)wrap(j + c1.lo + 1, g.N2) * g.N3};
    const int q[2] = {wrap(k + c2.lo, g.N3), wrap(k + c2.lo + 1, g.N3)};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e) c[a][b][e] = __ldg(f + p[a] + r[b] + q[e]);
}

// Per voxel x and offset e: K[e][x + e] = kappa_o(x) = sum_a dd_a d_a w_o when
// x + e is the corner o = 4 o0 + 2 o1 + o2 of the cell of x (e_a = lo_a + o_a,
// periodic; dd = -dt dv), else 0.  K is [27][V], e indexed (e0 + 1) 9 + (e1 + 1) 3
// + (e2 + 1); every entry is written exactly once (by x = y - e).
__global__ void __launch_bounds__(256)
k_newton_prep(const float *__restrict__ d, const float *__restrict__ dv, float dt,
              float *__restrict__ K, Grid3 g) {
    pdl_wait();
    const long long V = g.V, plane = (long long)g.N2 * g.N3;
    for (long long x = blockIdx.x * 256LL + threadIdx.x; x < V; x += (long long)gridDim.x * 256) {
        const Cell1 c[3] = {cell_of(__ldg(d + x)), cell_of(__ldg(d + V + x)),
                            cell_of(__ldg(d + 2 * V + x))};
        const float dd[3] = {-dt * __ldg(dv + x), -dt * __ldg(dv + V + x),
                             -dt * __ldg(dv + 2 * V + x)};
        const int i = (int)(x / plane), j = (int)((x - (long long)i * plane) / g.N3);
        const int k = (int)(x - (long long)i * plane - (long long)j * g.N3);
#pragma unroll
        for (int e0 = -1; e0 <= 1; ++e0) {
            const int o0 = e0 - c[0].lo;   // corner bit on axis 0 (0 or 1 when a corner)
            const long long py = (long long)wrap(i + e0, g.N1) * plane;
#pragma unroll
            for (int e1 = -1; e1 <= 1; ++e1) {
                const int o1 = e1 - c[1].lo;
                const long long ry = py + (long long)wrap(j + e1, g.N2) * g.N3;
#pragma unroll
                for (int e2 = -1; e2 <= 1; ++e2) {
                    const int o2 = e2 - c[2].lo;
                    float kap = 0.f;
                    if (o0 >= 0 && o0 <= 1 && o1 >= 0 && o1 <= 1 && o2 >= 0 && o2 <= 1) {
                        const float u0 = o0 ? c[0].wh : c[0].wl, u1 = o1 ? c[1].wh : c[1].wl,
                                    u2 = o2 ? c[2].wh : c[2].wl;
                        const float s0 = o0 ? dd[0] : -dd[0], s1 = o1 ? dd[1] : -dd[1],
                                    s2 = o2 ? dd[2] : -dd[2];
                        kap = s0 * u1 * u2 + u0 * s1 * u2 + u0 * u1 * s2;
                    }
                    K[(long long)((e0 + 1) * 9 + (e1 + 1) * 3 + (e2 + 1)) * V + ry +
                      wrap(k + e2, g.N3)] = kap;
                }
            }
        }
    }
}

// One stencil term: the neighbour x = y - e contributes K_e(y) lambda(x).
template <int E0, int E1, int E2>
__device__ __forceinline__ void stencil_one(const float *__restrict__ K,
                                            const float *__restrict__ lam1, long long V,
                                            long long y, const long long *p, const long long *r,
                                            const int *q, float &acc) {
    const long long x = p[E0 + 1] + r[E1 + 1] + q[E2 + 1];
    acc = fmaf(__ldg(K + (long long)((E0 + 1) * 9 + (E1 + 1) * 3 + (E2 + 1)) * V + y),
               __ldg(lam1 + x), acc);
}

template <bool TRANSPOSE_TERM, bool HAVE_DM>
__global__ void __launch_bounds__(NK *NJ)
k_newton_terms(const float *__restrict__ d, const float *__restrict__ dv,
               const float *__restrict__ lam1, const float *__restrict__ mn,
               const float *__restrict__ dmn, const float *__restrict__ K,
               float *__restrict__ dlam, float *__restrict__ b, float dt, Grid3 g) {
    pdl_wait();
    const int k = blockIdx.x * NK + (threadIdx.x & (NK - 1));
    const int j = blockIdx.y * NJ + (threadIdx.x / NK);
    const int i = blockIdx.z;
    if (k >= g.N3 || j >= g.N2) return;
    const long long plane = (long long)g.N2 * g.N3;
    const long long y = (long long)i * plane + (long long)j * g.N3 + k;
    const long long V = g.V;

    // --- the body-force terms at y --------------------------------------------
    const Cell1 c0 = cell_of(__ldg(d + y)), c1 = cell_of(__ldg(d + V + y)),
                c2 = cell_of(__ldg(d + 2 * V + y));
    const float w0[2] = {c0.wl, c0.wh}, w1[2] = {c1.wl, c1.wh}, w2[2] = {c2.wl, c2.wh};
    float m[2][2][2];
    corners(mn, i, j, k, c0, c1, c2, g, m);
    // mixed second partials of the cell polynomial of m^n
    const float h01 = w2[0] * (m[1][1][0] - m[1][0][0] - m[0][1][0] + m[0][0][0]) +
                      w2[1] * (m[1][1][1] - m[1][0][1] - m[0][1][1] + m[0][0][1]);
    const float h02 = w1[0] * (m[1][0][1] - m[1][0][0] - m[0][0][1] + m[0][0][0]) +
                      w1[1] * (m[1][1][1] - m[1][1][0] - m[0][1][1] + m[0][1][0]);
    const float h12 = w0[0] * (m[0][1][1] - m[0][1][0] - m[0][0][1] + m[0][0][0]) +
                      w0[1] * (m[1][1][1] - m[1][1][0] - m[1][0][1] + m[1][0][0]);
    const float dd0 = -dt * __ldg(dv + y), dd1 = -dt * __ldg(dv + V + y),
                dd2 = -dt * __ldg(dv + 2 * V + y);
    float t0 = h01 * dd1 + h02 * dd2;
    float t1 = h01 * dd0 + h12 * dd2;
    float t2 = h02 * dd0 + h12 * dd1;
    if constexpr (HAVE_DM) {
        float c[2][2][2];
        corners(dmn, i, j, k, c0, c1, c2, g, c);
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;   // gradient of the cell polynomial of dm^n
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                g0 += w1[a] * w2[e] * (c[1][a][e] - c[0][a][e]);
                g1 += w0[a] * w2[e] * (c[a][1][e] - c[a][0][e]);
                g2 += w0[a] * w1[e] * (c[a][e][1] - c[a][e][0]);
            }
        t0 += g0;
        t1 += g1;
        t2 += g2;
    }
    const float sl = dt * __ldg(lam1 + y);
    b[y] = fmaf(sl, t0, b[y]);
    b[V + y] = fmaf(sl, t1, b[V + y]);
    b[2 * V + y] = fmaf(sl, t2, b[2 * V + y]);

    // --- the variation of S^T: gather over the neighbours x = y - e -----------
    if constexpr (TRANSPOSE_TERM) {
        const long long p[3] = {(long long)wrap(i + 1, g.N1) * plane, (long long)i * plane,
                                (long long)wrap(i - 1, g.N1) * plane};   // index e0 + 1
        const long long r[3] = {(long long)wrap(j + 1, g.N2) * g.N3, (long long)j * g.N3,
                                (long long)wrap(j - 1, g.N2) * g.N3};
        const int q[3] = {wrap(k + 1, g.N3), k, wrap(k - 1, g.N3)};
        float acc = 0.f;
#define BLR_G(A, B, C) stencil_one<A, B, C>(K, lam1, V, y, p, r, q, acc)
        BLR_G(-1, -1, -1); BLR_G(-1, -1, 0); BLR_G(-1, -1, 1);
        BLR_G(-1, 0, -1);  BLR_G(-1, 0, 0);  BLR_G(-1, 0, 1);
        BLR_G(-1, 1, -1);  BLR_G(-1, 1, 0);  BLR_G(-1, 1, 1);
        BLR_G(0, -1, -1);  BLR_G(0, -1, 0);  BLR_G(0, -1, 1);
        BLR_G(0, 0, -1);   BLR_G(0, 0, 0);   BLR_G(0, 0, 1);
        BLR_G(0, 1, -1);   BLR_G(0, 1, 0);   BLR_G(0, 1, 1);
        BLR_G(1, -1, -1);  BLR_G(1, -1, 0);  BLR_G(1, -1, 1);
        BLR_G(1, 0, -1);   BLR_G(1, 0, 0);   BLR_G(1, 0, 1);
        BLR_G(1, 1, -1);   BLR_G(1, 1, 0);   BLR_G(1, 1, 1);
#undef BLR_G
        dlam[y] += acc;
    }
}

}  // namespace

int newton_prep(blr_plan *P, cudaStream_t s) {
    long long blocks = ceil_div_ll(P->V, 256);
    const long long cap = (long long)P->sms * 8;
    if (blocks > cap) blocks = cap;
    launch_pdl(k_newton_prep, dim3((unsigned)blocks), dim3(256), 0, s, (const float *)P->d,
               (const float *)P->dv, P->dt, P->nt_kap, P->grid);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int newton_terms(blr_plan *P, bool transpose_term, const float *lam1, const float *mn,
                 const float *dmn, float *dlam, float *b, cudaStream_t s) {
    const dim3 grid((unsigned)ceil_div_ll(P->N3, NK), (unsigned)ceil_div_ll(P->N2, NJ),
                    (unsigned)P->N1);
    const dim3 block(NK * NJ);
#define BLR_NT(TT, DM)                                                                       \
    launch_pdl(k_newton_terms<TT, DM>, grid, block, 0, s, (const float *)P->d,                \
               (const float *)P->dv, lam1, mn, dmn, (const float *)P->nt_kap, dlam, b,    \
               P->dt, P->grid)
    if (transpose_term && dmn) BLR_NT(true, true);
    else if (transpose_term) BLR_NT(true, false);
    else if (dmn) BLR_NT(false, true);
    else BLR_NT(false, false);
#undef BLR_NT
    BLR_CK_LAUNCH();
    return BLR_OK;
}
