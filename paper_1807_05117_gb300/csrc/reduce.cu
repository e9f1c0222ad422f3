// Reductions and Krylov vector updates on band coefficients (Sections 3.2, 3.4).
//
// Energy (Eq. 35): E = 1/2 sum A |v~|^2 + sigma^-2 sum_x (m^nt - I1)^2, FP64.
// PCG (Eq. 55) with preconditioner K~ = 1/A: FP32 vectors, FP64 inner products
// and step scalars kept on the device.  Every reduction writes one partial per
// block and the last block to finish (ticket counter) sums the partials in
// block order, so results do not depend on scheduling.
#include "blr_internal.cuh"

namespace {

constexpr int RT = 256;        // threads of the vector kernels
constexpr int RBLOCKS = 120;   // blocks of the vector kernels

template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) t += red[w];
    return t;   // valid in thread 0
}

// Band index of float i of an interleaved complex [3][B1][B2][B3] array.
__device__ __forceinline__ long long coef_index(long long i, long long nb) {
    const long long c = i >> 1;
    return c < nb ? c : (c < 2 * nb ? c - nb : (c < 3 * nb ? c - 2 * nb : c % nb));
}

// Returns true in every thread of the last block to arrive.
__device__ __forceinline__ bool last_block(unsigned int *ticket) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    return is_last;
}

// Sum of `count` partial slots (stride `stride`, offset `slot`) by the whole
// block, in a fixed tree order (thread i takes slots i, i + RT, ... in order,
// then the block sum), so the result does not depend on scheduling.  Every
// thread calls it; the result is valid in thread 0.
__device__ __forceinline__ double ordered_sum(const double *part, int count, int stride, int slot,
                                              double *red) {
    double t = 0.0;
    for (int i = threadIdx.x; i < count; i += RT) t += part[i * stride + slot];
    return block_sum<RT>(t, red);
}

// Energy of Eq. 35: every block sums a strided share of the per-block image-term
// partials of the last state step and of A |v~|^2; the last block adds the
// block partials in block order.
__global__ void __launch_bounds__(RT)
k_energy(const double *__restrict__ partials, int np, const float *__restrict__ vt,
         const float *__restrict__ A, long long nb, int nvel, double wreg, double inv_sigma2,
         double *__restrict__ part2, unsigned int *ticket, double *__restrict__ sc,
         double *__restrict__ out, int *status) {
    pdl_wait();
    __shared__ double red[RT / 32];
    double sd = 0.0;
    for (int i = blockIdx.x * RT + threadIdx.x; i < np; i += gridDim.x * RT) sd += partials[i];
    sd = block_sum<RT>(sd, red);
    if (threadIdx.x == 0) part2[2 * blockIdx.x] = sd;
    double sr = 0.0;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < 3 * nb * nvel;
         i += (long long)gridDim.x * RT) {
        const long long kk = coef_index(2 * i, nb);
        const double re = vt[2 * i], im = vt[2 * i + 1];
        sr += (double)A[kk] * (re * re + im * im);
    }
    sr = block_sum<RT>(sr, red);
    if (threadIdx.x == 0) part2[2 * blockIdx.x + 1] = sr;
    if (!last_block(ticket)) return;
    const double sdt = ordered_sum(part2, gridDim.x, 2, 0, red);
    const double srt = ordered_sum(part2, gridDim.x, 2, 1, red);
    if (threadIdx.x == 0) {
        *ticket = 0;
        const double edata = sdt * inv_sigma2, ereg = 0.5 * wreg * srt, e = ereg + edata;
        sc[SC_E] = e;
        sc[SC_EREG] = ereg;
        sc[SC_EDATA] = edata;
        if (out) {
            out[0] = e;
            out[1] = ereg;
            out[2] = edata;
        }
        if (!isfinite(e)) atomicOr(status, BLR_FLAG_NAN);
    }
}

// out = sum a_i b_i (w == nullptr) or sum a_i b_i / w_{coef(i)} over 2*3*nb floats.
__global__ void __launch_bounds__(RT)
k_dot(const float *__restrict__ a, const float *__restrict__ b, const float *__restrict__ w,
      long long n, long long nb, double *__restrict__ part, unsigned int *ticket,
      double *__restrict__ out) {
    pdl_wait();
    __shared__ double red[RT / 32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        double t = (double)a[i] * (double)b[i];
        if (w) t /= (double)w[coef_index(i, nb)];
        acc += t;
    }
    acc = block_sum<RT>(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
    if (last_block(ticket)) {
        const double t = ordered_sum(part, gridDim.x, 1, 0, red);
        if (threadIdx.x == 0) {
            *out = t;
            *ticket = 0;
        }
    }
}

__global__ void __launch_bounds__(RT)
k_maxabs(const float *__restrict__ a, long long n, double *__restrict__ part,
         unsigned int *ticket, double *__restrict__ out) {
    pdl_wait();
    __shared__ float red[RT / 32];
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT)
        m = fmaxf(m, fabsf(a[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < RT / 32; ++w) t = fmaxf(t, red[w]);
        part[blockIdx.x] = (double)t;
    }
    if (last_block(ticket)) {
        double t = 0.0;
        for (unsigned i = threadIdx.x; i < gridDim.x; i += RT) t = fmax(t, part[i]);
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (float)t;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m2 = 0.f;
            for (int w = 0; w < RT / 32; ++w) m2 = fmaxf(m2, red[w]);
            *out = (double)m2;
            *ticket = 0;
        }
    }
}

// x = 0, r = rhs, p = rhs / A; rz = <r, r/A>, rr = <r, r>, rr0 = rr.
__global__ void __launch_bounds__(RT)
k_pcg_init(const float *__restrict__ rhs, float *__restrict__ x, float *__restrict__ r,
           float *__restrict__ p, const float *__restrict__ A, long long n, long long nb,
           double *__restrict__ part, unsigned int *ticket, double *__restrict__ sc) {
    pdl_wait();
    __shared__ double red[RT / 32];
    double rz = 0.0, rr = 0.0;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        const float ri = rhs[i];
        const float zi = ri / A[coef_index(i, nb)];
        x[i] = 0.f;
        r[i] = ri;
        p[i] = zi;
        rz += (double)ri * (double)zi;
        rr += (double)ri * (double)ri;
    }
    rz = block_sum<RT>(rz, red);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = rz;
    rr = block_sum<RT>(rr, red);
    if (threadIdx.x == 0) part[2 * blockIdx.x + 1] = rr;
    if (last_block(ticket)) {
        const double trz = ordered_sum(part, gridDim.x, 2, 0, red);
        const double trr = ordered_sum(part, gridDim.x, 2, 1, red);
        if (threadIdx.x == 0) {
            sc[SC_RZ] = trz;
            sc[SC_RR] = sc[SC_RR0] = trr;
            *ticket = 0;
        }
    }
}

// alpha = rz / <p, q>; x += alpha p; r -= alpha q; rz' = <r, r/A>, rr = <r, r>;
// beta = rz' / rz.  With `live` (device [running, code, updates]) the kernel
// also takes the stopping decision of the PCG loop: it does nothing once
// stopped, stops without updating when <p, q> is not positive (or NaN), and
// after an update stops when ||r|| / ||r0|| <= eta (or is NaN).
__global__ void __launch_bounds__(RT)
k_pcg_update(float *__restrict__ x, float *__restrict__ r, const float *__restrict__ p,
             const float *__restrict__ q, const float *__restrict__ A, long long n, long long nb,
             double *__restrict__ part, unsigned int *ticket, double *__restrict__ sc,
             const int *active, int *live, double eta) {
    pdl_wait();
    __shared__ double red[RT / 32];
    if (active && *active == 0) return;   // batch member whose PCG has stopped
    if (live && live[0] == 0) return;     // this plan's PCG has stopped
    const double pq = sc[SC_PQ];
    if (live && !(pq > 0.0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            live[1] = isfinite(pq) ? PCG_CURV : PCG_NAN_PQ;
            live[0] = 0;
        }
        return;
    }
    const double alpha_d = sc[SC_RZ] / pq;
    const float alpha = (float)alpha_d;
    double rz = 0.0, rr = 0.0;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        x[i] = fmaf(alpha, p[i], x[i]);
        const float ri = fmaf(-alpha, q[i], r[i]);
        r[i] = ri;
        const float zi = ri / A[coef_index(i, nb)];
        rz += (double)ri * (double)zi;
        rr += (double)ri * (double)ri;
    }
    rz = block_sum<RT>(rz, red);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = rz;
    rr = block_sum<RT>(rr, red);
    if (threadIdx.x == 0) part[2 * blockIdx.x + 1] = rr;
    if (last_block(ticket)) {
        const double rz_new = ordered_sum(part, gridDim.x, 2, 0, red);
        const double rr_new = ordered_sum(part, gridDim.x, 2, 1, red);
        if (threadIdx.x == 0) {
            sc[SC_BETA] = rz_new / sc[SC_RZ];
            sc[SC_ALPHA] = alpha_d;
            sc[SC_RZ] = rz_new;
            sc[SC_RR] = rr_new;
            if (live) {
                const double rel = sqrt(rr_new / sc[SC_RR0]);
                sc[SC_REL] = rel;
                live[2] += 1;
                if (!isfinite(rel)) {
                    live[1] = PCG_NAN_REL;
                    live[0] = 0;
                } else if (rel <= eta) {
                    live[0] = 0;
                }
            }
            *ticket = 0;
        }
    }
}

// p = r / A + beta p.
__global__ void __launch_bounds__(RT)
k_pcg_direction(float *__restrict__ p, const float *__restrict__ r, const float *__restrict__ A,
                long long n, long long nb, const double *__restrict__ sc, const int *active,
                const int *live) {
    pdl_wait();
    if (active && *active == 0) return;
    if (live && live[0] == 0) return;
    const float beta = (float)sc[SC_BETA];
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT)
        p[i] = fmaf(beta, p[i], r[i] / A[coef_index(i, nb)]);
}

// y = a + alpha x (FP32; alpha from the host).
__global__ void __launch_bounds__(RT)
k_axpy(float *__restrict__ y, const float *__restrict__ a, const float *__restrict__ x,
       float alpha, long long n) {
    pdl_wait();
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT)
        y[i] = fmaf(alpha, x[i], a[i]);
}

// Leray projection of band coefficients (the incompressible form: Eq. 4 with
// gamma = 1, imposed in the band): out(k) = P(k) in(k) with P(k) = I - kappa
// kappa^T / |kappa|^2, kappa_d proportional to k_d / N_d (the common factor 2 pi
// cancels), P(0) = I.  One thread per frequency, the three components' real and
// imaginary parts projected alike (P is real).  out may alias in.
__global__ void __launch_bounds__(RT)
k_leray(float2 *out, const float2 *in, long long nb, int B1, int B2, int B3, int N1, int N2,
        int N3) {
    pdl_wait();
    const float r1 = 1.0f / (float)N1, r2 = 1.0f / (float)N2, r3 = 1.0f / (float)N3;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < nb; i += (long long)gridDim.x * RT) {
        const int j3 = (int)(i % B3);
        const int j2 = (int)((i / B3) % B2);
        const int j1 = (int)(i / ((long long)B2 * B3));
        const float k1 = (float)(j1 - B1 / 2) * r1, k2 = (float)(j2 - B2 / 2) * r2,
                    k3 = (float)(j3 - B3 / 2) * r3;
        const float kk = k1 * k1 + k2 * k2 + k3 * k3;
        float2 a = in[i], b = in[nb + i], c = in[2 * nb + i];
        if (kk > 0.0f) {
            const float inv = 1.0f / kk;
            const float wr = (k1 * a.x + k2 * b.x + k3 * c.x) * inv;
            const float wi = (k1 * a.y + k2 * b.y + k3 * c.y) * inv;
            a.x -= k1 * wr; a.y -= k1 * wi;
            b.x -= k2 * wr; b.y -= k2 * wi;
            c.x -= k3 * wr; c.y -= k3 * wi;
        }
        out[i] = a;
        out[nb + i] = b;
        out[2 * nb + i] = c;
    }
}

int vec_blocks(const blr_plan *P) {
    long long b = ceil_div_ll(P->nfloat, RT);
    return (int)(b < RBLOCKS ? (b < 1 ? 1 : b) : RBLOCKS);
}

}  // namespace

int reduce_partials_needed() { return 2 * RBLOCKS; }

int energy_finalize(blr_plan *P, const float *vt, double *energy_out, int nblocks, cudaStream_t s) {
    launch_pdl(k_energy, dim3(vec_blocks(P)), dim3(RT), 0, s, (const double *)P->partials, nblocks,
               vt, (const float *)P->A, P->nb, P->nvel, P->nvel > 1 ? 1.0 / P->p.nt : 1.0,
               1.0 / (P->p.sigma * P->p.sigma), P->partials2,
               P->ticket, P->dsc, energy_out, P->dstatus);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int vec_dot(blr_plan *P, const float *a, const float *b, const float *w, double *out, cudaStream_t s) {
    launch_pdl(k_dot, dim3(vec_blocks(P)), dim3(RT), 0, s, a, b, w, P->nfloat, P->nb, P->partials,
               P->ticket, out);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int vec_maxabs(blr_plan *P, const float *a, double *out, cudaStream_t s) {
    launch_pdl(k_maxabs, dim3(vec_blocks(P)), dim3(RT), 0, s, a, P->nfloat, P->partials, P->ticket,
               out);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int pcg_init(blr_plan *P, const float *rhs, float *x, cudaStream_t s) {
    launch_pdl(k_pcg_init, dim3(vec_blocks(P)), dim3(RT), 0, s, rhs, x, P->r, P->pv,
               (const float *)P->A, P->nfloat, P->nb, P->partials, P->ticket, P->dsc);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int pcg_update(blr_plan *P, float *x, cudaStream_t s, int *live, double eta) {
    launch_pdl(k_pcg_update, dim3(vec_blocks(P)), dim3(RT), 0, s, x, P->r, (const float *)P->pv,
               (const float *)P->q, (const float *)P->A, P->nfloat, P->nb, P->partials, P->ticket,
               P->dsc, P->active, live, eta);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int pcg_direction(blr_plan *P, cudaStream_t s, const int *live) {
    launch_pdl(k_pcg_direction, dim3(vec_blocks(P)), dim3(RT), 0, s, P->pv, (const float *)P->r,
               (const float *)P->A, P->nfloat, P->nb, (const double *)P->dsc, P->active, live);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int vec_axpy(blr_plan *P, float *y, const float *a, const float *x, double alpha, cudaStream_t s) {
    launch_pdl(k_axpy, dim3(vec_blocks(P)), dim3(RT), 0, s, y, a, x, (float)alpha, P->nfloat);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int vec_leray(blr_plan *P, float *out, const float *in, cudaStream_t s) {
    long long b = ceil_div_ll(P->nb, RT);
    const int blocks = (int)(b < RBLOCKS ? (b < 1 ? 1 : b) : RBLOCKS);
    for (int v = 0; v < P->nvel; ++v) {   // one launch per velocity of the parameter vector
        launch_pdl(k_leray, dim3(blocks), dim3(RT), 0, s,
                   reinterpret_cast<float2 *>(out + (size_t)v * P->nf1),
                   reinterpret_cast<const float2 *>(in + (size_t)v * P->nf1), P->nb, P->B1, P->B2,
                   P->B3, P->N1, P->N2, P->N3);
        BLR_CK_LAUNCH();
    }
    return BLR_OK;
}
