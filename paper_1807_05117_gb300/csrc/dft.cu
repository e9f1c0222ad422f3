// Truncated DFTs of the band-limited space (Section 3.1, Eq. 33), FP32 path.
//
// iota(v~)_c(x) = Re sum_k v~_c(k) e^{2 pi i k.x/N} is evaluated as three
// axis-wise contractions against small DFT tables:
//   stage A (axis 3): A1[c,k1,k2,x3] = sum_k3 v~[c,k1,k2,k3] E3[k3,x3]          complex
//   stage B (axis 2): A2[c,k1,x2,x3] = sum_k2 E2[k2,x2] A1[c,k1,k2,x3]          complex
//   stage C (axis 1): v[c,x1,x2,x3]  = sum_{k1,re/im} W1[(k1,re/im), x1] A2[...] real GEMM
// pi = iota^T runs the transposed stages in reverse order (C', B', A').
// Intermediates are planar: [slab = c*B1 + k1][re|im][row][x3].
#include "blr_internal.cuh"

namespace {

__device__ inline void phase_cs(int k, int x, int N, double *c, double *s) {
    long long r = ((long long)k * (long long)x) % N;   // exact integer phase
    if (r < 0) r += N;
    sincospi(2.0 * (double)r / (double)N, s, c);
}

// T[j][x] = cos / sin(2 pi k_j x / N), k_j = j - B/2.
__global__ void k_table_kx(float *C, float *S, int N, int B) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * N) return;
    int j = idx / N, x = idx - j * N;
    double c, s;
    phase_cs(j - B / 2, x, N, &c, &s);
    C[idx] = (float)c;
    S[idx] = (float)s;
}

// W1[2j][x] = cos, W1[2j+1][x] = -sin: the real form of the complex axis-1 sum.
__global__ void k_table_w1(float *W1, int N, int B) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * N) return;
    int j = idx / N, x = idx - j * N;
    double c, s;
    phase_cs(j - B / 2, x, N, &c, &s);
    W1[(2 * j) * (long long)N + x] = (float)c;
    W1[(2 * j + 1) * (long long)N + x] = (float)(-s);
}

// A(k) = (alpha omega(k) + gamma)^(2s), omega = sum_d 2(1 - cos(2 pi k_d / N_d)).
__global__ void k_regulariser(float *A, int N1, int N2, int N3, int B1, int B2, int B3,
                              double alpha, double gamma, int s) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nb = (long long)B1 * B2 * B3;
    if (idx >= nb) return;
    int j3 = (int)(idx % B3);
    int j2 = (int)((idx / B3) % B2);
    int j1 = (int)(idx / ((long long)B2 * B3));
    double om = 2.0 * (1.0 - cospi(2.0 * (j1 - B1 / 2) / (double)N1)) +
                2.0 * (1.0 - cospi(2.0 * (j2 - B2 / 2) / (double)N2)) +
                2.0 * (1.0 - cospi(2.0 * (j3 - B3 / 2) / (double)N3));
    double base = alpha * om + gamma, a = 1.0;
    for (int t = 0; t < 2 * s; ++t) a *= base;
    A[idx] = (float)a;
}

// ---------------------------------------------------------------------------
// stage A: axis 3, band -> grid.  One thread per (row, x3); rows = 3*B1*B2.
constexpr int EA_ROWS = 8;
__global__ void __launch_bounds__(128)
k_expand_axis3(const float *__restrict__ vt, const float *__restrict__ T3c,
               const float *__restrict__ T3s, float *__restrict__ out,
               int rows, int B2, int B3, int N3) {
    extern __shared__ float sh[];   // EA_ROWS * B3 * 2
    int row0 = blockIdx.x * EA_ROWS;
    for (int i = threadIdx.x; i < EA_ROWS * B3 * 2; i += blockDim.x) {
        int r = row0 + i / (2 * B3);
        sh[i] = r < rows ? vt[(long long)row0 * B3 * 2 + i] : 0.f;
    }
    __syncthreads();
    int x3 = blockIdx.y * blockDim.x + threadIdx.x;
    if (x3 >= N3) return;
    for (int r = 0; r < EA_ROWS; ++r) {
        int row = row0 + r;
        if (row >= rows) break;
        float re = 0.f, im = 0.f;
        for (int k3 = 0; k3 < B3; ++k3) {
            float c = __ldg(T3c + (long long)k3 * N3 + x3);
            float s = __ldg(T3s + (long long)k3 * N3 + x3);
            float vr = sh[(r * B3 + k3) * 2], vi = sh[(r * B3 + k3) * 2 + 1];
            re = fmaf(vr, c, fmaf(-vi, s, re));
            im = fmaf(vr, s, fmaf(vi, c, im));
        }
        int slab = row / B2, k2 = row - slab * B2;
        out[((long long)(slab * 2 + 0) * B2 + k2) * N3 + x3] = re;
        out[((long long)(slab * 2 + 1) * B2 + k2) * N3 + x3] = im;
    }
}

// ---------------------------------------------------------------------------
// stage B (SIGN = +1, expand) and stage B' (SIGN = -1, project): per slab,
//   out[r][x3] = sum_s (T2c[?] + i SIGN T2s[?]) in[s][x3]
// expand : r = x2, s = k2, table index [k2][x2]; in rows = B2, out rows = N2
// project: r = k2, s = x2, table index [k2][x2]; in rows = N2, out rows = B2
template <int SIGN>
__global__ void __launch_bounds__(256)
k_axis2(const float *__restrict__ in, const float *__restrict__ T2c,
        const float *__restrict__ T2s, float *__restrict__ out,
        int in_rows, int out_rows, int N2, int N3) {
    __shared__ float sre[16][33], sim[16][33];
    __shared__ float sc[16][33], ss[16][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int x3 = blockIdx.x * 32 + tx;
    const int rb = blockIdx.y * 32;
    const long long slab = blockIdx.z;
    const float *inre = in + slab * 2 * (long long)in_rows * N3;
    const float *inim = inre + (long long)in_rows * N3;
    float are[4] = {0.f, 0.f, 0.f, 0.f}, aim[4] = {0.f, 0.f, 0.f, 0.f};
    for (int s0 = 0; s0 < in_rows; s0 += 16) {
        for (int i = threadIdx.x; i < 512; i += 256) {
            int ss_ = i >> 5, xx = i & 31;
            int sidx = s0 + ss_;
            int gx3 = blockIdx.x * 32 + xx;
            int gr = rb + xx;
            bool ok = sidx < in_rows;
            sre[ss_][xx] = (ok && gx3 < N3) ? inre[(long long)sidx * N3 + gx3] : 0.f;
            sim[ss_][xx] = (ok && gx3 < N3) ? inim[(long long)sidx * N3 + gx3] : 0.f;
            float c = 0.f, s = 0.f;
            if (ok && gr < out_rows) {
                // table [k2][x2]
                long long t = (SIGN > 0) ? (long long)sidx * N2 + gr : (long long)gr * N2 + sidx;
                c = T2c[t];
                s = T2s[t];
            }
            sc[ss_][xx] = c;
            ss[ss_][xx] = s;
        }
        __syncthreads();
#pragma unroll 4
        for (int q = 0; q < 16; ++q) {
            float vr = sre[q][tx], vi = sim[q][tx];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float c = sc[q][ty * 4 + r], s = ss[q][ty * 4 + r];
                if (SIGN > 0) {   // (c + i s)(vr + i vi)
                    are[r] = fmaf(c, vr, fmaf(-s, vi, are[r]));
                    aim[r] = fmaf(s, vr, fmaf(c, vi, aim[r]));
                } else {          // (c - i s)(vr + i vi)
                    are[r] = fmaf(c, vr, fmaf(s, vi, are[r]));
                    aim[r] = fmaf(c, vi, fmaf(-s, vr, aim[r]));
                }
            }
        }
        __syncthreads();
    }
    if (x3 >= N3) return;
    float *ore = out + slab * 2 * (long long)out_rows * N3;
    float *oim = ore + (long long)out_rows * N3;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int row = rb + ty * 4 + r;
        if (row < out_rows) {
            ore[(long long)row * N3 + x3] = are[r];
            oim[(long long)row * N3 + x3] = aim[r];
        }
    }
}

// ---------------------------------------------------------------------------
// stage C / C': C[M][Ncol] = sum_k A(m, k) B[k][Ncol], batched over components.
// A_TRANS: A(m, k) = A[k*lda + m] (expand, A = W1 [2B1][N1], m = x1, k = (k1,re/im))
// else   : A(m, k) = A[m*lda + k] (project, m = (k1,re/im), k = x1)
// MODE 0 stores scale*acc; MODE 1 stores the clamped displacement and latches
// the CFL / NaN flags.
template <bool A_TRANS, int MODE>
__global__ void __launch_bounds__(256)
k_gemm_axis1(const float *__restrict__ A, int lda, const float *__restrict__ B,
             long long strideB, float *__restrict__ C, long long strideC,
             int M, int K, long long Ncol, float scale, int *status) {
    __shared__ __align__(16) float As[16][64];
    __shared__ __align__(16) float Bs[16][128];
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int m0 = blockIdx.y * 64;
    const long long c0 = (long long)blockIdx.x * 128;
    B += blockIdx.z * strideB;
    C += blockIdx.z * strideC;
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[r][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = tid; i < 16 * 64; i += 256) {
            int kk = i >> 6, mm = i & 63;
            int gm = m0 + mm, gk = k0 + kk;
            float a = 0.f;
            if (gm < M && gk < K) a = A_TRANS ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            As[kk][mm] = a;
        }
        for (int i = tid; i < 16 * 128; i += 256) {
            int kk = i >> 7, cc = i & 127;
            int gk = k0 + kk;
            long long gc = c0 + cc;
            Bs[kk][cc] = (gk < K && gc < Ncol) ? B[(long long)gk * Ncol + gc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 8]);
            float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][ty * 8 + 4]);
            float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float b[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 32 * j];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[r][j] = fmaf(a[r], b[j], acc[r][j]);
        }
        __syncthreads();
    }
    int flags = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        int gm = m0 + ty * 8 + r;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            long long gc = c0 + tx + 32 * j;
            if (gc >= Ncol) continue;
            float v = acc[r][j] * scale;
            if (MODE == 1) {
                if (!(fabsf(v) < 1.f)) flags |= (v != v) ? BLR_FLAG_NAN : BLR_FLAG_CFL;
                v = fminf(fmaxf(v, -1.f), 0.99999994f);
            }
            C[(long long)gm * Ncol + gc] = v;
        }
    }
    if (MODE == 1 && flags) atomicOr(status, flags);
}

// ---------------------------------------------------------------------------
// stage A': axis 3, grid -> band.  Block: 8 rows (one per warp) x all k3;
// x3 in chunks of 32.
//   out[row][k3] = sum_x3 (c - i s)[k3][x3] P2[row][x3]  (+ A * vadd)
constexpr int PA_ROWS = 8;
__global__ void __launch_bounds__(256)
k_project_axis3(const float *__restrict__ in, const float *__restrict__ T3c,
                const float *__restrict__ T3s, float *__restrict__ out,
                const float *__restrict__ Aw, const float *__restrict__ vadd,
                int rows, int B2, int B3, int N3, int nb12) {
    __shared__ float pre[PA_ROWS][33], pim[PA_ROWS][33];
    __shared__ float tc[32][65], ts[32][65];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row0 = blockIdx.x * PA_ROWS;
    const int nk = (B3 + 31) / 32;     // k3 sub-blocks per lane (B3 <= 64)
    constexpr int RW = PA_ROWS / 8;    // rows per warp
    float are[RW][2], aim[RW][2];
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int t = 0; t < 2; ++t) are[r][t] = aim[r][t] = 0.f;
    for (int x0 = 0; x0 < N3; x0 += 32) {
        for (int i = tid; i < PA_ROWS * 32; i += 256) {
            int rr = i >> 5, xx = i & 31;
            int row = row0 + rr, gx = x0 + xx;
            float a = 0.f, b = 0.f;
            if (row < rows && gx < N3) {
                int slab = row / B2, k2 = row - slab * B2;
                a = in[((long long)(slab * 2 + 0) * B2 + k2) * N3 + gx];
                b = in[((long long)(slab * 2 + 1) * B2 + k2) * N3 + gx];
            }
            pre[rr][xx] = a;
            pim[rr][xx] = b;
        }
        for (int i = tid; i < 32 * 64; i += 256) {
            int xx = i & 31, kk = i >> 5;
            int gx = x0 + xx;
            float c = 0.f, s = 0.f;
            if (kk < B3 && gx < N3) {
                c = T3c[(long long)kk * N3 + gx];
                s = T3s[(long long)kk * N3 + gx];
            }
            tc[xx][kk] = c;
            ts[xx][kk] = s;
        }
        __syncthreads();
        for (int xx = 0; xx < 32; ++xx) {
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                if (t >= nk) break;
                float c = tc[xx][lane + 32 * t], s = ts[xx][lane + 32 * t];
#pragma unroll
                for (int r = 0; r < RW; ++r) {
                    float pr = pre[warp * RW + r][xx], pi = pim[warp * RW + r][xx];
                    are[r][t] = fmaf(c, pr, fmaf(s, pi, are[r][t]));
                    aim[r][t] = fmaf(c, pi, fmaf(-s, pr, aim[r][t]));
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        int row = row0 + warp * RW + r;
        if (row >= rows) continue;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            int k3 = lane + 32 * t;
            if (t >= nk || k3 >= B3) continue;
            long long o = ((long long)row * B3 + k3) * 2;
            float re = are[r][t], im = aim[r][t];
            if (vadd) {
                float a = Aw[(long long)(row % nb12) * B3 + k3];
                re = fmaf(a, vadd[o], re);
                im = fmaf(a, vadd[o + 1], im);
            }
            out[o] = re;
            out[o + 1] = im;
        }
    }
}

}  // namespace

int dft_init_tables(blr_plan *P, cudaStream_t s) {
    const int T = 256;
    k_table_w1<<<(int)ceil_div_ll((long long)P->B1 * P->N1, T), T, 0, s>>>(P->W1, P->N1, P->B1);
    BLR_CK_LAUNCH();
    k_table_kx<<<(int)ceil_div_ll((long long)P->B2 * P->N2, T), T, 0, s>>>(P->T2c, P->T2s, P->N2, P->B2);
    BLR_CK_LAUNCH();
    k_table_kx<<<(int)ceil_div_ll((long long)P->B3 * P->N3, T), T, 0, s>>>(P->T3c, P->T3s, P->N3, P->B3);
    BLR_CK_LAUNCH();
    k_regulariser<<<(int)ceil_div_ll(P->nb, T), T, 0, s>>>(
        P->A, P->N1, P->N2, P->N3, P->B1, P->B2, P->B3, P->p.alpha, P->p.gamma, P->p.s);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int dft_expand(blr_plan *P, const float *vt, float *out, int mode, cudaStream_t s) {
    const int rows = 3 * P->B1 * P->B2;
    // stage A
    dim3 ga((unsigned)ceil_div_ll(rows, EA_ROWS), (unsigned)ceil_div_ll(P->N3, 128));
    k_expand_axis3<<<ga, 128, EA_ROWS * P->B3 * 2 * sizeof(float), s>>>(
        vt, P->T3c, P->T3s, P->dft_small, rows, P->B2, P->B3, P->N3);
    BLR_CK_LAUNCH();
    // stage B
    if (P->tc_tab2_expand) {
        int rc = tc_axis2(P, 0, P->dft_small, P->dft_big, s);
        if (rc) return rc;
    } else {
        dim3 gb((unsigned)ceil_div_ll(P->N3, 32), (unsigned)ceil_div_ll(P->N2, 32), 3u * P->B1);
        k_axis2<+1><<<gb, 256, 0, s>>>(P->dft_small, P->T2c, P->T2s, P->dft_big, P->B2, P->N2,
                                       P->N2, P->N3);
        BLR_CK_LAUNCH();
    }
    // stage C
    if (P->p.precision == BLR_MIXED) {
        int rc = tc_axis1(P, 0, P->dft_big, out, mode == 0 ? 1.f : -P->dt, mode, s);
        if (rc || mode == 0 || out != P->d) return rc;
        return sweep_pack_d4(P, s);
    }
    const long long ncol = (long long)P->N2 * P->N3;
    dim3 gc((unsigned)ceil_div_ll(ncol, 128), (unsigned)ceil_div_ll(P->N1, 64), 3u);
    if (mode == 0)
        k_gemm_axis1<true, 0><<<gc, 256, 0, s>>>(P->W1, P->N1, P->dft_big, 2LL * P->B1 * ncol,
                                                 out, P->V, P->N1, 2 * P->B1, ncol, 1.f,
                                                 P->dstatus);
    else
        k_gemm_axis1<true, 1><<<gc, 256, 0, s>>>(P->W1, P->N1, P->dft_big, 2LL * P->B1 * ncol,
                                                 out, P->V, P->N1, 2 * P->B1, ncol, -P->dt,
                                                 P->dstatus);
    BLR_CK_LAUNCH();
    if (mode == 1 && out == P->d) return sweep_pack_d4(P, s);
    return BLR_OK;
}

int dft_project(blr_plan *P, const float *f, float *ft, const float *vadd, cudaStream_t s) {
    const long long ncol = (long long)P->N2 * P->N3;
    // stage C'
    if (P->p.precision == BLR_MIXED) {
        int rc = tc_axis1(P, 1, f, P->dft_big, 1.f, 0, s);
        if (rc) return rc;
    } else {
        dim3 gc((unsigned)ceil_div_ll(ncol, 128), (unsigned)ceil_div_ll(2 * P->B1, 64), 3u);
        k_gemm_axis1<false, 0><<<gc, 256, 0, s>>>(P->W1, P->N1, f, P->V, P->dft_big,
                                                  2LL * P->B1 * ncol, 2 * P->B1, P->N1, ncol,
                                                  1.f, P->dstatus);
        BLR_CK_LAUNCH();
    }
    // stage B'
    if (P->tc_tab2_project) {
        int rc = tc_axis2(P, 1, P->dft_big, P->dft_small, s);
        if (rc) return rc;
    } else {
        dim3 gb((unsigned)ceil_div_ll(P->N3, 32), (unsigned)ceil_div_ll(P->B2, 32), 3u * P->B1);
        k_axis2<-1><<<gb, 256, 0, s>>>(P->dft_big, P->T2c, P->T2s, P->dft_small, P->N2, P->B2,
                                       P->N2, P->N3);
        BLR_CK_LAUNCH();
    }
    // stage A'
    const int rows = 3 * P->B1 * P->B2;
    k_project_axis3<<<(unsigned)ceil_div_ll(rows, PA_ROWS), 256, 0, s>>>(
        P->dft_small, P->T3c, P->T3s, ft, P->A, vadd, rows, P->B2, P->B3, P->N3, P->B1 * P->B2);
    BLR_CK_LAUNCH();
    return BLR_OK;
}
