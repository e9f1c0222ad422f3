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

// A(k) = (alpha omega(k) + gamma)^q, q = 2s, omega = sum_d 2(1 - cos(2 pi k_d / N_d)).
__global__ void k_regulariser(float *A, int N1, int N2, int N3, int B1, int B2, int B3,
                              double alpha, double gamma, int q) {
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
    for (int t = 0; t < q; ++t) a *= base;
    A[idx] = (float)a;
}

// ---------------------------------------------------------------------------
// stage A: axis 3, band -> grid.  A block owns XR rows (c, k1, k2) and XC x3
// columns; the rows' coefficients and the E3 table for those columns are staged
// in shared memory and each thread accumulates a 2 (rows) x 4 (x3, 32 apart)
// register tile over k3 in order.
constexpr int XR = 16, XC = 128;
__global__ void __launch_bounds__(256)
k_expand_axis3(const float *__restrict__ vt, const float *__restrict__ T3c,
               const float *__restrict__ T3s, float *__restrict__ out,
               int rows, int B2, int B3, int N3) {
    extern __shared__ float2 sh2[];
    float2 *sc = sh2;                // [XR][B3] coefficients
    float2 *st = sh2 + XR * B3;      // [B3][XC] (cos, sin)
    const int r0 = blockIdx.x * XR, x0 = blockIdx.y * XC;
    pdl_wait();   // the tables may come from the previous kernel (allocation-free expand)
    for (int i = threadIdx.x; i < B3 * XC; i += 256) {
        const int k3 = i / XC, x = x0 + (i - k3 * XC);
        st[i] = x < N3 ? make_float2(__ldg(T3c + (long long)k3 * N3 + x), __ldg(T3s + (long long)k3 * N3 + x))
                       : make_float2(0.f, 0.f);
    }
    for (int i = threadIdx.x; i < XR * B3; i += 256) {
        const int rr = i / B3, k3 = i - rr * B3, row = r0 + rr;
        const long long o = ((long long)row * B3 + k3) * 2;
        sc[i] = row < rows ? make_float2(vt[o], vt[o + 1]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float are[2][4], aim[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) are[r][q] = aim[r][q] = 0.f;
    for (int k3 = 0; k3 < B3; ++k3) {
        const float2 v[2] = {sc[(2 * w) * B3 + k3], sc[(2 * w + 1) * B3 + k3]};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 e = st[k3 * XC + lane + 32 * q];
#pragma unroll
            for (int r = 0; r < 2; ++r) {   // (vr + i vi)(c + i s)
                are[r][q] = fmaf(v[r].x, e.x, fmaf(-v[r].y, e.y, are[r][q]));
                aim[r][q] = fmaf(v[r].x, e.y, fmaf(v[r].y, e.x, aim[r][q]));
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int row = r0 + 2 * w + r;
        if (row >= rows) continue;
        const int slab = row / B2, k2 = row - slab * B2;
        float *ore = out + ((long long)(slab * 2 + 0) * B2 + k2) * N3;
        float *oim = out + ((long long)(slab * 2 + 1) * B2 + k2) * N3;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int x = x0 + lane + 32 * q;
            if (x < N3) {
                ore[x] = are[r][q];
                oim[x] = aim[r][q];
            }
        }
    }
}

size_t expand_axis3_smem(int B3) { return (size_t)(XR * B3 + B3 * XC) * sizeof(float2); }

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
    pdl_wait();
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
    pdl_wait();
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
// stage A': axis 3, grid -> band (+ A * vadd).  A block owns XR rows and every
// k3; x3 runs in chunks of XC staged in shared memory together with the
// conjugate table, transposed to [x3][k3] so that the lanes (one k3 each, two
// when B3 > 32) read consecutive words.  Each thread accumulates 2 rows over x3
// in order.
constexpr int PXC = 128;
__global__ void __launch_bounds__(256)
k_project_axis3(const float *__restrict__ in, const float *__restrict__ T3c,
                const float *__restrict__ T3s, float *__restrict__ out,
                const float *__restrict__ Aw, const float *__restrict__ vadd, float areg,
                int rows, int B2, int B3, int N3, int nb12) {
    extern __shared__ float2 sh2[];
    const int B3p = B3 + 1;
    float2 *sp = sh2;                // [XR][PXC] (re, im) of the rows
    float2 *st = sh2 + XR * PXC;     // [PXC][B3p] (cos, sin)
    const int r0 = blockIdx.x * XR;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nk = (B3 + 31) / 32;   // k3 per lane (B3 <= 64)
    pdl_wait();
    float are[2][2], aim[2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int t = 0; t < 2; ++t) are[r][t] = aim[r][t] = 0.f;
    for (int x0 = 0; x0 < N3; x0 += PXC) {
        __syncthreads();
        for (int i = threadIdx.x; i < XR * PXC; i += 256) {
            const int rr = i / PXC, x = x0 + (i - rr * PXC), row = r0 + rr;
            float a = 0.f, b = 0.f;
            if (row < rows && x < N3) {
                const int slab = row / B2, k2 = row - slab * B2;
                a = in[((long long)(slab * 2 + 0) * B2 + k2) * N3 + x];
                b = in[((long long)(slab * 2 + 1) * B2 + k2) * N3 + x];
            }
            sp[i] = make_float2(a, b);
        }
        for (int i = threadIdx.x; i < B3 * PXC; i += 256) {
            const int k3 = i / PXC, xx = i - k3 * PXC, x = x0 + xx;
            st[xx * B3p + k3] = x < N3 ? make_float2(__ldg(T3c + (long long)k3 * N3 + x),
                                                     __ldg(T3s + (long long)k3 * N3 + x))
                                       : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int xn = min(PXC, N3 - x0);
        for (int xx = 0; xx < xn; ++xx) {
            const float2 p[2] = {sp[(2 * w) * PXC + xx], sp[(2 * w + 1) * PXC + xx]};
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                if (t >= nk) break;
                // lanes past the last k3 read a valid entry; their sums are not stored
                const float2 e = st[xx * B3p + min(lane + 32 * t, B3 - 1)];
#pragma unroll
                for (int r = 0; r < 2; ++r) {   // (c - i s)(pr + i pi)
                    are[r][t] = fmaf(e.x, p[r].x, fmaf(e.y, p[r].y, are[r][t]));
                    aim[r][t] = fmaf(e.x, p[r].y, fmaf(-e.y, p[r].x, aim[r][t]));
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int row = r0 + 2 * w + r;
        if (row >= rows) continue;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int k3 = lane + 32 * t;
            if (t >= nk || k3 >= B3) continue;
            const long long o = ((long long)row * B3 + k3) * 2;
            float re = are[r][t], im = aim[r][t];
            if (vadd) {
                const float a = areg * Aw[(long long)(row % nb12) * B3 + k3];
                re = fmaf(a, vadd[o], re);
                im = fmaf(a, vadd[o + 1], im);
            }
            out[o] = re;
            out[o + 1] = im;
        }
    }
}

size_t project_axis3_smem(int B3) { return (size_t)(XR * PXC + PXC * (B3 + 1)) * sizeof(float2); }

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
        P->A, P->N1, P->N2, P->N3, P->B1, P->B2, P->B3, P->p.alpha, P->p.gamma,
        (int)(2.0 * P->p.s + 0.5));
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int dft_expand(blr_plan *P, const float *vt, float *out, int mode, cudaStream_t s) {
    if (P->fz_tab[0]) {   // mixed precision, fused tensor-core transform
        int rc = fz_expand(P, vt, out, mode == 0 ? 1.f : -P->dt, mode, s);
        if (rc || mode == 0 || out != P->d) return rc;
        return sweep_pack_d4(P, s);
    }
    const int rows = 3 * P->B1 * P->B2;
    // stage A
    dim3 ga((unsigned)ceil_div_ll(rows, XR), (unsigned)ceil_div_ll(P->N3, XC));
    const size_t sa = expand_axis3_smem(P->B3);
    BLR_CK(cudaFuncSetAttribute(k_expand_axis3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa));
    launch_pdl(k_expand_axis3, ga, dim3(256), sa, s, vt, (const float *)P->T3c,
               (const float *)P->T3s, P->dft_small, rows, P->B2, P->B3, P->N3);
    BLR_CK_LAUNCH();
    // stage B
    if (P->tc_tab2_expand) {
        int rc = tc_axis2(P, 0, P->dft_small, P->dft_big, s);
        if (rc) return rc;
    } else {
        dim3 gb((unsigned)ceil_div_ll(P->N3, 32), (unsigned)ceil_div_ll(P->N2, 32), 3u * P->B1);
        launch_pdl(k_axis2<+1>, gb, dim3(256), 0, s, (const float *)P->dft_small,
                   (const float *)P->T2c, (const float *)P->T2s, P->dft_big, P->B2, P->N2, P->N2,
                   P->N3);
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
        launch_pdl(k_gemm_axis1<true, 0>, gc, dim3(256), 0, s, (const float *)P->W1, P->N1,
                   (const float *)P->dft_big, 2LL * P->B1 * ncol, out, P->V, P->N1, 2 * P->B1, ncol,
                   1.f, P->dstatus);
    else
        launch_pdl(k_gemm_axis1<true, 1>, gc, dim3(256), 0, s, (const float *)P->W1, P->N1,
                   (const float *)P->dft_big, 2LL * P->B1 * ncol, out, P->V, P->N1, 2 * P->B1, ncol,
                   -P->dt, P->dstatus);
    BLR_CK_LAUNCH();
    if (mode == 1 && out == P->d) return sweep_pack_d4(P, s);
    return BLR_OK;
}

int dft_project(blr_plan *P, const float *f, float *ft, const float *vadd, cudaStream_t s,
                float areg) {
    if (P->fz_tab[0]) return fz_project(P, f, ft, vadd, areg, s);
    const long long ncol = (long long)P->N2 * P->N3;
    // stage C'
    if (P->p.precision == BLR_MIXED) {
        int rc = tc_axis1(P, 1, f, P->dft_big, 1.f, 0, s);
        if (rc) return rc;
    } else {
        dim3 gc((unsigned)ceil_div_ll(ncol, 128), (unsigned)ceil_div_ll(2 * P->B1, 64), 3u);
        launch_pdl(k_gemm_axis1<false, 0>, gc, dim3(256), 0, s, (const float *)P->W1, P->N1, f,
                   P->V, P->dft_big, 2LL * P->B1 * ncol, 2 * P->B1, P->N1, ncol, 1.f, P->dstatus);
        BLR_CK_LAUNCH();
    }
    // stage B'
    if (P->tc_tab2_project) {
        int rc = tc_axis2(P, 1, P->dft_big, P->dft_small, s);
        if (rc) return rc;
    } else {
        dim3 gb((unsigned)ceil_div_ll(P->N3, 32), (unsigned)ceil_div_ll(P->B2, 32), 3u * P->B1);
        launch_pdl(k_axis2<-1>, gb, dim3(256), 0, s, (const float *)P->dft_big,
                   (const float *)P->T2c, (const float *)P->T2s, P->dft_small, P->N2, P->B2, P->N2,
                   P->N3);
        BLR_CK_LAUNCH();
    }
    // stage A'
    const int rows = 3 * P->B1 * P->B2;
    const size_t sp = project_axis3_smem(P->B3);
    BLR_CK(cudaFuncSetAttribute(k_project_axis3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp));
    launch_pdl(k_project_axis3, dim3((unsigned)ceil_div_ll(rows, XR)), dim3(256), sp, s,
               (const float *)P->dft_small, (const float *)P->T3c, (const float *)P->T3s, ft,
               (const float *)P->A, vadd, areg, rows, P->B2, P->B3, P->N3, P->B1 * P->B2);
    BLR_CK_LAUNCH();
    return BLR_OK;
}
