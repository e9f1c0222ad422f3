// Truncated DFTs of the band-limited space (Section 3.1, Eq. 33), FP32 path.
//
// iota(v~)_c(x) = Re sum_k v~_c(k) e^{2 pi i k.x/N} is evaluated as three
// axis-wise contractions against small DFT tables:
//   stage A (axis 3): A1[c,k1,k2,x3] = sum_k3 v~[c,k1,k2,k3] E3[k3,x3]          complex
//   stage B (axis 2): A2[c,k1,x2,x3] = sum_k2 E2[k2,x2] A1[c,k1,k2,x3]          complex
//   stage C (axis 1): v[c,x1,x2,x3]  = sum_{k1,re/im} W1[(k1,re/im), x1] A2[...] real GEMM
// pi = iota^T runs the transposed stages in reverse order (C', B', A').
// Intermediates are planar: [slab = c*B1 + k1][re|im][row][x3].
#include <algorithm>

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

// W1[2j][x] = cos, W1[2j+1][x] = -sin: the real form of the complex axis-1 sum
// (and, when W1t is given, its transpose W1t[x][2j + (0|1)]).
__global__ void k_table_w1(float *W1, float *W1t, int N, int B) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * N) return;
    int j = idx / N, x = idx - j * N;
    double c, s;
    phase_cs(j - B / 2, x, N, &c, &s);
    W1[(2 * j) * (long long)N + x] = (float)c;
    W1[(2 * j + 1) * (long long)N + x] = (float)(-s);
    if (W1t) {
        W1t[(long long)x * 2 * B + 2 * j] = (float)c;
        W1t[(long long)x * 2 * B + 2 * j + 1] = (float)(-s);
    }
}

// The axis-2 stages' A operands in [k][m] order (see k_sgemm): expand
// T2e[(ki, k2)][(mi, x2)] and project T2p[(ki, x2)][(mi, k2)], each entry C, S or
// -S of the phase (k2 - B/2) x2.
__global__ void k_table_axis2(float *T2e, float *T2p, int N, int B) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * N) return;
    const int j = idx / N, x = idx - j * N;
    double c, s;
    phase_cs(j - B / 2, x, N, &c, &s);
    const float C = (float)c, S = (float)s;
    const long long M2e = 2LL * N, M2p = 2LL * B;
    // expand: out (mi, x2) from in (ki, k2): [[C, -S], [S, C]]
    T2e[(long long)j * M2e + x] = C;                 // ki 0, mi 0
    T2e[(long long)j * M2e + N + x] = S;             // ki 0, mi 1
    T2e[(long long)(B + j) * M2e + x] = -S;          // ki 1, mi 0
    T2e[(long long)(B + j) * M2e + N + x] = C;       // ki 1, mi 1
    // project: out (mi, k2) from in (ki, x2): [[C, S], [-S, C]]
    T2p[(long long)x * M2p + j] = C;                 // ki 0, mi 0
    T2p[(long long)x * M2p + B + j] = -S;            // ki 0, mi 1
    T2p[(long long)(N + x) * M2p + j] = S;           // ki 1, mi 0
    T2p[(long long)(N + x) * M2p + B + j] = C;       // ki 1, mi 1
}

// The expand axis-3 stage's B operand T3e[(k3, ri')][(ri, x3)], entries C, S or
// -S of the phase (k3 - B/2) x3.
__global__ void k_table_axis3(float *T3e, int N, int B) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * N) return;
    const int j = idx / N, x = idx - j * N;
    double c, s;
    phase_cs(j - B / 2, x, N, &c, &s);
    const float C = (float)c, S = (float)s;
    const long long ne = 2LL * N;
    // expand: (vr + i vi)(C + i S): re = vr C - vi S, im = vr S + vi C
    T3e[(2LL * j) * ne + x] = C;
    T3e[(2LL * j) * ne + N + x] = S;
    T3e[(2LL * j + 1) * ne + x] = -S;
    T3e[(2LL * j + 1) * ne + N + x] = C;
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
// Stages A, B, B', C and C' are real GEMMs batched over z,
//   C_z[m][n] = scale * sum_k A(m, k) B_z[k][n],   B_z = B + z strideB ([K][N]),
// run by one FP32 kernel; the A operand and the output mapping differ:
//   AK_KM  A(m, k) = A[k lda + m]    stage C  (A = W1 [2B1][N1]: m = x1, k = (k1, re|im))
//   AK_MK  A(m, k) = A[m lda + k]    stage C' (A = W1: m = (k1, re|im), k = x1)
//   AK_E2  stage B  on a planar slab [re|im][k2][x3] -> [re|im][x2][x3]:
//          m = (re|im, x2), k = (re|im, k2), A = [[C, -S], [S, C]]  (C + i S)(re + i im)
//   AK_P2  stage B' on a planar slab [re|im][x2][x3] -> [re|im][k2][x3]:
//          m = (re|im, k2), k = (re|im, x2), A = [[C, S], [-S, C]]  (C - i S)(re + i im)
// with C = T2c[k2][x2], S = T2s[k2][x2].  Stage A takes AK_MK (A = v~ as
// [(c, k1, k2)][(k3, re|im)], B = T3e [(k3, re|im)][(re|im, x3)]) and writes
// its rows to the planar layout (EPI 1).  Row-major A operands (AK_MK) are
// fetched k-fastest, the others m-fastest, so that every fetch is coalesced.  NT
// threads (256 or 128) as TR = NT / 16 rows x 16 columns, each thread a TM x TN
// register tile (rows tm*4 + i + 4 TR h, columns tn*4 + j + 64 h'): tiles of
// (TR TM) x (16 TN) outputs; k in chunks of 16 through two shared-memory buffers,
// the next chunk's loads in flight (registers) during this chunk's products.  The
// sum over k runs in order, the same for every tile shape: all shapes give the
// same results bit for bit.  MODE 1 stores the clamped displacement and latches
// the CFL / NaN flags.
enum { AK_KM = 0, AK_MK = 1, AK_E2 = 2, AK_P2 = 3 };

struct GemmArgs {
    const float *A;
    int lda;
    const float *Tc, *Ts;   // AK_E2 / AK_P2
    int N2, B2;
    const float *B;
    long long strideB;
    float *C;
    long long strideC;
    int M, K;
    long long N;
    float scale;
    int *status;
    int pN3, pB2;             // planar rows (EPI 1): x3 extent, k2 rows per slab
};

template <int AK>
__device__ __forceinline__ float a_elem(const GemmArgs &p, int m, int k) {
    if (m >= p.M || k >= p.K) return 0.f;
    if (AK == AK_KM) return __ldg(p.A + (long long)k * p.lda + m);
    if (AK == AK_MK) return __ldg(p.A + (long long)m * p.lda + k);
    if (AK == AK_E2) {
        const int mi = m >= p.N2, ki = k >= p.B2;
        const long long t = (long long)(k - ki * p.B2) * p.N2 + (m - mi * p.N2);
        return mi == ki ? __ldg(p.Tc + t) : (mi ? __ldg(p.Ts + t) : -__ldg(p.Ts + t));
    }
    const int mi = m >= p.B2, ki = k >= p.N2;
    const long long t = (long long)(m - mi * p.B2) * p.N2 + (k - ki * p.N2);
    return mi == ki ? __ldg(p.Tc + t) : (mi ? -__ldg(p.Ts + t) : __ldg(p.Ts + t));
}

constexpr int GK = 16;   // k per chunk

template <int AK, int MODE, int TM, int TN, int EPI = 0, int NT = 256>
__global__ void __launch_bounds__(NT, 512 / NT)
k_sgemm(GemmArgs p) {
    constexpr int TR = NT / 16;                                // thread rows
    constexpr int BM = TR * TM, BN = 16 * TN, AP = BM + 4;   // padded A rows
    constexpr int NB4 = GK * BN / 4 / NT;                      // B float4 per thread and chunk
    static_assert(NT == 256 || NT == 128, "16 x 16 or 8 x 16 threads");
    static_assert(NB4 * NT * 4 == GK * BN, "B chunk split over the threads");
    constexpr bool KFAST = AK == AK_MK;
    __shared__ __align__(16) float As[2][GK][AP];
    __shared__ __align__(16) float Bs[2][GK][BN];
    const int tid = threadIdx.x, tn = tid & 15, tm = tid >> 4;
    const int m0 = blockIdx.y * BM;
    const long long n0 = (long long)blockIdx.x * BN;
    const float *Bz = p.B + blockIdx.z * p.strideB;
    const bool vec = (p.N & 3) == 0;
    float ra[TM];
    float4 rb[NB4];
    auto load = [&](int k0) {
#pragma unroll
        for (int i = 0; i < TM; ++i) {   // BM x GK = NT TM elements
            const int e = tid + NT * i;
            const int mm = KFAST ? e / GK : e % BM, kk = KFAST ? e % GK : e / BM;
            ra[i] = a_elem<AK>(p, m0 + mm, k0 + kk);
        }
#pragma unroll
        for (int i = 0; i < NB4; ++i) {
            const int e = tid + NT * i, kk = e / (BN / 4), k = k0 + kk;
            const long long n = n0 + 4 * (e % (BN / 4));
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < p.K) {
                const float *src = Bz + (long long)k * p.N + n;
                if (vec && n + 3 < p.N) {
                    v = __ldg(reinterpret_cast<const float4 *>(src));
                } else {
                    if (n < p.N) v.x = __ldg(src);
                    if (n + 1 < p.N) v.y = __ldg(src + 1);
                    if (n + 2 < p.N) v.z = __ldg(src + 2);
                    if (n + 3 < p.N) v.w = __ldg(src + 3);
                }
            }
            rb[i] = v;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int e = tid + NT * i;
            const int mm = KFAST ? e / GK : e % BM, kk = KFAST ? e % GK : e / BM;
            As[buf][kk][mm] = ra[i];
        }
#pragma unroll
        for (int i = 0; i < NB4; ++i) {
            const int e = tid + NT * i;
            *reinterpret_cast<float4 *>(&Bs[buf][e / (BN / 4)][4 * (e % (BN / 4))]) = rb[i];
        }
    };
    float acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = 0.f;
    pdl_wait();
    load(0);
    store(0);
    __syncthreads();
    for (int k0 = 0, cur = 0; k0 < p.K; k0 += GK, cur ^= 1) {
        const bool more = k0 + GK < p.K;
        if (more) load(k0 + GK);
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[TM], b[TN];
#pragma unroll
            for (int h = 0; h < TM / 4; ++h) {
                const float4 v = *reinterpret_cast<const float4 *>(&As[cur][kk][4 * TR * h + tm * 4]);
                a[4 * h] = v.x;
                a[4 * h + 1] = v.y;
                a[4 * h + 2] = v.z;
                a[4 * h + 3] = v.w;
            }
#pragma unroll
            for (int h = 0; h < TN / 4; ++h) {
                const float4 v = *reinterpret_cast<const float4 *>(&Bs[cur][kk][64 * h + tn * 4]);
                b[4 * h] = v.x;
                b[4 * h + 1] = v.y;
                b[4 * h + 2] = v.z;
                b[4 * h + 3] = v.w;
            }
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        if (more) store(cur ^ 1);
        __syncthreads();
    }
    float *Cz = p.C + blockIdx.z * p.strideC;
    int flags = 0;
#pragma unroll
    for (int r = 0; r < TM; ++r) {
        const int m = m0 + 4 * TR * (r / 4) + tm * 4 + (r & 3);
        if (m >= p.M) continue;
#pragma unroll
        for (int h = 0; h < TN / 4; ++h) {
            const long long n = n0 + 64 * h + tn * 4;
            float v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float x = acc[r][4 * h + j] * p.scale;
                if (MODE == 1) {
                    if (n + j < p.N && !(fabsf(x) < 1.f)) flags |= (x != x) ? BLR_FLAG_NAN : BLR_FLAG_CFL;
                    x = fminf(fmaxf(x, -1.f), 0.99999994f);
                }
                v[j] = x;
            }
            float *dst;
            bool vst = vec && n + 3 < p.N;
            if (EPI == 1) {   // row m = (slab, k2), column n = (re|im, x3) of the planar layout
                const int slab = m / p.pB2, k2 = m - slab * p.pB2;
                const int ri = n >= p.pN3;
                dst = Cz + ((long long)(slab * 2 + ri) * p.pB2 + k2) * p.pN3 + (n - ri * p.pN3);
                vst = vst && (p.pN3 & 3) == 0;
                if (!vst) {   // the four columns may straddle the re | im halves
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const long long nj = n + j;
                        if (nj >= p.N) continue;
                        const int rj = nj >= p.pN3;
                        Cz[((long long)(slab * 2 + rj) * p.pB2 + k2) * p.pN3 + (nj - rj * p.pN3)] = v[j];
                    }
                    continue;
                }
            } else {
                dst = Cz + (long long)m * p.N + n;
            }
            if (vst) {
                *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (n + j < p.N) dst[j] = v[j];
            }
        }
    }
    if (MODE == 1 && flags) atomicOr(p.status, flags);
}

// Launch k_sgemm with the register tile and thread count of candidate `forced`
// (1 .. SG_CANDS, chosen per plan by timing), else the modelled choice among the
// 256-thread tiles: the largest that still gives every SM two blocks (or the
// smallest when even that does not).  The 128-thread tiles (32 rows) serve the
// stages whose 64-row tiles leave most SMs idle.

template <int AK, int MODE, int EPI = 0>
int launch_sgemm(const GemmArgs &p, int batch, int sms, cudaStream_t s, int forced = 0) {
    // candidates: {TM, TN, threads}
    const int tms[SG_CANDS] = {8, 8, 4, 4, 4, 4}, tns[SG_CANDS] = {8, 4, 8, 4, 4, 8};
    const int nts[SG_CANDS] = {256, 256, 256, 256, 128, 128};
    // modelled time: waves of resident blocks x a block's padded tile over the
    // register tile's relative FMA rate (smem operand traffic per FMA)
    const int res[4] = {2, 2, 2, 3};
    const double rate[4] = {1.0, 0.75, 0.75, 0.55};
    int pick = 0;
    double best = 1e300;
    for (int c = 0; c < 4; ++c) {
        const long long bm = 16LL * tms[c], bn = 16LL * tns[c];
        const long long blocks = ceil_div_ll(p.N, bn) * ceil_div_ll(p.M, bm) * batch;
        const long long waves = ceil_div_ll(blocks, (long long)res[c] * sms);
        const long long share = std::min<long long>(res[c], ceil_div_ll(blocks, sms));
        const double t = (double)waves * (double)(bm * bn) * share / rate[c];
        if (t < best * 0.999) {
            best = t;
            pick = c;
        }
    }
    if (forced >= 1 && forced <= SG_CANDS) pick = forced - 1;
    const int TMc = tms[pick], TNc = tns[pick], NTc = nts[pick];
    const dim3 grid((unsigned)ceil_div_ll(p.N, 16LL * TNc), (unsigned)ceil_div_ll(p.M, (NTc / 16LL) * TMc),
                    (unsigned)batch);
    switch (pick) {
        case 0: launch_pdl(k_sgemm<AK, MODE, 8, 8, EPI>, grid, dim3(256), 0, s, p); break;
        case 1: launch_pdl(k_sgemm<AK, MODE, 8, 4, EPI>, grid, dim3(256), 0, s, p); break;
        case 2: launch_pdl(k_sgemm<AK, MODE, 4, 8, EPI>, grid, dim3(256), 0, s, p); break;
        case 3: launch_pdl(k_sgemm<AK, MODE, 4, 4, EPI>, grid, dim3(256), 0, s, p); break;
        case 4: launch_pdl(k_sgemm<AK, MODE, 4, 4, EPI, 128>, grid, dim3(128), 0, s, p); break;
        default: launch_pdl(k_sgemm<AK, MODE, 4, 8, EPI, 128>, grid, dim3(128), 0, s, p); break;
    }
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int device_sms(const blr_plan *P) {
    if (P->sms > 0) return P->sms;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 148;
    return sms;
}

// The GEMM stages of the FP32 transforms: 0 B (expand, axis 2), 1 C (expand,
// axis 1), 2 C' (project, axis 1), 3 B' (project, axis 2), 4 A (expand, axis 3).
// `in` / `out` are the stage's data operand and result; mode 1 (stage C only)
// stores the displacement.
int launch_stage(const blr_plan *P, int stage, const float *in, float *out, float scale, int mode,
                 cudaStream_t s, int nc = 3) {
    const long long ncol = (long long)P->N2 * P->N3;
    const int sms = device_sms(P), forced = P->gemm_tile[stage];
    GemmArgs g{};
    g.Tc = P->T2c;
    g.Ts = P->T2s;
    g.N2 = P->N2;
    g.B2 = P->B2;
    g.B = in;
    g.C = out;
    g.scale = scale;
    g.status = P->dstatus;
    switch (stage) {
        case 0:
            g.A = P->T2e;
            g.lda = 2 * P->N2;
            g.strideB = 2LL * P->B2 * P->N3;
            g.strideC = 2LL * P->N2 * P->N3;
            g.M = 2 * P->N2;
            g.K = 2 * P->B2;
            g.N = P->N3;
            return P->T2e ? launch_sgemm<AK_KM, 0>(g, nc * P->B1, sms, s, forced)
                          : launch_sgemm<AK_E2, 0>(g, nc * P->B1, sms, s, forced);
        case 1:
            g.A = P->W1;
            g.lda = P->N1;
            g.strideB = 2LL * P->B1 * ncol;
            g.strideC = P->V;
            g.M = P->N1;
            g.K = 2 * P->B1;
            g.N = ncol;
            return mode == 0 ? launch_sgemm<AK_KM, 0>(g, nc, sms, s, forced)
                             : launch_sgemm<AK_KM, 1>(g, nc, sms, s, forced);
        case 2:
            g.A = P->W1t ? P->W1t : P->W1;
            g.lda = P->W1t ? 2 * P->B1 : P->N1;
            g.strideB = P->V;
            g.strideC = 2LL * P->B1 * ncol;
            g.M = 2 * P->B1;
            g.K = P->N1;
            g.N = ncol;
            return P->W1t ? launch_sgemm<AK_KM, 0>(g, nc, sms, s, forced)
                          : launch_sgemm<AK_MK, 0>(g, nc, sms, s, forced);
        case 4:
            g.A = in;
            g.lda = 2 * P->B3;
            g.B = P->T3e;
            g.strideB = 0;
            g.pN3 = P->N3;
            g.pB2 = P->B2;
            g.M = nc * P->B1 * P->B2;
            g.K = 2 * P->B3;
            g.N = 2LL * P->N3;
            return launch_sgemm<AK_MK, 0, 1>(g, 1, sms, s, forced);
        default:
            g.A = P->T2p;
            g.lda = 2 * P->B2;
            g.strideB = 2LL * P->N2 * P->N3;
            g.strideC = 2LL * P->B2 * P->N3;
            g.M = 2 * P->B2;
            g.K = 2 * P->N2;
            g.N = P->N3;
            return P->T2p ? launch_sgemm<AK_KM, 0>(g, nc * P->B1, sms, s, forced)
                          : launch_sgemm<AK_P2, 0>(g, nc * P->B1, sms, s, forced);
    }
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
    k_table_w1<<<(int)ceil_div_ll((long long)P->B1 * P->N1, T), T, 0, s>>>(P->W1, P->W1t, P->N1, P->B1);
    BLR_CK_LAUNCH();
    k_table_kx<<<(int)ceil_div_ll((long long)P->B2 * P->N2, T), T, 0, s>>>(P->T2c, P->T2s, P->N2, P->B2);
    BLR_CK_LAUNCH();
    k_table_kx<<<(int)ceil_div_ll((long long)P->B3 * P->N3, T), T, 0, s>>>(P->T3c, P->T3s, P->N3, P->B3);
    BLR_CK_LAUNCH();
    if (P->T3e) {
        k_table_axis3<<<(int)ceil_div_ll((long long)P->B3 * P->N3, T), T, 0, s>>>(P->T3e, P->N3,
                                                                                 P->B3);
        BLR_CK_LAUNCH();
    }
    if (P->T2e && P->T2p) {
        k_table_axis2<<<(int)ceil_div_ll((long long)P->B2 * P->N2, T), T, 0, s>>>(P->T2e, P->T2p,
                                                                                 P->N2, P->B2);
        BLR_CK_LAUNCH();
    }
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
    if (P->T3e) {
        int rc = launch_stage(P, 4, vt, P->dft_small, 1.f, 0, s);
        if (rc) return rc;
    } else {
        dim3 ga((unsigned)ceil_div_ll(rows, XR), (unsigned)ceil_div_ll(P->N3, XC));
        const size_t sa = expand_axis3_smem(P->B3);
        BLR_CK(cudaFuncSetAttribute(k_expand_axis3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa));
        launch_pdl(k_expand_axis3, ga, dim3(256), sa, s, vt, (const float *)P->T3c,
                   (const float *)P->T3s, P->dft_small, rows, P->B2, P->B3, P->N3);
        BLR_CK_LAUNCH();
    }
    // stage B
    if (P->tc_tab2_expand) {
        int rc = tc_axis2(P, 0, P->dft_small, P->dft_big, s);
        if (rc) return rc;
    } else {
        int rc = launch_stage(P, 0, P->dft_small, P->dft_big, 1.f, 0, s);
        if (rc) return rc;
    }
    // stage C
    if (P->p.precision == BLR_MIXED) {
        int rc = tc_axis1(P, 0, P->dft_big, out, mode == 0 ? 1.f : -P->dt, mode, s);
        if (rc || mode == 0 || out != P->d) return rc;
        return sweep_pack_d4(P, s);
    }
    const int rc = launch_stage(P, 1, P->dft_big, out, mode == 0 ? 1.f : -P->dt, mode, s);
    if (rc) return rc;
    if (mode == 1 && out == P->d) return sweep_pack_d4(P, s);
    return BLR_OK;
}

int dft_project(blr_plan *P, const float *f, float *ft, const float *vadd, cudaStream_t s,
                float areg) {
    if (P->fz_tab[0]) return fz_project(P, f, ft, vadd, areg, s);
    // stage C'
    if (P->p.precision == BLR_MIXED) {
        int rc = tc_axis1(P, 1, f, P->dft_big, 1.f, 0, s);
        if (rc) return rc;
    } else {
        int rc = launch_stage(P, 2, f, P->dft_big, 1.f, 0, s);
        if (rc) return rc;
    }
    // stage B'
    if (P->tc_tab2_project) {
        int rc = tc_axis2(P, 1, P->dft_big, P->dft_small, s);
        if (rc) return rc;
    } else {
        int rc = launch_stage(P, 3, P->dft_big, P->dft_small, 1.f, 0, s);
        if (rc) return rc;
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

// Tile shapes of the FP32 GEMM stages, chosen by timing each candidate on the
// plan's own buffers (at creation, while they hold nothing).
int dft_autotune(blr_plan *P, cudaStream_t s) {
    for (int st = 0; st < 5; ++st) P->gemm_tile[st] = 0;
    if (!P->T2e || !P->T2p || !P->W1t || !P->T3e) return BLR_OK;   // FP32 plans only
    cudaEvent_t e0, e1;
    BLR_CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return BLR_ECUDA;
    }
    const float *ins[5] = {P->dft_small, P->dft_big, P->dv, P->dft_big, P->vt};
    float *outs[5] = {P->dft_big, P->dv, P->dft_big, P->dft_small, P->dft_small};
    int rc = BLR_OK;
    for (int st = 0; st < 5 && !rc; ++st) {
        float best = 1e30f;
        int pick = 0;
        for (int c = 1; c <= SG_CANDS && !rc; ++c) {
            P->gemm_tile[st] = c;
            float tot = 0.f;
            for (int rep = 0; rep < 4 && !rc; ++rep) {
                if (cudaEventRecord(e0, s) != cudaSuccess) rc = BLR_ECUDA;
                if (!rc) rc = launch_stage(P, st, ins[st], outs[st], 1.f, 0, s);
                if (!rc && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                    rc = BLR_ECUDA;
                float ms = 0.f;
                if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = BLR_ECUDA;
                if (rep) tot += ms;
            }
            if (tot < best) {
                best = tot;
                pick = c;
            }
        }
        P->gemm_tile[st] = pick;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// nc fields (3 per velocity) in one transform: the fused kernels, or the FP32 GEMM
// stages (the plan's intermediates then hold nvel velocities).  Mode 1 writes the
// displacements without packing d4 (the caller packs each step's copy).
int dft_expand_nc(blr_plan *P, const float *vt, float *out, int mode, cudaStream_t s, int nc) {
    if (P->fz_tab[0]) return fz_expand(P, vt, out, mode == 0 ? 1.f : -P->dt, mode, s, nc);
    if (P->p.precision != BLR_FP32 || !P->T3e || nc > 3 * P->nvel) return BLR_EINVAL;
    int rc = launch_stage(P, 4, vt, P->dft_small, 1.f, 0, s, nc);
    if (!rc) rc = launch_stage(P, 0, P->dft_small, P->dft_big, 1.f, 0, s, nc);
    if (!rc) rc = launch_stage(P, 1, P->dft_big, out, mode == 0 ? 1.f : -P->dt, mode, s, nc);
    return rc;
}

int dft_project_nc(blr_plan *P, const float *f, float *ft, const float *vadd, cudaStream_t s,
                   float areg, int nc) {
    if (P->fz_tab[0]) return fz_project(P, f, ft, vadd, areg, s, nc);
    if (P->p.precision != BLR_FP32 || !P->W1t || nc > 3 * P->nvel) return BLR_EINVAL;
    int rc = launch_stage(P, 2, f, P->dft_big, 1.f, 0, s, nc);
    if (!rc) rc = launch_stage(P, 3, P->dft_big, P->dft_small, 1.f, 0, s, nc);
    if (rc) return rc;
    const int rows = nc * P->B1 * P->B2;
    const size_t sp = project_axis3_smem(P->B3);
    BLR_CK(cudaFuncSetAttribute(k_project_axis3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp));
    launch_pdl(k_project_axis3, dim3((unsigned)ceil_div_ll(rows, XR)), dim3(256), sp, s,
               (const float *)P->dft_small, (const float *)P->T3c, (const float *)P->T3s, ft,
               (const float *)P->A, vadd, areg, rows, P->B2, P->B3, P->N3, P->B1 * P->B2);
    BLR_CK_LAUNCH();
    return BLR_OK;
}
