// Fused truncated DFTs of the mixed-precision path (BLR_MIXED), Section 3.1, Eq. 33:
//
//   iota(v~)_c(x) = Re sum_{j1 j2 j3} v~_c(j) E1[j1][x1] E2[j2][x2] E3[j3][x3],
//   pi(f)_c(j)    = sum_x f_c(x) conj(E1[j1][x1] E2[j2][x2] E3[j3][x3]),
//   E_d[j][x] = exp(2 pi i k_j x / N_d) = C_d + i S_d,  k_j = j - B_d / 2.
//
// The contraction order puts the axis-1 sum on the band-sized data, so that the
// grid-sized field is produced (iota) or consumed (pi) by a single kernel:
//
//   expand  k_ex1 (SIMT, FP32):  P1[c][x1][j2][j3] = sum_j1 v~_c(j) E1[j1][x1]
//           k_fx  (tcgen05):     per unit (c, x1, x2 tile of 128 rows)
//                                D2[x2][j3 re|im] = sum_j2 E2 P1        (GEMM 2)
//                                v[c][x1][x2][x3] = Re sum_j3 D2 E3     (GEMM 3)
//   project k_fp  (tcgen05):     per unit (c, x1, x2 tile)
//                                Q3[x2][j3 re|im] = sum_x3 f conj(E3)   (GEMM 3')
//                                Q2[j2][j3] = sum_{x2 in tile} conj(E2) Q3  (GEMM 2')
//           k_p1  (SIMT, FP32):  pi(f)_c(j) = sum_{x1, tiles} conj(E1) Q2 (+ A v~ term)
//
// Tensor-core operands are split into BF16 hi + lo parts and every product is
// Ah Bh + Ah Bl + Al Bh accumulated in FP32 in tensor memory, as in dft_tc.cu.
// The DFT tables are built once per plan in FP64, split and stored pre-swizzled;
// a CTA fetches them once by bulk copy (before the programmatic-launch wait) and
// keeps them in shared memory.  The field operand of GEMM 3' is read from global
// memory, split and swizzled by the CTA; the intermediates D2 and Q3 go from
// tensor memory through registers (and for Q3 a shared-memory transpose) into
// the next GEMM's operand without touching global memory.
//
// Every wait is bounded: a wait that expires sets BLR_FLAG_TIMEOUT, the CTA
// waits (bounded) for its table copy if one was issued, frees tensor memory and
// returns.  blr_test_expire_waits makes each CTA take that path on purpose before
// it issues anything.
#include <cuda.h>
#include <cuda_bf16.h>

#include <atomic>

#include "blr_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int FZ_THREADS = 256;   // 8 warps
constexpr int FZ_M = 128;         // rows of every MMA (x2 tile, or (j3, re|im) padded)
constexpr int PZ_MAX_SMEM = 227 * 1024;

__host__ __device__ inline int up16(int v) { return (v + 15) & ~15; }
__host__ __device__ inline int up64(int v) { return (v + 63) & ~63; }

// Geometry of the two fused kernels of a plan.
struct FzGeom {
    int MT;              // x2 tiles of 128 rows
    // expand: GEMM 2 is [128 x K2e] x [K2e x N2e], GEMM 3 is [128 x K3e] x [K3e x N3e]
    int K2e, N2e, K3e, N3e;
    // project: GEMM 3' is [128 x K3p] x [K3p x N3p], GEMM 2' is [128 x 128] x [128 x N2p]
    int K3p, N3p, N2p;
};

FzGeom fz_geometry(const blr_plan *P) {
    FzGeom g;
    g.MT = (P->N2 + FZ_M - 1) / FZ_M;
    g.K2e = up64(2 * P->B2);
    g.N2e = up16(2 * P->B3);
    g.K3e = up64(2 * P->B3);
    g.N3e = up16(P->N3);
    g.K3p = up64(P->N3);
    g.N3p = up16(2 * P->B3);
    g.N2p = up16(2 * P->B2);
    return g;
}

// bytes of one hi or lo BF16 operand tile of `rows` x `k`
__host__ __device__ inline size_t tile_bytes(int rows, int k) { return (size_t)rows * k * 2; }

// Shared memory: tables, then the operand region (expand: B operand of GEMM 2,
// then A operand of GEMM 3, then the epilogue transposes, one after the other in
// the same bytes), then three barriers and the TMEM slot.
size_t fx_smem(const FzGeom &g) {
    const size_t t2 = 2 * tile_bytes(FZ_M, g.K2e), t3 = 2 * tile_bytes(g.N3e, g.K3e);
    size_t r = 2 * tile_bytes(g.N2e, g.K2e);
    r = r > 2 * tile_bytes(FZ_M, g.K3e) ? r : 2 * tile_bytes(FZ_M, g.K3e);
    r = r > (size_t)(FZ_THREADS / 32) * 4096 ? r : (size_t)(FZ_THREADS / 32) * 4096;
    return 1024 + t2 + t3 + r + 4 * 8 + 16;
}

// project: tables, the A operand region (field tile, then the transposed Q3),
// and the FP32 staging of Q3 (then of GEMM 2's result).
inline int qpitch(const FzGeom &g) { return g.N3p + 4; }
inline int epitch(const FzGeom &g) { return g.N2p + 1; }
size_t fp_smem(const FzGeom &g) {
    const size_t t3 = 2 * tile_bytes(g.N3p, g.K3p), t2 = 2 * tile_bytes(g.N2p, FZ_M);
    const size_t ka = g.K3p > FZ_M ? g.K3p : FZ_M;
    const size_t a = 2 * tile_bytes(FZ_M, (int)ka);
    size_t q = (size_t)FZ_M * qpitch(g) * 4;
    const size_t e = (size_t)FZ_M * epitch(g) * 4;
    q = q > e ? q : e;
    return 1024 + t3 + t2 + a + q + 4 * 8 + 16;
}

int pow2_cols(int v) {
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}

// ---------------------------------------------------------------------------
// Tables.  kind 0: expand GEMM 2 A operand, per x2 tile, rows x2, k = (C | S)(j2);
// kind 1: expand GEMM 3 B operand, rows x3, k = (C | -S)(j3);
// kind 2: project GEMM 3' B operand, rows n = (C | -S)(j3), k = x3;
// kind 3: project GEMM 2' B operand, per x2 tile, rows n = (C | S)(j2), k = x2 in tile.
// Values in FP64 (exact integer phase), split into BF16 hi and lo.
__global__ void k_fz_table(uint8_t *tab, int tiles, int rows, int K, int kind, int N, int B) {
    const long long per = (long long)rows * K;
    const long long total = per * tiles;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(e / per);
        const int r = (int)((e % per) / K), k = (int)(e % K);
        int j = -1, x = -1, part = 0;   // part 0: C, 1: S, 2: -S
        if (kind == 0) {
            x = t * FZ_M + r;
            if (k < B) j = k;
            else if (k < 2 * B) { j = k - B; part = 1; }
        } else if (kind == 1) {
            x = r;
            if (k < B) j = k;
            else if (k < 2 * B) { j = k - B; part = 2; }
        } else if (kind == 2) {
            x = k;
            if (r < B) j = r;
            else if (r < 2 * B) { j = r - B; part = 2; }
        } else {
            x = t * FZ_M + k;
            if (r < B) j = r;
            else if (r < 2 * B) { j = r - B; part = 1; }
        }
        double w = 0.0;
        if (j >= 0 && x < N) {
            long long ph = ((long long)(j - B / 2) * x) % N;
            if (ph < 0) ph += N;
            double sn, cs;
            sincospi(2.0 * (double)ph / (double)N, &sn, &cs);
            w = part == 0 ? cs : part == 1 ? sn : -sn;
        }
        const __nv_bfloat16 h = __double2bfloat16(w);
        const __nv_bfloat16 l = __double2bfloat16(w - (double)__bfloat162float(h));
        const size_t tb = tile_bytes(rows, K);
        uint8_t *hi = tab + (size_t)t * 2 * tb, *lo = hi + tb;
        const uint32_t off = swz_chunk(r, k >> 3, rows) + (uint32_t)((k & 7) * 2);
        *reinterpret_cast<__nv_bfloat16 *>(hi + off) = h;
        *reinterpret_cast<__nv_bfloat16 *>(lo + off) = l;
    }
}

// One bf16 MMA chain D (+)= A B over K (multiple of 16) with the split products:
// A tile of `arows` rows, B tile of `brows` rows, both K-major with `kp` columns.
__device__ __forceinline__ void mma_split(uint32_t d, uint32_t a_hi, uint32_t a_lo, int arows,
                                          uint32_t b_hi, uint32_t b_lo, int brows, int kp,
                                          uint32_t idesc) {
    for (int j = 0; j < kp / 16; ++j) {
        const uint32_t oa = (uint32_t)((j >> 2) * arows * 128 + (j & 3) * 32);
        const uint32_t ob = (uint32_t)((j >> 2) * brows * 128 + (j & 3) * 32);
        const uint64_t ah = umma_desc(a_hi + oa), al = umma_desc(a_lo + oa);
        const uint64_t bh = umma_desc(b_hi + ob), bl = umma_desc(b_lo + ob);
        umma_bf16(d, ah, bh, idesc, j > 0);
        umma_bf16(d, ah, bl, idesc, 1u);
        umma_bf16(d, al, bh, idesc, 1u);
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        bar));
}

__device__ __forceinline__ void store_chunk(uint8_t *hi_tile, size_t tb, uint32_t off, const float *x) {
    uint4 h, l;
    split8(x, h, l);
    *reinterpret_cast<uint4 *>(hi_tile + off) = h;
    *reinterpret_cast<uint4 *>(hi_tile + tb + off) = l;
}

// ---------------------------------------------------------------------------
// k_ex1: P1[c][x1][j2 j3] = sum_j1 v~[c][j1][j2 j3] (cos + i sin)(2 pi k_j1 x1 / N1),
// cos / sin from W1 (rows 2j = cos, 2j+1 = -sin).  A block owns 8 planes x1 and
// 256 columns (j2, j3); each thread sums over j1 in order.
constexpr int EX1_XB = 8;
__global__ void __launch_bounds__(256)
k_ex1(const float2 *__restrict__ vt, const float *__restrict__ W1, float2 *__restrict__ P1,
      int N1, int B1, int nb23) {
    extern __shared__ float2 sE[];   // [B1][EX1_XB]
    const int nxb = (N1 + EX1_XB - 1) / EX1_XB;
    const int c = blockIdx.y / nxb, x1b = (blockIdx.y % nxb) * EX1_XB;
    for (int i = threadIdx.x; i < B1 * EX1_XB; i += blockDim.x) {
        const int j = i / EX1_XB, x1 = x1b + (i % EX1_XB);
        sE[i] = x1 < N1 ? make_float2(W1[(2LL * j) * N1 + x1], -W1[(2LL * j + 1) * N1 + x1])
                        : make_float2(0.f, 0.f);
    }
    pdl_wait();   // v~ may come from the previous kernel
    __syncthreads();
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= nb23) return;
    float2 acc[EX1_XB];
#pragma unroll
    for (int q = 0; q < EX1_XB; ++q) acc[q] = make_float2(0.f, 0.f);
    const float2 *src = vt + (long long)c * B1 * nb23 + col;
    for (int j = 0; j < B1; ++j) {
        const float2 v = src[(long long)j * nb23];
#pragma unroll
        for (int q = 0; q < EX1_XB; ++q) {
            const float2 e = sE[j * EX1_XB + q];
            acc[q].x = fmaf(v.x, e.x, fmaf(-v.y, e.y, acc[q].x));
            acc[q].y = fmaf(v.x, e.y, fmaf(v.y, e.x, acc[q].y));
        }
    }
#pragma unroll
    for (int q = 0; q < EX1_XB; ++q)
        if (x1b + q < N1) P1[((long long)c * N1 + x1b + q) * nb23 + col] = acc[q];
}

// ---------------------------------------------------------------------------
// k_p1: pi(f)_c(j1, j2 j3) = sum_x1 sum_t Q2[c][x1][t][j2 j3] (cos - i sin)(2 pi k_j1 x1/N1)
// (+ areg A(j) vadd).  A block owns 4 frequencies j1 and 128 columns; x1 is
// summed in order, table pieces of 256 planes staged in shared memory.
constexpr int P1_JB = 4, P1_XC = 256;
__global__ void __launch_bounds__(128)
k_p1(const float2 *__restrict__ Q2, const float *__restrict__ W1, float2 *__restrict__ ft,
     const float *__restrict__ Aw, const float2 *__restrict__ vadd, float areg, int N1, int B1,
     int MT, int nb23) {
    __shared__ float2 sE[P1_XC * P1_JB];   // [x1][jj]
    const int njb = (B1 + P1_JB - 1) / P1_JB;
    const int c = blockIdx.y / njb, j1b = (blockIdx.y % njb) * P1_JB;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    float2 acc[P1_JB];
#pragma unroll
    for (int q = 0; q < P1_JB; ++q) acc[q] = make_float2(0.f, 0.f);
    bool waited = false;
    for (int x0 = 0; x0 < N1; x0 += P1_XC) {
        const int xn = min(P1_XC, N1 - x0);
        __syncthreads();
        for (int i = threadIdx.x; i < xn * P1_JB; i += blockDim.x) {
            const int xx = i / P1_JB, j = j1b + i % P1_JB, x1 = x0 + xx;
            sE[i] = j < B1 ? make_float2(W1[(2LL * j) * N1 + x1], W1[(2LL * j + 1) * N1 + x1])
                           : make_float2(0.f, 0.f);   // (cos, -sin)
        }
        if (!waited) {
            pdl_wait();   // Q2 comes from the previous kernel
            waited = true;
        }
        __syncthreads();
        if (col < nb23) {
            const float2 *src = Q2 + ((long long)c * N1 + x0) * MT * nb23 + col;
            for (int xx = 0; xx < xn; ++xx) {
                float2 q = src[(long long)xx * MT * nb23];
                for (int t = 1; t < MT; ++t) {
                    const float2 r = src[((long long)xx * MT + t) * nb23];
                    q.x += r.x;
                    q.y += r.y;
                }
#pragma unroll
                for (int jj = 0; jj < P1_JB; ++jj) {   // (qr + i qi)(cos - i sin)
                    const float2 e = sE[xx * P1_JB + jj];
                    acc[jj].x = fmaf(q.x, e.x, fmaf(-q.y, e.y, acc[jj].x));
                    acc[jj].y = fmaf(q.y, e.x, fmaf(q.x, e.y, acc[jj].y));
                }
            }
        }
    }
    if (!waited) pdl_wait();
    if (col >= nb23) return;
#pragma unroll
    for (int jj = 0; jj < P1_JB; ++jj) {
        const int j = j1b + jj;
        if (j >= B1) continue;
        const long long o = ((long long)c * B1 + j) * nb23 + col;
        float2 r = acc[jj];
        if (vadd) {
            const float a = areg * Aw[(long long)j * nb23 + col];
            const float2 v = vadd[o];
            r.x = fmaf(a, v.x, r.x);
            r.y = fmaf(a, v.y, r.y);
        }
        ft[o] = r;
    }
}

// ---------------------------------------------------------------------------
struct FxArgs {
    const uint8_t *tab2;   // [MT][hi|lo][128 x K2e]
    const uint8_t *tab3;   // [hi|lo][N3e x K3e]
    const float2 *P1;      // [3][N1][B2 B3]
    float *out;            // [3][N1][N2][N3]
    int N1, N2, N3, B2, B3, MT;
    int K2e, N2e, K3e, N3e;
    int units;             // 3 N1 MT
    int tmem_cols;
    float scale;
    int mode;              // 0: store scale * v; 1: displacement (clamp, CFL / NaN flags)
    int *status;
    int probe;
};

// TMEM -> (scale, clamp) -> XOR-swizzled 32 x 32 transpose -> rows of 128 bytes.
template <int CW>
__device__ __forceinline__ void fz_epi_chunk(uint32_t ta, float *T, float *dst_rows, int row0,
                                             int rows_valid, int ld, int c0, int cols_valid,
                                             float scale, int mode, int lane, int &flags) {
    uint32_t rv[CW];
    if constexpr (CW == 32) tmem_ld32(ta, rv);
    else tmem_ld16(ta, rv);
#pragma unroll
    for (int q = 0; q < CW; ++q) {
        float v = __uint_as_float(rv[q]) * scale;
        if (mode == 1) {
            const bool valid = (row0 + lane < rows_valid) && (c0 + q < cols_valid);
            if (valid && !(fabsf(v) < 1.f)) flags |= (v != v) ? BLR_FLAG_NAN : BLR_FLAG_CFL;
            v = fminf(fmaxf(v, -1.f), 0.99999994f);
        }
        T[lane * 32 + (q ^ lane)] = v;
    }
    __syncwarp();
    const bool col_ok = lane < CW && (c0 + lane) < cols_valid;
#pragma unroll 8
    for (int q = 0; q < 32; ++q) {
        const int row = row0 + q;
        if (row < rows_valid && col_ok) dst_rows[(long long)row * ld + c0 + lane] = T[q * 32 + (lane ^ q)];
    }
    __syncwarp();
}

__global__ void __launch_bounds__(FZ_THREADS, 2)
k_fx(FxArgs p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023) & ~1023u) - raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t tb2 = tile_bytes(FZ_M, p.K2e), tb3 = tile_bytes(p.N3e, p.K3e);
    const size_t tbB = tile_bytes(p.N2e, p.K2e), tbA = tile_bytes(FZ_M, p.K3e);
    uint8_t *sT2 = base;
    uint8_t *sT3 = sT2 + 2 * tb2;
    uint8_t *sR = sT3 + 2 * tb3;   // B operand of GEMM 2 / A operand of GEMM 3 / epilogue
    size_t rb = 2 * tbB > 2 * tbA ? 2 * tbB : 2 * tbA;
    if (rb < (size_t)(FZ_THREADS / 32) * 4096) rb = (size_t)(FZ_THREADS / 32) * 4096;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sR + rb);   // table, mma, probe
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 4);
    __shared__ int s_fail, s_table;
    const uint32_t bar_tab = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]),
                   bar_probe = smem_u32(&bars[2]);
    const int mt = blockIdx.x % p.MT;   // the grid is a multiple of MT: one x2 tile per CTA

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(p.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(bar_tab, 1);
        mbar_init(bar_mma, 1);
        mbar_init(bar_probe, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_fail = 0;
        s_table = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    bool run = (int)blockIdx.x < p.units;
    if (p.probe) {   // test hook: a wait that expires while nothing is in flight
        const bool expired = tid == 0 ? !mbar_wait(bar_probe, 0u, TC_PROBE_CYCLES) : false;
        if (__syncthreads_or(expired)) run = false;
        if (tid == 0 && expired) s_fail = 1;
    }
    // the tables are plan data written at creation: fetched before the wait for
    // the previous kernel in the stream
    if (tid == 0 && run) {
        mbar_expect_arrive(bar_tab, (uint32_t)(2 * tb2 + 2 * tb3));
        bulk_g2s(smem_u32(sT2), p.tab2 + (size_t)mt * 2 * tb2, (uint32_t)(2 * tb2), bar_tab);
        bulk_g2s(smem_u32(sT3), p.tab3, (uint32_t)(2 * tb3), bar_tab);
        s_table = 1;
    }
    pdl_wait();
    if (run) {
        const bool ok = tid == 0 ? mbar_wait(bar_tab, 0u) : true;
        if (__syncthreads_or(!ok)) {
            run = false;
            if (tid == 0) s_fail = 1;
        }
    }
    const int nb23 = p.B2 * p.B3;
    const uint32_t idesc2 = umma_idesc(FZ_M, p.N2e), idesc3 = umma_idesc(FZ_M, p.N3e);
    const long long V = (long long)p.N1 * p.N2 * p.N3;
    uint32_t phase = 0;
    int flags = 0;
    for (int u = blockIdx.x; run && u < p.units; u += gridDim.x) {
        const int rest = u / p.MT, c = rest / p.N1, x1 = rest - c * p.N1;
        const float2 *src = p.P1 + ((long long)c * p.N1 + x1) * nb23;
        // B operand of GEMM 2, [n = (re | im)(j3)][k = (C | S)(j2)]:
        //   (C, re) P1re  (C, im) P1im  (S, re) -P1im  (S, im) P1re
        {
            const int nkc = p.K2e >> 3;
            for (int it = tid; it < p.N2e * nkc; it += FZ_THREADS) {
                const int n = it % p.N2e, kc = it / p.N2e;
                float x[8];
                const bool im = n >= p.B3;
                const int j3 = im ? n - p.B3 : n;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = kc * 8 + q;
                    float v = 0.f;
                    if (n < 2 * p.B3 && k < 2 * p.B2) {
                        const bool sp = k >= p.B2;
                        const float2 w = src[(sp ? k - p.B2 : k) * p.B3 + j3];
                        v = sp ? (im ? w.x : -w.y) : (im ? w.y : w.x);
                    }
                    x[q] = v;
                }
                store_chunk(sR, tbB, swz_chunk(n, kc, p.N2e), x);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            mma_split(tmem, smem_u32(sT2), smem_u32(sT2) + (uint32_t)tb2, FZ_M, smem_u32(sR),
                      smem_u32(sR) + (uint32_t)tbB, p.N2e, p.K2e, idesc2);
            mma_commit(bar_mma);
        }
        bool ok = tid == 0 ? mbar_wait(bar_mma, phase) : true;
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) s_fail = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // D2 rows (TMEM lane = x2 row) -> A operand of GEMM 3, [x2][k = (re | im)(j3)]
        if (warp < 4) {
            const int r = warp * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
            for (int c0 = 0; c0 < p.N2e; c0 += 16) {
                uint32_t rv[16];
                tmem_ld16(trow + (uint32_t)c0, rv);
                store_chunk(sR, tbA, swz_chunk(r, c0 >> 3, FZ_M), reinterpret_cast<const float *>(rv));
                store_chunk(sR, tbA, swz_chunk(r, (c0 >> 3) + 1, FZ_M),
                            reinterpret_cast<const float *>(rv) + 8);
            }
            const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int kc = p.N2e >> 3; kc < (p.K3e >> 3); ++kc) store_chunk(sR, tbA, swz_chunk(r, kc, FZ_M), z);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            mma_split(tmem + (uint32_t)p.N2e, smem_u32(sR), smem_u32(sR) + (uint32_t)tbA, FZ_M,
                      smem_u32(sT3), smem_u32(sT3) + (uint32_t)tb3, p.N3e, p.K3e, idesc3);
            mma_commit(bar_mma);
        }
        ok = tid == 0 ? mbar_wait(bar_mma, phase) : true;
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) s_fail = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (x2 rows), the two warps of
        // a quadrant alternate 32-column chunks (x3)
        {
            const int lg = warp & 3, half = warp >> 2;
            float *T = reinterpret_cast<float *>(sR) + warp * 1024;
            const int row0 = mt * FZ_M + lg * 32;
            float *dst = p.out + c * V + (long long)x1 * p.N2 * p.N3;
            const uint32_t tq = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)p.N2e;
            for (int c0 = half * 32; c0 < p.N3e; c0 += 64) {
                if (c0 + 32 <= p.N3e)
                    fz_epi_chunk<32>(tq + (uint32_t)c0, T, dst, row0, p.N2, p.N3, c0, p.N3, p.scale,
                                     p.mode, lane, flags);
                else
                    fz_epi_chunk<16>(tq + (uint32_t)c0, T, dst, row0, p.N2, p.N3, c0, p.N3, p.scale,
                                     p.mode, lane, flags);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    if (flags) atomicOr(p.status, flags);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (s_fail && tid == 0) {
        atomicOr(p.status, BLR_FLAG_TIMEOUT);
        if (s_table) mbar_wait(bar_tab, 0u);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(p.tmem_cols));
}

// ---------------------------------------------------------------------------
struct FpArgs {
    const uint8_t *tab3;   // [hi|lo][N3p x K3p]
    const uint8_t *tab2;   // [MT][hi|lo][N2p x 128]
    const float *f;        // [3][N1][N2][N3]
    float2 *Q2;            // [3][N1][MT][B2 B3]
    int N1, N2, N3, B2, B3, MT;
    int K3p, N3p, N2p;
    int units;
    int tmem_cols;
    int vec4;              // rows of f are 16-byte aligned (N3 % 4 == 0, aligned base)
    int *status;
    int probe;
};

__global__ void __launch_bounds__(FZ_THREADS, 1)
k_fp(FpArgs p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023) & ~1023u) - raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t tb3 = tile_bytes(p.N3p, p.K3p), tb2 = tile_bytes(p.N2p, FZ_M);
    const int ka = p.K3p > FZ_M ? p.K3p : FZ_M;
    const size_t tbA = tile_bytes(FZ_M, p.K3p), tbA2 = tile_bytes(FZ_M, FZ_M);
    uint8_t *sT3 = base;
    uint8_t *sT2 = sT3 + 2 * tb3;
    uint8_t *sA = sT2 + 2 * tb2;                  // field tile, then the transposed Q3
    float *sQ = reinterpret_cast<float *>(sA + 2 * tile_bytes(FZ_M, ka));
    const int qp = p.N3p + 4, ep = p.N2p + 1;
    const size_t qbytes = (size_t)FZ_M * (qp > ep ? qp : ep) * 4;
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(sQ) + qbytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 4);
    __shared__ int s_fail, s_table;
    const uint32_t bar_tab = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]),
                   bar_probe = smem_u32(&bars[2]);
    const int mt = blockIdx.x % p.MT;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(p.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(bar_tab, 1);
        mbar_init(bar_mma, 1);
        mbar_init(bar_probe, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_fail = 0;
        s_table = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    bool run = (int)blockIdx.x < p.units;
    if (p.probe) {
        const bool expired = tid == 0 ? !mbar_wait(bar_probe, 0u, TC_PROBE_CYCLES) : false;
        if (__syncthreads_or(expired)) run = false;
        if (tid == 0 && expired) s_fail = 1;
    }
    if (tid == 0 && run) {
        mbar_expect_arrive(bar_tab, (uint32_t)(2 * tb3 + 2 * tb2));
        bulk_g2s(smem_u32(sT3), p.tab3, (uint32_t)(2 * tb3), bar_tab);
        bulk_g2s(smem_u32(sT2), p.tab2 + (size_t)mt * 2 * tb2, (uint32_t)(2 * tb2), bar_tab);
        s_table = 1;
    }
    pdl_wait();
    if (run) {
        const bool ok = tid == 0 ? mbar_wait(bar_tab, 0u) : true;
        if (__syncthreads_or(!ok)) {
            run = false;
            if (tid == 0) s_fail = 1;
        }
    }
    const int nb23 = p.B2 * p.B3;
    const uint32_t idesc3 = umma_idesc(FZ_M, p.N3p), idesc2 = umma_idesc(FZ_M, p.N2p);
    const long long V = (long long)p.N1 * p.N2 * p.N3;
    const int rows = min(FZ_M, p.N2 - mt * FZ_M);   // x2 rows of this CTA's tile
    uint32_t phase = 0;
    for (int u = blockIdx.x; run && u < p.units; u += gridDim.x) {
        const int rest = u / p.MT, c = rest / p.N1, x1 = rest - c * p.N1;
        const float *src = p.f + c * V + ((long long)x1 * p.N2 + (long long)mt * FZ_M) * p.N3;
        // field tile -> A operand of GEMM 3', [x2][k = x3]: each thread loads all its
        // chunks first (many loads in flight), then splits and stores them
        {
            const int nkc = p.K3p >> 3, total = FZ_M * nkc;
            constexpr int PER = 8;
            for (int base_it = 0; base_it < total; base_it += FZ_THREADS * PER) {
                float x[PER][8];
#pragma unroll
                for (int s = 0; s < PER; ++s) {
                    const int it = base_it + s * FZ_THREADS + tid;
                    const int r = it / nkc, kc = it - r * nkc, k0 = kc * 8;
                    const bool live = it < total && r < rows;
                    if (live && p.vec4 && k0 + 8 <= p.N3) {
                        const float4 a = __ldg(reinterpret_cast<const float4 *>(src + (long long)r * p.N3 + k0));
                        const float4 b = __ldg(reinterpret_cast<const float4 *>(src + (long long)r * p.N3 + k0 + 4));
                        x[s][0] = a.x; x[s][1] = a.y; x[s][2] = a.z; x[s][3] = a.w;
                        x[s][4] = b.x; x[s][5] = b.y; x[s][6] = b.z; x[s][7] = b.w;
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            x[s][q] = (live && k0 + q < p.N3) ? __ldg(src + (long long)r * p.N3 + k0 + q) : 0.f;
                    }
                }
#pragma unroll
                for (int s = 0; s < PER; ++s) {
                    const int it = base_it + s * FZ_THREADS + tid;
                    if (it < total) {
                        const int r = it / nkc, kc = it - r * nkc;
                        store_chunk(sA, tbA, swz_chunk(r, kc, FZ_M), x[s]);
                    }
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            mma_split(tmem, smem_u32(sA), smem_u32(sA) + (uint32_t)tbA, FZ_M, smem_u32(sT3),
                      smem_u32(sT3) + (uint32_t)tb3, p.N3p, p.K3p, idesc3);
            mma_commit(bar_mma);
        }
        bool ok = tid == 0 ? mbar_wait(bar_mma, phase) : true;
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) s_fail = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // Q3 rows (TMEM lane = x2) -> FP32 staging [x2][n]
        if (warp < 4) {
            const int r = warp * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
            for (int c0 = 0; c0 < p.N3p; c0 += 16) {
                uint32_t rv[16];
                tmem_ld16(trow + (uint32_t)c0, rv);
                float4 *d = reinterpret_cast<float4 *>(sQ + (size_t)r * qp + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    d[q] = make_float4(__uint_as_float(rv[4 * q]), __uint_as_float(rv[4 * q + 1]),
                                       __uint_as_float(rv[4 * q + 2]), __uint_as_float(rv[4 * q + 3]));
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        // transposed Q3 -> A operand of GEMM 2', [m = (re | im)(j3)][k = x2 in tile];
        // rows m >= N3p keep stale values: their products land in rows that are
        // never read
        for (int it = tid; it < p.N3p * (FZ_M / 8); it += FZ_THREADS) {
            const int m = it % p.N3p, kc = it / p.N3p;
            float x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = sQ[(size_t)(kc * 8 + q) * qp + m];
            store_chunk(sA, tbA2, swz_chunk(m, kc, FZ_M), x);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            mma_split(tmem + (uint32_t)p.N3p, smem_u32(sA), smem_u32(sA) + (uint32_t)tbA2, FZ_M,
                      smem_u32(sT2), smem_u32(sT2) + (uint32_t)tb2, p.N2p, FZ_M, idesc2);
            mma_commit(bar_mma);
        }
        ok = tid == 0 ? mbar_wait(bar_mma, phase) : true;
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) s_fail = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // GEMM 2' rows m < 2 B3 -> FP32 staging [m][n] (odd pitch: column reads below)
        if (warp < 4) {
            const int m = warp * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)p.N3p;
            for (int c0 = 0; c0 < p.N2p; c0 += 16) {
                uint32_t rv[16];
                tmem_ld16(trow + (uint32_t)c0, rv);
                if (m < 2 * p.B3) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) sQ[(size_t)m * ep + c0 + q] = __uint_as_float(rv[q]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        // Q2[j2][j3] = (C re + S im, C im - S re) combinations of the four blocks
        float2 *dst = p.Q2 + (((long long)c * p.N1 + x1) * p.MT + mt) * nb23;
        for (int e = tid; e < nb23; e += FZ_THREADS) {
            const int j2 = e / p.B3, j3 = e - j2 * p.B3;
            const float *re = sQ + (size_t)j3 * ep, *im = sQ + (size_t)(p.B3 + j3) * ep;
            dst[e] = make_float2(re[j2] + im[p.B2 + j2], im[j2] - re[p.B2 + j2]);
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (s_fail && tid == 0) {
        atomicOr(p.status, BLR_FLAG_TIMEOUT);
        if (s_table) mbar_wait(bar_tab, 0u);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(p.tmem_cols));
}

// CTAs of a fused kernel per SM from its shared memory and TMEM columns.
int fz_ctas_per_sm(size_t smem, int cols) {
    constexpr size_t SM_SMEM = 228 * 1024, RESERVED = 1024;
    int k = 1;
    while ((size_t)(k + 1) * (smem + RESERVED) <= SM_SMEM && (k + 1) * cols <= 512 && k < 2) ++k;
    return k;
}

int fz_grid(const blr_plan *P, int units, int per_sm, int MT) {
    int grid = per_sm * (P->sms > 0 ? P->sms : 148);
    if (grid > units) grid = units;
    grid = grid / MT * MT;
    return grid < MT ? MT : grid;
}

}  // namespace

extern std::atomic<int> g_tc_probe;   // dft_tc.cu (blr_test_expire_waits)

// ---------------------------------------------------------------------------
// host side

bool fz_supported(const blr_plan *P) {
    const FzGeom g = fz_geometry(P);
    if (P->N3 > 256 || P->B2 > 128 || 2 * P->B3 > FZ_M) return false;
    if (g.N2e + g.N3e > 512 || g.N3p + g.N2p > 512) return false;
    return fx_smem(g) <= PZ_MAX_SMEM && fp_smem(g) <= PZ_MAX_SMEM;
}

size_t fz_table_bytes(const blr_plan *P, int kind) {
    const FzGeom g = fz_geometry(P);
    switch (kind) {
        case 0: return (size_t)g.MT * 2 * tile_bytes(FZ_M, g.K2e);
        case 1: return 2 * tile_bytes(g.N3e, g.K3e);
        case 2: return 2 * tile_bytes(g.N3p, g.K3p);
        default: return (size_t)g.MT * 2 * tile_bytes(g.N2p, FZ_M);
    }
}

// floats of the intermediate: P1 [3][N1][B2 B3] complex, or Q2 [3][N1][MT][B2 B3]
size_t fz_buffer_floats(const blr_plan *P) {
    const FzGeom g = fz_geometry(P);
    return (size_t)2 * 3 * P->N1 * g.MT * P->B2 * P->B3;
}

int fz_init_tables(blr_plan *P, cudaStream_t s) {
    const FzGeom g = fz_geometry(P);
    struct T { uint8_t *tab; int tiles, rows, K, kind, N, B; } t[4] = {
        {P->fz_tab[0], g.MT, FZ_M, g.K2e, 0, P->N2, P->B2},
        {P->fz_tab[1], 1, g.N3e, g.K3e, 1, P->N3, P->B3},
        {P->fz_tab[2], 1, g.N3p, g.K3p, 2, P->N3, P->B3},
        {P->fz_tab[3], g.MT, g.N2p, FZ_M, 3, P->N2, P->B2}};
    for (const T &x : t) {
        k_fz_table<<<256, 256, 0, s>>>(x.tab, x.tiles, x.rows, x.K, x.kind, x.N, x.B);
        BLR_CK_LAUNCH();
    }
    return BLR_OK;
}

int fz_expand(blr_plan *P, const float *vt, float *out, float scale, int mode, cudaStream_t s) {
    const FzGeom g = fz_geometry(P);
    const int nb23 = P->B2 * P->B3;
    float2 *P1 = reinterpret_cast<float2 *>(P->fz_buf);
    const int nxb = (P->N1 + EX1_XB - 1) / EX1_XB;
    launch_pdl(k_ex1, dim3((unsigned)((nb23 + 255) / 256), (unsigned)(3 * nxb)), dim3(256),
               (size_t)P->B1 * EX1_XB * sizeof(float2), s, reinterpret_cast<const float2 *>(vt),
               (const float *)P->W1, P1, P->N1, P->B1, nb23);
    BLR_CK_LAUNCH();
    FxArgs a;
    a.tab2 = P->fz_tab[0];
    a.tab3 = P->fz_tab[1];
    a.P1 = P1;
    a.out = out;
    a.N1 = P->N1;
    a.N2 = P->N2;
    a.N3 = P->N3;
    a.B2 = P->B2;
    a.B3 = P->B3;
    a.MT = g.MT;
    a.K2e = g.K2e;
    a.N2e = g.N2e;
    a.K3e = g.K3e;
    a.N3e = g.N3e;
    a.units = 3 * P->N1 * g.MT;
    a.tmem_cols = pow2_cols(g.N2e + g.N3e);
    a.scale = scale;
    a.mode = mode;
    a.status = P->dstatus;
    a.probe = g_tc_probe.load(std::memory_order_relaxed);
    const size_t smem = fx_smem(g);
    BLR_CK(cudaFuncSetAttribute(k_fx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = fz_grid(P, a.units, fz_ctas_per_sm(smem, a.tmem_cols), g.MT);
    launch_pdl(k_fx, dim3(grid), dim3(FZ_THREADS), smem, s, a);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int fz_project(blr_plan *P, const float *f, float *ft, const float *vadd, float areg,
               cudaStream_t s) {
    const FzGeom g = fz_geometry(P);
    const int nb23 = P->B2 * P->B3;
    float2 *Q2 = reinterpret_cast<float2 *>(P->fz_buf);
    FpArgs a;
    a.tab3 = P->fz_tab[2];
    a.tab2 = P->fz_tab[3];
    a.f = f;
    a.Q2 = Q2;
    a.N1 = P->N1;
    a.N2 = P->N2;
    a.N3 = P->N3;
    a.B2 = P->B2;
    a.B3 = P->B3;
    a.MT = g.MT;
    a.K3p = g.K3p;
    a.N3p = g.N3p;
    a.N2p = g.N2p;
    a.units = 3 * P->N1 * g.MT;
    a.tmem_cols = pow2_cols(g.N3p + g.N2p);
    a.vec4 = (P->N3 % 4 == 0) && ((uintptr_t)f % 16 == 0);
    a.status = P->dstatus;
    a.probe = g_tc_probe.load(std::memory_order_relaxed);
    const size_t smem = fp_smem(g);
    BLR_CK(cudaFuncSetAttribute(k_fp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = fz_grid(P, a.units, fz_ctas_per_sm(smem, a.tmem_cols), g.MT);
    launch_pdl(k_fp, dim3(grid), dim3(FZ_THREADS), smem, s, a);
    BLR_CK_LAUNCH();
    const int njb = (P->B1 + P1_JB - 1) / P1_JB;
    launch_pdl(k_p1, dim3((unsigned)((nb23 + 127) / 128), (unsigned)(3 * njb)), dim3(128), 0, s,
               (const float2 *)Q2, (const float *)P->W1, reinterpret_cast<float2 *>(ft),
               (const float *)P->A, reinterpret_cast<const float2 *>(vadd), areg, P->N1, P->B1,
               g.MT, nb23);
    BLR_CK_LAUNCH();
    return BLR_OK;
}
