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

int pow2_cols(int v) {
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}

size_t up1k(size_t v) { return (v + 1023) & ~(size_t)1023; }

// Launch shape of a fused kernel: G warpgroups of 128 threads, each with `gbytes`
// of operand buffer and `gcols` TMEM columns, after `fixed` bytes of tables.
struct FzShape {
    int G, gcols, tmem_cols;
    size_t gbytes, smem;
};

// G: the most warpgroups that fit (shared memory, 512 TMEM columns), at most 4 and
// at most the units a CTA gets when every SM has one (gmax, 0: no cap).
FzShape fz_shape(size_t fixed, size_t gbytes, int gcols, size_t tail, int gmax = 0) {
    FzShape sh;
    sh.gbytes = up1k(gbytes);
    sh.gcols = gcols;
    sh.G = 4;
    while (sh.G > 0 && (fixed + sh.G * sh.gbytes + tail > (size_t)PZ_MAX_SMEM || sh.G * gcols > 512))
        --sh.G;
    if (gmax > 0 && sh.G > gmax) sh.G = gmax;
    sh.tmem_cols = pow2_cols(sh.G * gcols);
    sh.smem = fixed + sh.G * sh.gbytes + tail;
    return sh;
}

// expand: tables T2e (A of GEMM 2) and T3e (B of GEMM 3); per warpgroup the B
// operand of GEMM 2 (with the unit's P1 slab, or a 1/parts share of it, beside
// it), then the A operand of GEMM 3, then four epilogue transposes, one after
// the other in the same bytes; D3 reuses the TMEM columns of D2.
FzShape fx_shape(const FzGeom &g, int B2, int B3, int gmax = 0, int parts = 1) {
    const size_t fixed = 1024 + 2 * tile_bytes(FZ_M, g.K2e) + 2 * tile_bytes(g.N3e, g.K3e);
    size_t r = 2 * tile_bytes(g.N2e, g.K2e) + (size_t)B2 * B3 * 8 / parts;   // + the P1 slab
    r = r > 2 * tile_bytes(FZ_M, g.K3e) ? r : 2 * tile_bytes(FZ_M, g.K3e);
    r = r > 4 * 4096 ? r : 4 * 4096;
    const int cols = pow2_cols(g.N2e > g.N3e ? g.N2e : g.N3e);
    return fz_shape(fixed, r, cols, 8 * (2 + 2 * 4) + 16, gmax);
}

// project: tables T3p (A of GEMM 3', N3p rows, plus the rows the MMA reads past
// them) and T2p; per warpgroup a field chunk, then the A operand of GEMM 2' (N3p
// rows), then the FP32 staging of its result; D2t reuses the columns of D3t.
FzShape fp_shape(const FzGeom &g, int gmax = 0) {
    const size_t slack = (size_t)(FZ_M - g.N3p) * 128;
    const size_t fixed = 1024 + 2 * tile_bytes(g.N3p, g.K3p) + slack + 2 * tile_bytes(g.N2p, FZ_M);
    size_t r = 2 * tile_bytes(FZ_M, 64);
    r = r > 2 * tile_bytes(g.N3p, FZ_M) ? r : 2 * tile_bytes(g.N3p, FZ_M);
    const size_t e = (size_t)g.N3p * (g.N2p + 1) * 4;
    r = r > e ? r : e;
    const int cols = pow2_cols(FZ_M > g.N2p ? FZ_M : g.N2p);
    return fz_shape(fixed, r, cols, slack + 8 * (2 + 4) + 16, gmax);
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
// k_ex1: P1[c][x1][col] = sum_j1 (cos + i sin)(2 pi k_j1 x1 / N1) v~[c][j1][col], col = (j2, j3),
// a complex GEMM [N1 x B1] x [B1 x B2 B3] per component (cos / sin from W1, rows
// 2j = cos, 2j+1 = -sin).  A block computes a 16 (x1) x 64 (col) tile; j1 runs in
// chunks of 32 staged in shared memory (the next chunk's loads in flight during
// this chunk's sums), summed in order.  Thread (ty, tx) owns x1 row ty and
// columns tx + 16 q (q < 4): stores are coalesced.
constexpr int EX_TX = 16, EX_TC = 64, EX_TK = 32;
constexpr int EX_NE = EX_TK * EX_TX / 256, EX_NV = EX_TK * EX_TC / 256;   // loads per thread
__global__ void __launch_bounds__(256)
k_ex1(const float2 *__restrict__ vt, const float *__restrict__ W1, float2 *__restrict__ P1,
      int N1, int B1, int nb23) {
    __shared__ float2 sE[EX_TK][EX_TX + 1];   // [j1][x1]
    __shared__ float2 sV[EX_TK][EX_TC];       // [j1][col]
    const int c = blockIdx.z, x0 = blockIdx.y * EX_TX, c0 = blockIdx.x * EX_TC;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    pdl_trigger();   // k_fx may launch and fetch its tables meanwhile
    float2 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
    // chunk k0's operands into registers (every load issued before any is used)
    float2 re[EX_NE], rv[EX_NV];
    auto load_e = [&](int k0) {
#pragma unroll
        for (int s = 0; s < EX_NE; ++s) {
            const int i = tid + 256 * s, kk = i / EX_TX, j = k0 + kk, x1 = x0 + i % EX_TX;
            re[s] = (j < B1 && x1 < N1)
                        ? make_float2(W1[(2LL * j) * N1 + x1], -W1[(2LL * j + 1) * N1 + x1])
                        : make_float2(0.f, 0.f);
        }
    };
    auto load_v = [&](int k0) {
#pragma unroll
        for (int s = 0; s < EX_NV; ++s) {
            const int i = tid + 256 * s, kk = i / EX_TC, j = k0 + kk, col = c0 + i % EX_TC;
            rv[s] = (j < B1 && col < nb23) ? vt[((long long)c * B1 + j) * nb23 + col]
                                           : make_float2(0.f, 0.f);
        }
    };
    load_e(0);
    pdl_wait();   // v~ may come from the previous kernel
    load_v(0);
    for (int k0 = 0; k0 < B1; k0 += EX_TK) {
        __syncthreads();
#pragma unroll
        for (int s = 0; s < EX_NE; ++s) {
            const int i = tid + 256 * s;
            sE[i / EX_TX][i % EX_TX] = re[s];
        }
#pragma unroll
        for (int s = 0; s < EX_NV; ++s) {
            const int i = tid + 256 * s;
            sV[i / EX_TC][i % EX_TC] = rv[s];
        }
        __syncthreads();
        if (k0 + EX_TK < B1) {   // the next chunk's loads fly during this chunk's sums
            load_e(k0 + EX_TK);
            load_v(k0 + EX_TK);
        }
#pragma unroll 8
        for (int kk = 0; kk < EX_TK; ++kk) {
            const float2 e = sE[kk][ty];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 v = sV[kk][tx + 16 * q];
                acc[q].x = fmaf(e.x, v.x, fmaf(-e.y, v.y, acc[q].x));
                acc[q].y = fmaf(e.x, v.y, fmaf(e.y, v.x, acc[q].y));
            }
        }
    }
    const int x1 = x0 + ty;
    if (x1 >= N1) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int col = c0 + tx + 16 * q;
        if (col < nb23) P1[((long long)c * N1 + x1) * nb23 + col] = acc[q];
    }
}

// ---------------------------------------------------------------------------
// k_p1: pi(f)_c(j1, col) = sum_x1 (cos - i sin)(2 pi k_j1 x1 / N1) sum_t Q2[c][x1][t][col]
// (+ areg A(j) vadd), a complex GEMM [B1 x N1] x [N1 x B2 B3] per component.  A
// block computes an 8 (j1) x 32 (col) tile; x1 runs in chunks of 32 staged in
// shared memory (the x2-tile partial sums added while staging; the next chunk's
// loads in flight during this chunk's sums), summed in order.  Thread (ty, tx)
// owns frequency j1 = ty and column tx.
constexpr int P1_TJ = 8, P1_TC = 32, P1_TK = 32;
constexpr int P1_NE = P1_TK * P1_TJ / 256, P1_NQ = P1_TK * P1_TC / 256;   // loads per thread
__global__ void __launch_bounds__(256)
k_p1(const float2 *__restrict__ Q2, const float *__restrict__ W1, float2 *__restrict__ ft,
     const float *__restrict__ Aw, const float2 *__restrict__ vadd, float areg, int N1, int B1,
     int MT, int nb23) {
    __shared__ float2 sE[P1_TK][P1_TJ + 1];   // [x1][j1]: (cos, -sin)
    __shared__ float2 sQ[P1_TK][P1_TC];       // [x1][col]
    const int c = blockIdx.z, j0 = blockIdx.y * P1_TJ, c0 = blockIdx.x * P1_TC;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    float2 acc = make_float2(0.f, 0.f);
    float2 re[P1_NE], rq[P1_NQ];
    auto load_e = [&](int k0) {
#pragma unroll
        for (int s = 0; s < P1_NE; ++s) {
            const int i = tid + 256 * s, x1 = k0 + i / P1_TJ, j = j0 + i % P1_TJ;
            re[s] = (j < B1 && x1 < N1) ? make_float2(W1[(2LL * j) * N1 + x1], W1[(2LL * j + 1) * N1 + x1])
                                        : make_float2(0.f, 0.f);
        }
    };
    auto load_q = [&](int k0) {   // the x2-tile partial sums, added in tile order
#pragma unroll
        for (int s = 0; s < P1_NQ; ++s) {
            const int i = tid + 256 * s, x1 = k0 + i / P1_TC, col = c0 + i % P1_TC;
            float2 q = make_float2(0.f, 0.f);
            if (x1 < N1 && col < nb23) {
                const float2 *src = Q2 + ((long long)c * N1 + x1) * MT * nb23 + col;
                q = src[0];
                for (int t = 1; t < MT; ++t) {
                    const float2 r = src[(long long)t * nb23];
                    q.x += r.x;
                    q.y += r.y;
                }
            }
            rq[s] = q;
        }
    };
    load_e(0);
    pdl_wait();   // Q2 comes from the previous kernel
    load_q(0);
    for (int k0 = 0; k0 < N1; k0 += P1_TK) {
        __syncthreads();
#pragma unroll
        for (int s = 0; s < P1_NE; ++s) {
            const int i = tid + 256 * s;
            sE[i / P1_TJ][i % P1_TJ] = re[s];
        }
#pragma unroll
        for (int s = 0; s < P1_NQ; ++s) {
            const int i = tid + 256 * s;
            sQ[i / P1_TC][i % P1_TC] = rq[s];
        }
        __syncthreads();
        if (k0 + P1_TK < N1) {
            load_e(k0 + P1_TK);
            load_q(k0 + P1_TK);
        }
#pragma unroll 8
        for (int kk = 0; kk < P1_TK; ++kk) {   // (qr + i qi)(cos - i sin)
            const float2 e = sE[kk][ty], v = sQ[kk][tx];
            acc.x = fmaf(v.x, e.x, fmaf(-v.y, e.y, acc.x));
            acc.y = fmaf(v.y, e.x, fmaf(v.x, e.y, acc.y));
        }
    }
    const int j = j0 + ty, col = c0 + tx;
    if (j >= B1 || col >= nb23) return;
    const long long o = ((long long)c * B1 + j) * nb23 + col;
    float2 r = acc;
    if (vadd) {
        const float a = areg * Aw[(long long)j * nb23 + col];
        const float2 v = vadd[o];
        r.x = fmaf(a, v.x, r.x);
        r.y = fmaf(a, v.y, r.y);
    }
    ft[o] = r;
}

// ---------------------------------------------------------------------------
// Both tensor-core kernels run one CTA per SM with G independent warpgroups of
// 128 threads.  The DFT tables are loaded once per CTA and shared; each
// warpgroup owns an operand buffer in shared memory, a range of tensor-memory
// columns, an mbarrier for its MMAs and a named barrier, and walks its own units
// one after the other, so the units of the G warpgroups overlap.  Warp w of a
// warpgroup reaches TMEM lanes 32 w .. 32 w + 31.

__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
}

// The group's MMAs are complete (thread 0 of the group waits, bounded; the
// group learns the outcome through shared memory after the named barrier).
__device__ __forceinline__ bool group_wait(int g, int gt, uint32_t bar, uint32_t phase,
                                           volatile int *s_ok) {
    if (gt == 0) s_ok[g] = mbar_wait(bar, phase) ? 1 : 0;
    group_sync(g);
    const bool ok = s_ok[g] != 0;
    group_sync(g);   // everyone has read the flag before it is written again
    return ok;
}

constexpr int FZ_G_MAX = 4;

struct FxArgs {
    const uint8_t *tab2;   // [MT][hi|lo][128 x K2e]
    const uint8_t *tab3;   // [hi|lo][N3e x K3e]
    const float2 *P1;      // [3][N1][B2 B3]
    float *out;            // [3][N1][N2][N3]
    int N1, N2, N3, B2, B3, MT;
    int K2e, N2e, K3e, N3e;
    int G;                 // warpgroups per CTA
    size_t gbytes;         // operand buffer of a warpgroup
    int gcols;             // TMEM columns of a warpgroup
    int tmem_cols;
    float scale;
    int mode;              // 0: store scale * v; 1: displacement (clamp, CFL / NaN flags)
    int *status;
    int probe;
    int parts;             // the P1 slab is fetched in `parts` slices of B2 / parts j2 rows
    int NC;                // fields: 3 per velocity (the steps' velocities of a
                           // non-stationary plan are transformed in one launch)
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

__global__ void __launch_bounds__(FZ_G_MAX * 128, 1)
k_fx(FxArgs p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023) & ~1023u) - raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = tid >> 7, gt = tid & 127, gw = warp & 3;
    const size_t tb2 = tile_bytes(FZ_M, p.K2e), tb3 = tile_bytes(p.N3e, p.K3e);
    const size_t tbB = tile_bytes(p.N2e, p.K2e), tbA = tile_bytes(FZ_M, p.K3e);
    uint8_t *sT2 = base;
    uint8_t *sT3 = sT2 + 2 * tb2;
    uint8_t *sG = sT3 + 2 * tb3;                    // G operand buffers
    uint8_t *buf = sG + (size_t)g * p.gbytes;       // this warpgroup's
    uint64_t *bars = reinterpret_cast<uint64_t *>(sG + (size_t)p.G * p.gbytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 + 2 * FZ_G_MAX);
    __shared__ int s_fail, s_table;
    __shared__ int s_ok[FZ_G_MAX], s_ld[FZ_G_MAX];
    const uint32_t bar_tab = smem_u32(&bars[0]), bar_probe = smem_u32(&bars[1]);
    const uint32_t bar_mma = smem_u32(&bars[2 + g]), bar_ld = smem_u32(&bars[2 + FZ_G_MAX + g]);
    const int mt = blockIdx.x % p.MT;   // the grid is a multiple of MT: one x2 tile per CTA
    const int jn = p.B2 / p.parts;                       // j2 rows of a slab slice
    const size_t p1_bytes = (size_t)jn * p.B3 * 8;
    const float2 *sP1 = reinterpret_cast<const float2 *>(buf + 2 * tbB);   // the slab slice

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(p.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(bar_tab, 1);
        mbar_init(bar_probe, 1);
        for (int q = 0; q < p.G; ++q) {
            mbar_init(smem_u32(&bars[2 + q]), 1);
            mbar_init(smem_u32(&bars[2 + FZ_G_MAX + q]), 1);
            s_ld[q] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_fail = 0;
        s_table = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    bool run = true;
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
    const uint32_t tg = tmem + (uint32_t)(g * p.gcols);   // this warpgroup's columns
    const int units = p.NC * p.N1;                       // per x2 tile
    const int lanes = (int)(gridDim.x / p.MT) * p.G;
    uint32_t phase = 0, ld_phase = 0;
    int flags = 0;
    for (int u = (int)(blockIdx.x / p.MT) * p.G + g; run && u < units; u += lanes) {
        const int c = u / p.N1, x1 = u - c * p.N1;
        // the unit's P1 slab (contiguous, B2 B3 complex) by bulk copies, one per
        // slice of jn j2 rows; each slice's chunks of the GEMM 2 B operand are
        // built before the next slice overwrites it
        bool ok = true;
        for (int part = 0; part < p.parts && ok; ++part) {
            const int jlo = part * jn;
            if (part > 0) {   // every thread has read the previous slice
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                group_sync(g);
            }
            if (gt == 0) {
                mbar_expect_arrive(bar_ld, (uint32_t)p1_bytes);
                bulk_g2s(smem_u32(sP1), p.P1 + ((long long)c * p.N1 + x1) * nb23 + (long long)jlo * p.B3,
                         (uint32_t)p1_bytes, bar_ld);
                s_ld[g] = 1 + (int)ld_phase;   // in flight, with the parity of its phase
            }
            ok = group_wait(g, gt, bar_ld, ld_phase, s_ok);
            ld_phase ^= 1u;
            if (!ok) break;
            if (gt == 0) s_ld[g] = 0;
            const float2 *src = sP1;
            // B operand of GEMM 2, [n = (re | im)(j3)][k = (C | S)(j2)]:
            //   (C, re) P1re  (C, im) P1im  (S, re) -P1im  (S, im) P1re
            // (the chunks of this slice's j2 rows; the zero padding with the last)
            const int nkc = p.K2e >> 3;
            for (int it = gt; it < p.N2e * nkc; it += 128) {
                const int n = it % p.N2e, kc = it / p.N2e;
                const int k0 = kc * 8;
                const int j2c = k0 < p.B2 ? k0 : (k0 < 2 * p.B2 ? k0 - p.B2 : -1);
                if ((j2c < 0 ? p.parts - 1 : j2c / jn) != part) continue;
                float x[8];
                const bool im = n >= p.B3;
                const int j3 = im ? n - p.B3 : n;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = k0 + q;
                    float v = 0.f;
                    if (n < 2 * p.B3 && k < 2 * p.B2) {
                        const bool sp = k >= p.B2;
                        const float2 w = src[((sp ? k - p.B2 : k) - jlo) * p.B3 + j3];
                        v = sp ? (im ? w.x : -w.y) : (im ? w.y : w.x);
                    }
                    x[q] = v;
                }
                store_chunk(buf, tbB, swz_chunk(n, kc, p.N2e), x);
            }
        }
        if (!ok) {
            if (gt == 0) s_fail = 1;
            break;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        group_sync(g);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (gt == 0) {
            mma_split(tg, smem_u32(sT2), smem_u32(sT2) + (uint32_t)tb2, FZ_M, smem_u32(buf),
                      smem_u32(buf) + (uint32_t)tbB, p.N2e, p.K2e, idesc2);
            mma_commit(bar_mma);
        }
        ok = group_wait(g, gt, bar_mma, phase, s_ok);
        phase ^= 1u;
        if (!ok) {
            if (gt == 0) s_fail = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // D2 rows (TMEM lane = x2 row) -> A operand of GEMM 3, [x2][k = (re | im)(j3)],
        // in the same buffer (GEMM 2 has read its B operand)
        {
            const int r = gw * 32 + lane;
            const uint32_t trow = tg + ((uint32_t)(gw * 32) << 16);
            for (int c0 = 0; c0 < p.N2e; c0 += 16) {
                uint32_t rv[16];
                tmem_ld16(trow + (uint32_t)c0, rv);
                store_chunk(buf, tbA, swz_chunk(r, c0 >> 3, FZ_M), reinterpret_cast<const float *>(rv));
                store_chunk(buf, tbA, swz_chunk(r, (c0 >> 3) + 1, FZ_M),
                            reinterpret_cast<const float *>(rv) + 8);
            }
            const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int kc = p.N2e >> 3; kc < (p.K3e >> 3); ++kc) store_chunk(buf, tbA, swz_chunk(r, kc, FZ_M), z);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        group_sync(g);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (gt == 0) {   // D3 overwrites the columns of D2, which have been read
            mma_split(tg, smem_u32(buf), smem_u32(buf) + (uint32_t)tbA, FZ_M, smem_u32(sT3),
                      smem_u32(sT3) + (uint32_t)tb3, p.N3e, p.K3e, idesc3);
            mma_commit(bar_mma);
        }
        ok = group_wait(g, gt, bar_mma, phase, s_ok);
        phase ^= 1u;
        if (!ok) {
            if (gt == 0) s_fail = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // epilogue: warp gw of the group stores x2 rows 32 gw .. of the tile, all
        // x3 columns in chunks of 32 (transposes in the group's buffer)
        {
            float *T = reinterpret_cast<float *>(buf) + gw * 1024;
            const int row0 = mt * FZ_M + gw * 32;
            float *dst = p.out + c * V + (long long)x1 * p.N2 * p.N3;
            const uint32_t tq = tg + ((uint32_t)(gw * 32) << 16);
            for (int c0 = 0; c0 < p.N3e; c0 += 32) {
                if (c0 + 32 <= p.N3e)
                    fz_epi_chunk<32>(tq + (uint32_t)c0, T, dst, row0, p.N2, p.N3, c0, p.N3, p.scale,
                                     p.mode, lane, flags);
                else
                    fz_epi_chunk<16>(tq + (uint32_t)c0, T, dst, row0, p.N2, p.N3, c0, p.N3, p.scale,
                                     p.mode, lane, flags);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        group_sync(g);
    }
    if (flags) atomicOr(p.status, flags);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (s_fail && tid == 0) {
        // a wait expired: give the copies still in flight a bounded time to land
        atomicOr(p.status, BLR_FLAG_TIMEOUT);
        if (s_table) mbar_wait(bar_tab, 0u);
        for (int q = 0; q < p.G; ++q)
            if (s_ld[q]) mbar_wait(smem_u32(&bars[2 + FZ_G_MAX + q]), (uint32_t)(s_ld[q] - 1));
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(p.tmem_cols));
}

// ---------------------------------------------------------------------------
// Project.  GEMM 3' is computed transposed, D3t[n][x2] = sum_x3 T3p[n][x3] f[x2][x3]
// (A = the table, B = the field tile, x3 in chunks of 64), so that tensor-memory
// lane n holds row n of the next GEMM's A operand Q3t[n][x2] without a transpose.
// Only the N3p meaningful rows of the table and of Q3t are stored: the MMA's rows
// N3p .. 127 read whatever follows in shared memory and land in accumulator rows
// that are never read.
struct FpArgs {
    const uint8_t *tab3;   // [hi|lo][N3p x K3p]  (A operand, N3p rows stored)
    const uint8_t *tab2;   // [MT][hi|lo][N2p x 128]
    const float *f;        // [3][N1][N2][N3]
    float2 *Q2;            // [3][N1][MT][B2 B3]
    int N1, N2, N3, B2, B3, MT;
    int K3p, N3p, N2p;
    int G;
    size_t gbytes;
    int gcols;
    int tmem_cols;
    int vec4;              // rows of f are 16-byte aligned (N3 % 4 == 0, aligned base)
    int *status;
    int probe;
    int NC;                // fields (3 per velocity)
};

constexpr int FP_KC = 64;   // x3 per field chunk (one 128-byte swizzle atom)

__global__ void __launch_bounds__(FZ_G_MAX * 128, 1)
k_fp(FpArgs p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023) & ~1023u) - raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = tid >> 7, gt = tid & 127, gw = warp & 3;
    const size_t tb3 = tile_bytes(p.N3p, p.K3p), tb2 = tile_bytes(p.N2p, FZ_M);
    const size_t tbF = tile_bytes(FZ_M, FP_KC), tbQ = tile_bytes(p.N3p, FZ_M);
    const size_t slack = (size_t)(FZ_M - p.N3p) * 128;   // rows read past N3p
    uint8_t *sT3 = base;
    uint8_t *sT2 = sT3 + 2 * tb3 + slack;
    uint8_t *sG = sT2 + 2 * tb2;
    uint8_t *buf = sG + (size_t)g * p.gbytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sG + (size_t)p.G * p.gbytes + slack);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 + FZ_G_MAX);
    __shared__ int s_fail, s_table;
    __shared__ int s_ok[FZ_G_MAX];
    const uint32_t bar_tab = smem_u32(&bars[0]), bar_probe = smem_u32(&bars[1]);
    const uint32_t bar_mma = smem_u32(&bars[2 + g]);
    const int mt = blockIdx.x % p.MT;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(p.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(bar_tab, 1);
        mbar_init(bar_probe, 1);
        for (int q = 0; q < p.G; ++q) mbar_init(smem_u32(&bars[2 + q]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_fail = 0;
        s_table = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    bool run = true;
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
    const uint32_t idesc3 = umma_idesc(FZ_M, FZ_M), idesc2 = umma_idesc(FZ_M, p.N2p);
    const long long V = (long long)p.N1 * p.N2 * p.N3;
    const int rows = min(FZ_M, p.N2 - mt * FZ_M);   // x2 rows of this CTA's tile
    const uint32_t tg = tmem + (uint32_t)(g * p.gcols);
    const int units = p.NC * p.N1;
    const int lanes = (int)(gridDim.x / p.MT) * p.G;
    const int nchunk = p.K3p / FP_KC;
    const int ep = p.N2p + 1;
    uint32_t phase = 0;
    for (int u = (int)(blockIdx.x / p.MT) * p.G + g; run && u < units; u += lanes) {
        const int c = u / p.N1, x1 = u - c * p.N1;
        const float *src = p.f + c * V + ((long long)x1 * p.N2 + (long long)mt * FZ_M) * p.N3;
        bool ok = true;
        // field chunks -> B operand of GEMM 3', [x2][k = x3 in the chunk].  Each
        // thread holds its 8 pieces of 8 values of one chunk in registers: the
        // next chunk's loads are issued before the wait for this chunk's MMAs.
        constexpr int PER = FZ_M * (FP_KC / 8) / 128;   // 8 per thread
        float x[PER][8];
        auto load_chunk = [&](int ch) {
#pragma unroll
            for (int s = 0; s < PER; ++s) {
                const int it = s * 128 + gt, r = it >> 3, kc = it & 7;
                const int k0 = ch * FP_KC + kc * 8;
                const bool live = r < rows;
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
        };
        load_chunk(0);
        for (int ch = 0; ch < nchunk && ok; ++ch) {
#pragma unroll
            for (int s = 0; s < PER; ++s) {
                const int it = s * 128 + gt;
                store_chunk(buf, tbF, swz_chunk(it >> 3, it & 7, FZ_M), x[s]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            group_sync(g);
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (ch + 1 < nchunk) load_chunk(ch + 1);
            if (gt == 0) {
                // A: atom ch of the table (N3p rows per atom), B: the field chunk
                const uint32_t a0 = smem_u32(sT3) + (uint32_t)(ch * p.N3p * 128);
                for (int j = 0; j < FP_KC / 16; ++j) {
                    const uint32_t o = (uint32_t)(j * 32);
                    const uint64_t ah = umma_desc(a0 + o), al = umma_desc(a0 + (uint32_t)tb3 + o);
                    const uint64_t bh = umma_desc(smem_u32(buf) + o), bl = umma_desc(smem_u32(buf) + (uint32_t)tbF + o);
                    umma_bf16(tg, ah, bh, idesc3, (ch > 0 || j > 0) ? 1u : 0u);
                    umma_bf16(tg, ah, bl, idesc3, 1u);
                    umma_bf16(tg, al, bh, idesc3, 1u);
                }
                mma_commit(bar_mma);
            }
            ok = group_wait(g, gt, bar_mma, phase, s_ok);
            phase ^= 1u;
        }
        if (!ok) {
            if (gt == 0) s_fail = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // D3t row n (TMEM lane n) -> A operand of GEMM 2', [n][k = x2 in tile]
        if (gw * 32 < p.N3p) {
            const int n = gw * 32 + lane;
            const uint32_t trow = tg + ((uint32_t)(gw * 32) << 16);
            for (int c0 = 0; c0 < FZ_M; c0 += 32) {
                uint32_t rv[32];
                tmem_ld32(trow + (uint32_t)c0, rv);
                if (n < p.N3p) {
#pragma unroll
                    for (int h = 0; h < 4; ++h)
                        store_chunk(buf, tbQ, swz_chunk(n, (c0 >> 3) + h, p.N3p),
                                    reinterpret_cast<const float *>(rv) + 8 * h);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        group_sync(g);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (gt == 0) {   // D2t overwrites the first columns of D3t, which have been read
            mma_split(tg, smem_u32(buf), smem_u32(buf) + (uint32_t)tbQ, p.N3p, smem_u32(sT2),
                      smem_u32(sT2) + (uint32_t)tb2, p.N2p, FZ_M, idesc2);
            mma_commit(bar_mma);
        }
        ok = group_wait(g, gt, bar_mma, phase, s_ok);
        phase ^= 1u;
        if (!ok) {
            if (gt == 0) s_fail = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // D2t rows m < 2 B3 -> FP32 staging [m][n] in the group's buffer (odd pitch:
        // column reads below)
        float *sE = reinterpret_cast<float *>(buf);
        if (gw * 32 < 2 * p.B3) {
            const int m = gw * 32 + lane;
            const uint32_t trow = tg + ((uint32_t)(gw * 32) << 16);
            for (int c0 = 0; c0 < p.N2p; c0 += 16) {
                uint32_t rv[16];
                tmem_ld16(trow + (uint32_t)c0, rv);
                if (m < 2 * p.B3) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) sE[(size_t)m * ep + c0 + q] = __uint_as_float(rv[q]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        group_sync(g);
        // Q2[j2][j3] = (C re + S im, C im - S re) combinations of the four blocks
        float2 *dst = p.Q2 + (((long long)c * p.N1 + x1) * p.MT + mt) * nb23;
        for (int e = gt; e < nb23; e += 128) {
            const int j2 = e / p.B3, j3 = e - j2 * p.B3;
            const float *re = sE + (size_t)j3 * ep, *im = sE + (size_t)(p.B3 + j3) * ep;
            dst[e] = make_float2(re[j2] + im[p.B2 + j2], im[j2] - re[p.B2 + j2]);
        }
        group_sync(g);
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

// Slices of the expand's P1 slab: 1 when the whole slab fits beside one
// warpgroup's operands, 2 (halves of j2, each a whole number of 8-column
// chunks) when only half does, 0 when neither fits.
int fx_parts(const FzGeom &g, int B2, int B3) {
    if (fx_shape(g, B2, B3, 0, 1).G >= 1) return 1;
    if (B2 % 16 == 0 && fx_shape(g, B2, B3, 0, 2).G >= 1) return 2;
    return 0;
}

// CTAs per x2 tile when every SM holds one CTA, and the warpgroups that spreads
// a tile's units over: units are (component, x1 plane), per x2 tile.
int fz_ctas_per_tile(const blr_plan *P, int MT) {
    const int sms = P->sms > 0 ? P->sms : 148;
    return sms / MT > 1 ? sms / MT : 1;
}
int fz_gmax(const blr_plan *P, int MT, int nc) {
    const int per = fz_ctas_per_tile(P, MT), units = nc * P->N1;
    return (units + per - 1) / per;
}
// Grid of a fused kernel: at most one CTA per SM, a multiple of MT, and no CTA
// without units.
int fz_grid(const blr_plan *P, int G, int MT, int nc) {
    int per = fz_ctas_per_tile(P, MT);
    const int need = (nc * P->N1 + G - 1) / G;
    if (per > need) per = need;
    return per * MT;
}

}  // namespace

extern std::atomic<int> g_tc_probe;   // dft_tc.cu (blr_test_expire_waits)

// ---------------------------------------------------------------------------
// host side

bool fz_supported(const blr_plan *P) {
    const FzGeom g = fz_geometry(P);
    if (P->N3 > 256 || P->B2 > 128 || 2 * P->B3 > FZ_M) return false;
    return fx_parts(g, P->B2, P->B3) >= 1 && fp_shape(g).G >= 1;
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
    return (size_t)2 * 3 * P->nvel * P->N1 * g.MT * P->B2 * P->B3;
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

int fz_expand(blr_plan *P, const float *vt, float *out, float scale, int mode, cudaStream_t s,
              int nc) {
    const FzGeom g = fz_geometry(P);
    const int nb23 = P->B2 * P->B3;
    float2 *P1 = reinterpret_cast<float2 *>(P->fz_buf);
    launch_pdl(k_ex1, dim3((unsigned)((nb23 + EX_TC - 1) / EX_TC), (unsigned)((P->N1 + EX_TX - 1) / EX_TX), (unsigned)nc),
               dim3(256), 0, s, reinterpret_cast<const float2 *>(vt), (const float *)P->W1, P1,
               P->N1, P->B1, nb23);
    BLR_CK_LAUNCH();
    const int parts = fx_parts(g, P->B2, P->B3);
    const FzShape sh = fx_shape(g, P->B2, P->B3, fz_gmax(P, g.MT, nc), parts);
    FxArgs a;
    a.parts = parts;
    a.NC = nc;
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
    a.G = sh.G;
    a.gbytes = sh.gbytes;
    a.gcols = sh.gcols;
    a.tmem_cols = sh.tmem_cols;
    a.scale = scale;
    a.mode = mode;
    a.status = P->dstatus;
    a.probe = g_tc_probe.load(std::memory_order_relaxed);
    BLR_CK(cudaFuncSetAttribute(k_fx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem));
    launch_pdl(k_fx, dim3(fz_grid(P, sh.G, g.MT, nc)), dim3(128 * sh.G), sh.smem, s, a);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

int fz_project(blr_plan *P, const float *f, float *ft, const float *vadd, float areg,
               cudaStream_t s, int nc) {
    const FzGeom g = fz_geometry(P);
    const int nb23 = P->B2 * P->B3;
    float2 *Q2 = reinterpret_cast<float2 *>(P->fz_buf);
    const FzShape sh = fp_shape(g, fz_gmax(P, g.MT, nc));
    FpArgs a;
    a.NC = nc;
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
    a.G = sh.G;
    a.gbytes = sh.gbytes;
    a.gcols = sh.gcols;
    a.tmem_cols = sh.tmem_cols;
    a.vec4 = (P->N3 % 4 == 0) && ((uintptr_t)f % 16 == 0);
    a.status = P->dstatus;
    a.probe = g_tc_probe.load(std::memory_order_relaxed);
    BLR_CK(cudaFuncSetAttribute(k_fp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem));
    launch_pdl(k_fp, dim3(fz_grid(P, sh.G, g.MT, nc)), dim3(128 * sh.G), sh.smem, s, a);
    BLR_CK_LAUNCH();
    launch_pdl(k_p1, dim3((unsigned)((nb23 + P1_TC - 1) / P1_TC), (unsigned)((P->B1 + P1_TJ - 1) / P1_TJ), (unsigned)nc),
               dim3(256), 0, s,
               (const float2 *)Q2, (const float *)P->W1, reinterpret_cast<float2 *>(ft),
               (const float *)P->A, reinterpret_cast<const float2 *>(vadd), areg, P->N1, P->B1,
               g.MT, nb23);
    BLR_CK_LAUNCH();
    return BLR_OK;
}
