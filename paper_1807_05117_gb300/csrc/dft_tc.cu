// Mixed-precision axis-1 contractions of the truncated DFTs on tcgen05 tensor
// cores (BLR_MIXED): the two largest stages of iota and pi (Section 3.1, Eq. 33),
//   expand : v[c][x1][col]  = sum_kappa W1[kappa][x1] A2[c][kappa][col]
//   project: P1[c][kappa][col] = sum_x1  W1[kappa][x1] f[c][x1][col]
// with kappa = (k1, re|im) and col = (x2, x3).
//
// Both operands are split into BF16 hi + lo parts (x = hi + lo, lo = bf16(x - hi))
// and the product is accumulated in FP32 in tensor memory as
// Ah Bh + Ah Bl + Al Bh (the lo*lo term is below FP32 resolution).  The DFT table
// operand (A, 128-row M tiles, K-major, 128-byte swizzle) is built once per plan in
// FP64 and stored pre-swizzled; the field operand (B, N = columns of the tile) is
// read as FP32, split and transposed into the same K-major swizzled layout in
// shared memory by the CTA itself, so nothing extra goes through HBM.
// One elected thread issues the MMAs; completion is signalled through an mbarrier
// whose wait is bounded (timeout -> BLR_FLAG_TIMEOUT, TMEM freed, no output).
#include <cuda.h>
#include <string.h>
#include <cuda_bf16.h>

#include <atomic>

#include "blr_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_M = 128;


// An FP32 staging slot, rounded up to 1024 bytes so every slot (a TMA
// destination) and the swizzled tiles after them stay aligned.
__host__ __device__ inline size_t tp_stage_bytes(int K, int nt) {
    return ((size_t)K * nt * 4 + 1023) & ~(size_t)1023;
}
__host__ __device__ inline size_t tp_b_bytes(int Kpad, int nt) { return (size_t)nt * Kpad * 2; }

struct TcArgs {
    const uint8_t *tab;      // [mtiles][hi|lo][128 x Kpad] BF16, swizzled
    int mtiles, M;           // M tiles of 128 rows; rows written (< M)
    int K, Kpad;             // contraction length and its multiple of 64
    const float *X;          // field operand, per batch [K][ncols]
    long long xstride;       // batch stride of X (floats)
    float *D;                // output, per batch [M][ncols]
    long long dstride;
    long long ncols;
    int ntile;               // columns per tile (multiple of 32, <= 256)
    int col_tiles, tiles;    // column tiles per batch, tiles over the 3 batches
    int nstage;              // FP32 staging buffers (2: next tile prefetched)
    int bulk;                // rows may be fetched with cp.async.bulk (16-byte aligned)
    int tma;                 // tiles are fetched by one 2-D TMA copy (tensor map of X)
    int tmem_cols;           // power of two >= mtiles * ntile
    float scale;
    int mode;                // 0 store scale*acc; 1 displacement (clamp + flags)
    int *status;
    int probe;               // test hook (blr_test_expire_waits): a bounded wait that
                             // expires before anything is issued (k_tc_pipe)
};


// Persistent: each CTA loads the table once, then walks column tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ...; with two staging buffers the next
// tile's rows stream in (cp.async.bulk) while the current one is converted,
// multiplied and written.
__global__ void __launch_bounds__(TC_THREADS, 2)
k_tc_axis1(TcArgs p, const __grid_constant__ CUtensorMap xmap) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023) & ~1023u) - raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t tab_bytes = (size_t)TC_M * p.Kpad * 2;            // one hi or lo table tile
    const size_t all_tab = 2 * tab_bytes * p.mtiles;
    const size_t stage_bytes = tp_stage_bytes(p.K, p.ntile);      // 1024-byte aligned slots
    const size_t b_bytes = (size_t)p.ntile * p.Kpad * 2;           // one hi or lo field tile
    uint8_t *sA = base;
    float *stage0 = reinterpret_cast<float *>(sA + all_tab);
    uint8_t *sBh = reinterpret_cast<uint8_t *>(stage0) + p.nstage * stage_bytes;
    uint8_t *sBl = sBh + b_bytes;
    // epilogue transpose buffer, 8 warps x 32 x 32 floats: the staging buffer
    // itself when there is only one and it is large enough (tc_smem_bytes)
    const size_t epi_bytes = (size_t)TC_THREADS / 32 * 1024 * 4;
    const bool alias = p.nstage == 1 && stage_bytes >= epi_bytes;
    float *sE = alias ? stage0 : reinterpret_cast<float *>(sBl + b_bytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sBl + b_bytes + (alias ? 0 : epi_bytes));   // load[0], load[1], mma
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 3);
    __shared__ int s_fail;
    const uint32_t bar_load0 = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[2]);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(p.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(bar_load0, 1);
        mbar_init(bar_load0 + 8, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;

    // rows of tile t into staging buffer sb (warp 0; bulk path only)
    auto tile_cols = [&](int t, long long *col0, int *w, const float **src) {
        const int batch = t / p.col_tiles, ct = t - batch * p.col_tiles;
        *col0 = (long long)ct * p.ntile;
        const long long left = p.ncols - *col0;
        *w = (int)(left < p.ntile ? left : p.ntile);
        *src = p.X + batch * p.xstride + *col0;
    };
    auto issue_tile = [&](int t, int sb, uint32_t extra_bytes) {
        long long col0;
        int w;
        const float *src;
        tile_cols(t, &col0, &w, &src);
        const uint32_t bar = bar_load0 + 8u * sb;
        const uint32_t dst0 = smem_u32(stage0) + (uint32_t)(sb * stage_bytes);
        if (p.tma) {
            // the whole [K][ntile] box (columns past the end read as zeros)
            if (lane == 0) {
                mbar_expect_arrive(bar, (uint32_t)(p.K * p.ntile * 4) + extra_bytes);   // the box
                tma_load_2d(dst0, &xmap, (int)col0, (t / p.col_tiles) * p.K, bar);
            }
            __syncwarp();
            return;
        }
        const uint32_t row_bytes = (uint32_t)w * 4u;
        if (lane == 0) mbar_expect_arrive(bar, row_bytes * (uint32_t)p.K + extra_bytes);
        __syncwarp();
        for (int k = lane; k < p.K; k += 32)
            bulk_g2s(dst0 + (uint32_t)k * p.ntile * 4u, src + (long long)k * p.ncols, row_bytes, bar);
    };

    int first = blockIdx.x;
    // the table is written once at plan creation (which synchronises the device),
    // so it is fetched before the wait for the previous kernel in the stream
    // (programmatic dependent launch); the field tiles after
    if (warp == 0 && lane == 0) bulk_g2s(smem_u32(sA), p.tab, (uint32_t)all_tab, bar_load0);
    pdl_wait();
    if (warp == 0) {
        if (p.bulk && first < p.tiles) {
            issue_tile(first, 0, (uint32_t)all_tab);   // arms bar_load0 for table + tile
        } else {
            if (lane == 0) mbar_expect_arrive(bar_load0, (uint32_t)all_tab);
            __syncwarp();
        }
    }

    const uint32_t idesc = umma_idesc(TC_M, p.ntile);
    uint32_t pend_bar = 0, pend_par = 0;   // prefetch issued this iteration
    uint32_t own_bar = 0, own_par = 0;     // load whose wait expired
    int i = 0;
    for (int t = first; t < p.tiles; t += gridDim.x, ++i) {
        const int sb = (p.nstage == 2) ? (i & 1) : 0;
        const int nxt = t + gridDim.x;
        long long col0;
        int w;
        const float *src;
        tile_cols(t, &col0, &w, &src);
        float *stage = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(stage0) + sb * stage_bytes);
        bool ok = true;
        if (p.bulk) {
            if (p.nstage == 2) {
                if (nxt < p.tiles) {
                    if (warp == 0) issue_tile(nxt, sb ^ 1, 0u);
                    pend_bar = bar_load0 + 8u * (sb ^ 1);
                    pend_par = (uint32_t)((i + 1) >> 1) & 1u;
                } else {
                    pend_bar = 0;
                }
            } else if (i > 0 && warp == 0) {
                issue_tile(t, 0, 0u);   // the only buffer is free again
            }
            const uint32_t use = (p.nstage == 2) ? (uint32_t)(i >> 1) : (uint32_t)i;
            // one thread waits; the barrier below releases the others (no
            // polling warps competing for issue slots)
            ok = tid == 0 ? mbar_wait(bar_load0 + 8u * sb, use & 1u) : true;
            if (!ok) {
                own_bar = bar_load0 + 8u * sb;
                own_par = use & 1u;
            }
        } else {
            if (i == 0 && tid == 0) ok = mbar_wait(bar_load0, 0u);   // table
            for (int e = tid; e < p.K * p.ntile; e += TC_THREADS) {
                const int k = e / p.ntile, r = e - k * p.ntile;
                stage[e] = r < w ? __ldg(src + (long long)k * p.ncols + r) : 0.f;
            }
            __syncthreads();
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) s_fail = 1;
            break;
        }
        // FP32 staging [K][ntile] -> BF16 hi / lo, K-major swizzled [ntile][Kpad]
        const int nkc = p.Kpad >> 3;
        for (int it = tid; it < p.ntile * nkc; it += TC_THREADS) {
            const int r = it % p.ntile, kc = it / p.ntile;
            float x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = kc * 8 + q;
                x[q] = (k < p.K && r < w) ? stage[k * p.ntile + r] : 0.f;
            }
            uint4 hi, lo;
            split8(x, hi, lo);
            const uint32_t off = swz_chunk(r, kc, p.ntile);
            *reinterpret_cast<uint4 *>(sBh + off) = hi;
            *reinterpret_cast<uint4 *>(sBl + off) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t bh0 = smem_u32(sBh), bl0 = smem_u32(sBl);
            for (int mt = 0; mt < p.mtiles; ++mt) {
                const uint32_t ah0 = smem_u32(sA + (size_t)(2 * mt) * tab_bytes);
                const uint32_t al0 = ah0 + (uint32_t)tab_bytes;
                const uint32_t d = tmem + (uint32_t)(mt * p.ntile);
                for (int j = 0; j < p.Kpad / 16; ++j) {
                    // K step of 16 elements: atom column j/4, 32 bytes per step inside it
                    const uint32_t oa = (uint32_t)((j >> 2) * TC_M * 128 + (j & 3) * 32);
                    const uint32_t ob = (uint32_t)((j >> 2) * p.ntile * 128 + (j & 3) * 32);
                    const uint64_t ah = umma_desc(ah0 + oa), al = umma_desc(al0 + oa);
                    const uint64_t bh = umma_desc(bh0 + ob), bl = umma_desc(bl0 + ob);
                    umma_bf16(d, ah, bh, idesc, j > 0);
                    umma_bf16(d, ah, bl, idesc, 1u);
                    umma_bf16(d, al, bh, idesc, 1u);
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    bar_mma));
        }
        ok = tid == 0 ? mbar_wait(bar_mma, (uint32_t)(i & 1)) : true;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) s_fail = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // epilogue: warp w reads TMEM lanes 32*(w%4).. (rows), columns of half w/4,
        // 32 x 32 blocks transposed through an XOR-swizzled buffer so that each
        // store instruction writes 128 contiguous bytes of one output row
        float *D = p.D + (t / p.col_tiles) * p.dstride;
        // 32-column chunks alternate between the two warp halves, so no load
        // reaches past the tile's own TMEM columns (ntile may be 32)
        const int lg = warp & 3, half = warp >> 2;
        float *T = sE + warp * 1024;
        int flags = 0;
        for (int mt = 0; mt < p.mtiles; ++mt) {
            const int row0 = mt * TC_M + lg * 32;
            for (int c = half * 32; c < p.ntile; c += 64) {
                uint32_t rv[32];
                tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(mt * p.ntile + c), rv);
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    float v = __uint_as_float(rv[q]) * p.scale;
                    if (p.mode == 1) {
                        const bool valid = (row0 + lane < p.M) && (c + q < w);
                        if (valid && !(fabsf(v) < 1.f)) flags |= (v != v) ? BLR_FLAG_NAN : BLR_FLAG_CFL;
                        v = fminf(fmaxf(v, -1.f), 0.99999994f);
                    }
                    T[lane * 32 + (q ^ lane)] = v;
                }
                __syncwarp();
                const bool col_ok = (c + lane) < w;
                for (int q = 0; q < 32; ++q) {
                    const int row = row0 + q;
                    if (row < p.M && col_ok)
                        D[(long long)row * p.ncols + col0 + c + lane] = T[q * 32 + (lane ^ q)];
                }
                __syncwarp();
            }
        }
        if (flags) atomicOr(p.status, flags);
        // the epilogue's generic writes may share the staging buffer with the
        // next tile's asynchronous load
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    if (s_fail) {
        // a wait expired: record it, give this CTA's outstanding bulk copies a
        // bounded time to land, then release TMEM
        if (tid == 0) atomicOr(p.status, BLR_FLAG_TIMEOUT);
        if (own_bar) mbar_wait(own_bar, own_par);
        if (pend_bar) mbar_wait(pend_bar, pend_par);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(p.tmem_cols));
}

// ---------------------------------------------------------------------------
// Pipelined, warp-specialised form of the same contraction.  Per CTA, tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ... flow through double-buffered
// stages, each hand-off on an mbarrier:
//   warps 0-5 (192 threads): split the FP32 tile into BF16 hi / lo (swizzled
//     K-major B operand); thread 0 also issues the TMA loads, two tiles ahead;
//   warp 14, lane 0: issues the MMAs of a tile into one of two TMEM
//     accumulators and commits them to the "B free" and "accumulator full"
//     barriers;
//   warps 6-13 (two per TMEM lane quadrant, each half of the 32-column
//     chunks): epilogue, TMEM -> registers -> XOR-swizzled shared transpose ->
//     coalesced global stores.
// Each role is a chain of dependent loads, so it gets several warps per
// scheduler to hide their latency.
// So the split of tile i + 1, the MMAs of tile i and the epilogue of tile i - 1
// overlap.  Slot s = i & 1 of every buffer is used by tiles i = s, s + 2, ...; the
// u-th use (u = i >> 1) of a "full" barrier completes phase u, and a "free"
// barrier's phase u - 1 must complete before slot s is refilled.  Every wait is
// bounded: a wait that expires stops its role, the CTA waits (bounded) for its
// copies in flight, frees TMEM and sets BLR_FLAG_TIMEOUT.
constexpr int TP_CONV = 6, TP_EPI = 8;                  // converter / epilogue warps
constexpr int TP_MMA_WARP = TP_CONV + TP_EPI;          // warp 14
constexpr int TP_THREADS = (TP_MMA_WARP + 1) * 32;     // 480
constexpr int TP_CT = TP_CONV * 32;                    // converter threads
constexpr int TP_NBAR = 14;   // the last one: the test hook's, never arrived at


// Shared memory of the pipelined kernel (tc_pipe_smem on the host).

// Epilogue of one CW-column chunk of a 32-row group: TMEM -> registers (scale,
// and for the displacement clamp + flags) -> XOR-swizzled transpose -> stores of
// 128 contiguous bytes per row.
template <int CW>
__device__ __forceinline__ void tp_epi_chunk(uint32_t ta, float *T, float *D, const TcArgs &p,
                                             int row0, long long col0, int c, int w, int lane,
                                             int &flags) {
    uint32_t rv[CW];
    if constexpr (CW == 32) tmem_ld32(ta, rv);
    else tmem_ld16(ta, rv);
#pragma unroll
    for (int q = 0; q < CW; ++q) {
        float v = __uint_as_float(rv[q]) * p.scale;
        if (p.mode == 1) {
            const bool valid = (row0 + lane < p.M) && (c + q < w);
            if (valid && !(fabsf(v) < 1.f)) flags |= (v != v) ? BLR_FLAG_NAN : BLR_FLAG_CFL;
            v = fminf(fmaxf(v, -1.f), 0.99999994f);
        }
        T[lane * 32 + (q ^ lane)] = v;
    }
    __syncwarp();
    const bool col_ok = lane < CW && (c + lane) < w;
#pragma unroll 8
    for (int q = 0; q < 32; ++q) {
        const int row = row0 + q;
        if (row < p.M && col_ok) D[(long long)row * p.ncols + col0 + c + lane] = T[q * 32 + (lane ^ q)];
    }
    __syncwarp();
}

__global__ void __launch_bounds__(TP_THREADS, 1)
k_tc_pipe(TcArgs p, const __grid_constant__ CUtensorMap xmap) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023) & ~1023u) - raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t tab_bytes = (size_t)TC_M * p.Kpad * 2;       // one hi or lo table tile
    const size_t all_tab = 2 * tab_bytes * p.mtiles;
    const size_t stage_bytes = tp_stage_bytes(p.K, p.ntile);
    const size_t b_bytes = tp_b_bytes(p.Kpad, p.ntile);        // one hi or lo field tile
    uint8_t *sA = base;
    uint8_t *sStage = sA + all_tab;                            // [2][K][ntile] FP32
    uint8_t *sB = sStage + 2 * stage_bytes;                    // [2][hi|lo][ntile x Kpad]
    float *sE = reinterpret_cast<float *>(sB + 4 * b_bytes);   // [4 warps][32 x 32]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sE + TP_EPI * 1024);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + TP_NBAR);
    __shared__ int s_fail, s_issued, s_table;
    const uint32_t b0 = smem_u32(bars);
    // barriers: 0 table; 1+s stage full; 3+s stage free; 5+s B full; 7+s B free;
    // 9+s accumulator full; 11+s accumulator free; 13 test hook
    auto BAR = [&](int i) { return b0 + 8u * (uint32_t)i; };
    const int acc_cols = p.mtiles * p.ntile;
    int n = 0;   // tiles of this CTA
    for (int t = blockIdx.x; t < p.tiles; t += gridDim.x) ++n;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(p.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(BAR(0), 1);
        for (int sl = 0; sl < 2; ++sl) {
            mbar_init(BAR(1 + sl), 1);
            mbar_init(BAR(3 + sl), TP_CT);
            mbar_init(BAR(5 + sl), TP_CT);
            mbar_init(BAR(7 + sl), 1);
            mbar_init(BAR(9 + sl), 1);
            mbar_init(BAR(11 + sl), TP_EPI * 32);
        }
        mbar_init(BAR(13), 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_fail = 0;
        s_issued = 0;
        s_table = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    // Test hook: a bounded wait on a barrier nothing arrives at, taken while no
    // copy and no MMA has been issued, so that its expiry leaves nothing in flight.
    // The CTA then takes the timeout path below (no roles run, TMEM freed).
    if (p.probe) {
        const bool expired = tid == 0 ? !mbar_wait(BAR(13), 0u, TC_PROBE_CYCLES) : false;
        if (__syncthreads_or(expired)) n = 0;
        if (tid == 0 && expired) s_fail = 1;
    }
    // the table is written once at plan creation (which synchronises the device),
    // so it is fetched before the wait for the previous kernel in the stream
    if (tid == 0 && n > 0) {
        mbar_expect_arrive(BAR(0), (uint32_t)all_tab);
        bulk_g2s(smem_u32(sA), p.tab, (uint32_t)all_tab, BAR(0));
        s_table = 1;
    }
    pdl_wait();

    auto tile_of = [&](int i) { return blockIdx.x + i * gridDim.x; };
    auto issue = [&](int i) {   // thread 0: TMA load of tile i into slot i & 1
        const int t = tile_of(i), sl = i & 1;
        const int batch = t / p.col_tiles, ct = t - batch * p.col_tiles;
        mbar_expect_arrive(BAR(1 + sl), (uint32_t)(p.K * p.ntile * 4));   // the box
        tma_load_2d(smem_u32(sStage) + (uint32_t)(sl * stage_bytes), &xmap, ct * p.ntile,
                    batch * p.K, BAR(1 + sl));
        s_issued = i + 1;
    };
    bool ok = true;
    if (warp < TP_CONV) {
        // ---- split FP32 -> BF16 hi / lo (and the TMA producer in thread 0)
        if (tid == 0)
            for (int i = 0; i < n && i < 2; ++i) issue(i);
        const int nkc = p.Kpad >> 3;
        for (int i = 0; i < n && ok; ++i) {
            const int sl = i & 1;
            const uint32_t u = (uint32_t)(i >> 1);
            ok = mbar_wait(BAR(1 + sl), u & 1u);
            if (ok && i >= 2) ok = mbar_wait(BAR(7 + sl), (u - 1) & 1u);
            if (!ok) break;
            const int t = tile_of(i), ct = t % p.col_tiles;
            const long long left = p.ncols - (long long)ct * p.ntile;
            const int w = (int)(left < p.ntile ? left : p.ntile);
            const float *stage = reinterpret_cast<const float *>(sStage + sl * stage_bytes);
            uint8_t *sBh = sB + (size_t)(2 * sl) * b_bytes, *sBl = sBh + b_bytes;
            for (int it = tid; it < p.ntile * nkc; it += TP_CT) {
                const int r = it % p.ntile, kc = it / p.ntile;
                float x[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = kc * 8 + q;
                    x[q] = (k < p.K && r < w) ? stage[k * p.ntile + r] : 0.f;
                }
                uint4 hi, lo;
                split8(x, hi, lo);
                const uint32_t off = swz_chunk(r, kc, p.ntile);
                *reinterpret_cast<uint4 *>(sBh + off) = hi;
                *reinterpret_cast<uint4 *>(sBl + off) = lo;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(BAR(5 + sl));   // B full
            mbar_arrive(BAR(3 + sl));   // stage free
            if (tid == 0 && i + 2 < n) {
                ok = mbar_wait(BAR(3 + sl), u & 1u);   // every converter has read the stage
                if (ok) issue(i + 2);
            }
        }
    } else if (warp < TP_MMA_WARP) {
        // ---- epilogue: warp w reaches TMEM lanes 32 * (w % 4) .. + 31 (rows of the
        // tile); the two warps of a quadrant take alternate 32-column chunks
        const int lg = warp & 3;
        const int half = ((warp - TP_CONV) >> 2) & 1;
        float *T = sE + (warp - TP_CONV) * 1024;
        const int cw = p.ntile < 32 ? 16 : 32;
        int flags = 0;
        for (int i = 0; i < n && ok; ++i) {
            const int sl = i & 1;
            const uint32_t u = (uint32_t)(i >> 1);
            ok = mbar_wait(BAR(9 + sl), u & 1u);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int t = tile_of(i), batch = t / p.col_tiles, ct = t - batch * p.col_tiles;
            const long long col0 = (long long)ct * p.ntile;
            const long long left = p.ncols - col0;
            const int w = (int)(left < p.ntile ? left : p.ntile);
            float *D = p.D + batch * p.dstride;
            for (int mt = 0; mt < p.mtiles; ++mt) {
                const int row0 = mt * TC_M + lg * 32;
                for (int c = half * cw; c < p.ntile; c += 2 * cw) {
                    const uint32_t ta = tmem + ((uint32_t)(lg * 32) << 16) +
                                        (uint32_t)(sl * acc_cols + mt * p.ntile + c);
                    if (cw == 32)
                        tp_epi_chunk<32>(ta, T, D, p, row0, col0, c, w, lane, flags);
                    else
                        tp_epi_chunk<16>(ta, T, D, p, row0, col0, c, w, lane, flags);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(BAR(11 + sl));   // accumulator free
        }
        if (flags) atomicOr(p.status, flags);
    } else if (lane == 0 && n > 0) {
        // ---- MMA issue
        const uint32_t idesc = umma_idesc(TC_M, p.ntile);
        ok = mbar_wait(BAR(0), 0u);   // table
        for (int i = 0; i < n && ok; ++i) {
            const int sl = i & 1;
            const uint32_t u = (uint32_t)(i >> 1);
            ok = mbar_wait(BAR(5 + sl), u & 1u);
            if (ok && i >= 2) ok = mbar_wait(BAR(11 + sl), (u - 1) & 1u);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t bh0 = smem_u32(sB + (size_t)(2 * sl) * b_bytes);
            const uint32_t bl0 = bh0 + (uint32_t)b_bytes;
            for (int mt = 0; mt < p.mtiles; ++mt) {
                const uint32_t ah0 = smem_u32(sA + (size_t)(2 * mt) * tab_bytes);
                const uint32_t al0 = ah0 + (uint32_t)tab_bytes;
                const uint32_t d = tmem + (uint32_t)(sl * acc_cols + mt * p.ntile);
                for (int j = 0; j < p.Kpad / 16; ++j) {
                    const uint32_t oa = (uint32_t)((j >> 2) * TC_M * 128 + (j & 3) * 32);
                    const uint32_t ob = (uint32_t)((j >> 2) * p.ntile * 128 + (j & 3) * 32);
                    const uint64_t ah = umma_desc(ah0 + oa), al = umma_desc(al0 + oa);
                    const uint64_t bh = umma_desc(bh0 + ob), bl = umma_desc(bl0 + ob);
                    umma_bf16(d, ah, bh, idesc, j > 0);
                    umma_bf16(d, ah, bl, idesc, 1u);
                    umma_bf16(d, al, bh, idesc, 1u);
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    BAR(7 + sl)));   // B free
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    BAR(9 + sl)));   // accumulator full
        }
    }
    if (!ok) s_fail = 1;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (s_fail && tid == 0) {
        // a wait expired: record it and give every TMA load issued a bounded
        // time to land before the CTA leaves
        atomicOr(p.status, BLR_FLAG_TIMEOUT);
        for (int i = 0; i < s_issued; ++i) mbar_wait(BAR(1 + (i & 1)), (uint32_t)(i >> 1) & 1u);
        if (s_table) mbar_wait(BAR(0), 0u);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(p.tmem_cols));
}

// Table tiles, FP64 phases split into BF16 hi/lo, for stage kind
//   0 axis-1 expand : row x1, k kappa = 2 j + re/im       W = cos | -sin (2 pi k_j x1 / N)
//   1 axis-1 project: row kappa, k x1                       (the same values)
//   2 axis-2 expand : row (ro, x2), k (ri, j)   [[C, -S], [S, C]], C, S = cos, sin(2 pi k_j x2 / N)
//   3 axis-2 project: row (ro, j), k (ri, x2)   [[C,  S], [-S, C]]
// with k_j = j - B/2; the real and imaginary blocks are the real form of the
// complex sums of Eq. 33 along one axis (3: its transpose, conjugated).
__global__ void k_tc_table(uint8_t *tab, int mtiles, int M, int K, int Kpad, int N, int B,
                           int kind) {
    const long long total = (long long)mtiles * TC_M * Kpad;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % Kpad);
        const int rr = (int)((e / Kpad) % TC_M);
        const int mt = (int)(e / ((long long)Kpad * TC_M));
        const int row = mt * TC_M + rr;
        double w = 0.0;
        if (row < M && k < K) {
            int j, x, ro, ri;
            if (kind <= 1) {
                const int kappa = kind ? row : k;
                x = kind ? k : row;
                j = kappa >> 1;
                ri = kappa & 1;
                ro = 0;
            } else if (kind == 2) {
                ro = row / N;
                x = row - ro * N;
                ri = k / B;
                j = k - ri * B;
            } else {
                ro = row / B;
                j = row - ro * B;
                ri = k / N;
                x = k - ri * N;
            }
            long long ph = ((long long)(j - B / 2) * x) % N;
            if (ph < 0) ph += N;
            double sn, cs;
            sincospi(2.0 * (double)ph / (double)N, &sn, &cs);
            if (kind <= 1) w = ri ? -sn : cs;
            else if (ro == ri) w = cs;
            else if (kind == 2) w = ro ? sn : -sn;
            else w = ro ? -sn : sn;
        }
        const __nv_bfloat16 h = __double2bfloat16(w);
        const __nv_bfloat16 l = __double2bfloat16(w - (double)__bfloat162float(h));
        const size_t tile = (size_t)TC_M * Kpad * 2;
        uint8_t *hi = tab + (size_t)(2 * mt) * tile, *lo = hi + tile;
        const uint32_t off = swz_chunk(rr, k >> 3, TC_M) + (uint32_t)((k & 7) * 2);
        *reinterpret_cast<__nv_bfloat16 *>(hi + off) = h;
        *reinterpret_cast<__nv_bfloat16 *>(lo + off) = l;
    }
}

// cuTensorMapEncodeTiled from the driver (through the runtime, so the library
// needs no link against libcuda); nullptr when no driver is present.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
        else
            cudaGetLastError();
    }
    return fn;
}

int pow2_at_least(int v) {
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}

// Largest dynamic shared memory of a block (227 KB); tc_smem_bytes includes the
// 1024-byte alignment slack.
constexpr size_t TC_SMEM_MAX = 227 * 1024;

// With one staging buffer the epilogue's transpose buffer aliases it (the
// staging data are consumed before the MMAs, and the next tile's load is issued
// only after the epilogue), so it costs nothing extra when it fits there.
size_t tc_smem_bytes(int mtiles, int K, int Kpad, int nt, int nstage) {
    const size_t stage = (size_t)nstage * tp_stage_bytes(K, nt), epi = (size_t)TC_THREADS / 32 * 1024 * 4;
    const bool alias = nstage == 1 && stage >= epi;
    return 1024 + 2 * (size_t)TC_M * Kpad * 2 * mtiles + stage + 2 * (size_t)nt * Kpad * 2 +
           (alias ? 0 : epi) + 3 * 8 + 16;
}

// Blocks of this kernel that fit on one SM with `smem` bytes of dynamic shared
// memory and `cols` TMEM columns each (registers allow two).
constexpr size_t TC_SMEM_SM = 228 * 1024, TC_SMEM_RESERVED = 1024;
int tc_ctas_per_sm(size_t smem, int cols) {
    return (2 * (smem + TC_SMEM_RESERVED) <= TC_SMEM_SM && 2 * cols <= 512) ? 2 : 1;
}

// Column tile (256 .. 32) and staging depth: two staging buffers (the next
// tile's load overlaps the current tile's work) before one, then the largest
// tile that fits and still gives every SM a tile (else the largest that fits).
// A shape whose shared memory and TMEM allow two blocks per SM gets a grid of
// two blocks per SM (tc_run).
bool tc_shape(int mtiles, int K, int Kpad, long long ncols, int nbatch, int sms, int *ntile,
              int *nstage, size_t *smem) {
    for (int pass = 0; pass < 2; ++pass)
        for (int ns = 2; ns >= 1; --ns)
            for (int nt = 256; nt >= 32; nt >>= 1) {
                if (mtiles * nt > 512) continue;
                const size_t sb = tc_smem_bytes(mtiles, K, Kpad, nt, ns);
                if (sb > TC_SMEM_MAX) continue;
                const long long tiles = ceil_div_ll(ncols, nt) * nbatch;
                if (pass == 0 && tiles < sms) continue;
                *ntile = nt;
                *nstage = ns;
                *smem = sb;
                return true;
            }
    return false;
}

// Shared memory of the pipelined kernel: table, two FP32 stages, two hi/lo B
// tiles, the epilogue buffers and the barriers (+ 1024 bytes of alignment slack).
size_t tc_pipe_smem(int mtiles, int K, int Kpad, int nt) {
    return 1024 + 2 * (size_t)TC_M * Kpad * 2 * mtiles + 2 * tp_stage_bytes(K, nt) +
           4 * tp_b_bytes(Kpad, nt) + (size_t)TP_EPI * 1024 * 4 + TP_NBAR * 8 + 16;
}

// Column tile of the pipelined kernel (256 .. 16): the largest that fits with
// at least two tiles per SM (so the stages of consecutive tiles overlap), else
// one per SM, else any.  The field tile must be TMA-addressable (K <= 256 and
// no wider than the field).
bool tc_pipe_shape(int mtiles, int K, int Kpad, long long ncols, int nbatch, int sms, int *ntile,
                   size_t *smem) {
    if (K > 256) return false;
    for (int pass = 0; pass < 3; ++pass)
        for (int nt = 256; nt >= 16; nt >>= 1) {
            if (2 * mtiles * nt > 512 || nt > ncols) continue;
            const size_t sb = tc_pipe_smem(mtiles, K, Kpad, nt);
            if (sb > TC_SMEM_MAX) continue;
            const long long tiles = ceil_div_ll(ncols, nt) * nbatch;
            if (pass == 0 && tiles < 2LL * sms) continue;
            if (pass == 1 && tiles < sms) continue;
            *ntile = nt;
            *smem = sb;
            return true;
        }
    return false;
}

struct TcGeom {
    int mtiles, M, K, Kpad, nbatch, N, B;
    long long ncols;
};

// Geometry of tensor-core stage `kind` (see k_tc_table) of a plan.
TcGeom tc_geometry(const blr_plan *P, int kind) {
    TcGeom g;
    if (kind <= 1) {
        g.M = kind ? 2 * P->B1 : P->N1;
        g.K = kind ? P->N1 : 2 * P->B1;
        g.ncols = (long long)P->N2 * P->N3;
        g.nbatch = 3;
        g.N = P->N1;
        g.B = P->B1;
    } else {
        g.M = kind == 3 ? 2 * P->B2 : 2 * P->N2;
        g.K = kind == 3 ? 2 * P->N2 : 2 * P->B2;
        g.ncols = P->N3;
        g.nbatch = 3 * P->B1;
        g.N = P->N2;
        g.B = P->B2;
    }
    g.mtiles = (g.M + TC_M - 1) / TC_M;
    g.Kpad = (g.K + 63) / 64 * 64;
    return g;
}

int plan_sms(const blr_plan *P) { return P->sms > 0 ? P->sms : 148; }

bool tc_kind_ok(const blr_plan *P, int kind) {
    const TcGeom g = tc_geometry(P, kind);
    int nt, ns;
    size_t sm;
    return tc_shape(g.mtiles, g.K, g.Kpad, g.ncols, g.nbatch, plan_sms(P), &nt, &ns, &sm);
}

}  // namespace

// blr_test_expire_waits: the tensor-core kernels' test hook (k_tc_pipe here, k_fx
// and k_fp in dft_fused.cu), for every launch while set.
std::atomic<int> g_tc_probe{0};

size_t tc_table_bytes(const blr_plan *P, int kind) {
    const TcGeom g = tc_geometry(P, kind);
    return (size_t)g.mtiles * 2 * TC_M * g.Kpad * 2;
}

// Whether the mixed path supports this plan's shapes (the axis-1 stages).
bool tc_supported(const blr_plan *P) { return tc_kind_ok(P, 0) && tc_kind_ok(P, 1); }

// Whether the axis-2 stages also run on tensor cores: their whole table must fit
// in shared memory and the field tiles must be TMA-addressable (N3 % 4 == 0).
bool tc_axis2_supported(const blr_plan *P) {
    return P->N3 % 4 == 0 && 2 * P->N2 <= 256 && tc_kind_ok(P, 2) && tc_kind_ok(P, 3);
}

int tc_init_tables(blr_plan *P, cudaStream_t s) {
    uint8_t *tabs[4] = {P->tc_tab_expand, P->tc_tab_project, P->tc_tab2_expand, P->tc_tab2_project};
    for (int kind = 0; kind < 4; ++kind) {
        if (!tabs[kind]) continue;
        const TcGeom g = tc_geometry(P, kind);
        k_tc_table<<<256, 256, 0, s>>>(tabs[kind], g.mtiles, g.M, g.K, g.Kpad, g.N, g.B, kind);
        BLR_CK_LAUNCH();
    }
    return BLR_OK;
}

namespace {

// D[b] = W (x) X[b] for every batch b of stage `kind` on tensor cores; see TcArgs.
int tc_run(blr_plan *P, int kind, const float *X, float *D, float scale, int mode, cudaStream_t s) {
    const TcGeom g = tc_geometry(P, kind);
    TcArgs a;
    a.mtiles = g.mtiles;
    a.M = g.M;
    a.K = g.K;
    a.Kpad = g.Kpad;
    size_t smem = 0;
    const int sms = plan_sms(P);
    // the pipelined kernel when its shape fits and the field tiles can come by TMA
    // (checked below), else the sequential one
    const bool aligned = (g.ncols % 4 == 0) && ((uintptr_t)X % 16 == 0);
    bool pipe = aligned && encode_tiled() &&
                tc_pipe_shape(a.mtiles, a.K, a.Kpad, g.ncols, g.nbatch, sms, &a.ntile, &smem);
    if (pipe) a.nstage = 2;
    else if (!tc_shape(a.mtiles, a.K, a.Kpad, g.ncols, g.nbatch, sms, &a.ntile, &a.nstage, &smem))
        return BLR_EINVAL;
    uint8_t *tabs[4] = {P->tc_tab_expand, P->tc_tab_project, P->tc_tab2_expand, P->tc_tab2_project};
    a.tab = tabs[kind];
    if (!a.tab) return BLR_EINVAL;
    a.ncols = g.ncols;
    a.X = X;
    a.xstride = (long long)a.K * a.ncols;
    a.D = D;
    a.dstride = (long long)a.M * a.ncols;
    a.col_tiles = (int)ceil_div_ll(a.ncols, a.ntile);
    a.tiles = g.nbatch * a.col_tiles;
    // bulk row copies need 16-byte aligned rows and sizes
    a.bulk = (a.ncols % 4 == 0) && ((uintptr_t)X % 16 == 0);
    // one TMA box per tile: X as a 2-D tensor [nbatch K][ncols] (row stride a
    // 16-byte multiple), box [K][ntile] with K, ntile <= 256 and the box no wider
    // than the tensor
    CUtensorMap xmap;
    memset(&xmap, 0, sizeof(xmap));
    a.tma = 0;
    if (a.bulk && a.K <= 256 && a.ntile <= a.ncols) {
        EncodeTiledFn enc = encode_tiled();
        if (enc) {
            const cuuint64_t dims[2] = {(cuuint64_t)a.ncols, (cuuint64_t)g.nbatch * a.K};
            const cuuint64_t strides[1] = {(cuuint64_t)a.ncols * 4};
            const cuuint32_t box[2] = {(cuuint32_t)a.ntile, (cuuint32_t)a.K};
            const cuuint32_t estr[2] = {1, 1};
            if (enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(X), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
                a.tma = 1;
        }
    }
    if (pipe && !a.tma) {   // no tensor map after all: the sequential kernel
        pipe = false;
        if (!tc_shape(a.mtiles, a.K, a.Kpad, g.ncols, g.nbatch, sms, &a.ntile, &a.nstage, &smem))
            return BLR_EINVAL;
        a.col_tiles = (int)ceil_div_ll(a.ncols, a.ntile);
        a.tiles = g.nbatch * a.col_tiles;
    }
    a.scale = scale;
    a.mode = mode;
    a.status = P->dstatus;
    a.probe = g_tc_probe.load(std::memory_order_relaxed);
    if (pipe) {
        a.tmem_cols = pow2_at_least(2 * a.mtiles * a.ntile);
        BLR_CK(cudaFuncSetAttribute(k_tc_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int grid = a.tiles < sms ? a.tiles : sms;
        launch_pdl(k_tc_pipe, dim3(grid), dim3(TP_THREADS), smem, s, a, xmap);
        BLR_CK_LAUNCH();
        return BLR_OK;
    }
    a.tmem_cols = pow2_at_least(a.mtiles * a.ntile);
    BLR_CK(cudaFuncSetAttribute(k_tc_axis1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int slots = tc_ctas_per_sm(smem, a.tmem_cols) * sms;
    const int grid = a.tiles < slots ? a.tiles : slots;
    launch_pdl(k_tc_axis1, dim3(grid), dim3(TC_THREADS), smem, s, a, xmap);
    BLR_CK_LAUNCH();
    return BLR_OK;
}

}  // namespace

int tc_axis1(blr_plan *P, int project, const float *X, float *D, float scale, int mode,
             cudaStream_t s) {
    return tc_run(P, project ? 1 : 0, X, D, scale, mode, s);
}

int tc_axis2(blr_plan *P, int project, const float *X, float *D, cudaStream_t s) {
    return tc_run(P, project ? 3 : 2, X, D, 1.f, 0, s);
}

extern "C" int blr_test_expire_waits(int on) {
    g_tc_probe.store(on ? 1 : 0, std::memory_order_relaxed);
    return BLR_OK;
}
