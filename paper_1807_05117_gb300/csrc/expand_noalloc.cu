// blr_expand_noalloc: iota without a plan and without any device allocation.
//
// Some callers cannot allocate device memory themselves: a host framework that
// owns every device allocation through its own pool (so that its accounting
// stays exact and nothing else may call cudaMalloc), or a latency-critical loop
// in which cudaMalloc / cudaFree, which can synchronise the whole device, are
// not acceptable.  This entry point serves them: the DFT tables and the two
// intermediate arrays of the expand live in one fixed file-scope device array,
// reserved in every GPU that loads the library until the process exits.
//
// The kernels and launchers are the ones blr_expand uses (dft.cu); only the
// storage differs.
#include <cuda.h>

#include <mutex>

#include "blr_internal.cuh"

// 4 Mi floats = 16 MiB: enough for a 128^3 grid with a 32^3 band.
#define BLR_NOALLOC_SCRATCH_FLOATS (BLR_NOALLOC_SCRATCH_BYTES / 4u)

static __device__ __align__(256) float g_noalloc_scratch[BLR_NOALLOC_SCRATCH_FLOATS];

namespace {

constexpr int kMaxDevices = 256;

// Device address of g_noalloc_scratch per device ordinal, looked up once per
// device and context (host code may not use the symbol itself as a device
// pointer: in host code it names a host-side stand-in).  The context's unique
// id is kept beside it: after the device's primary context is torn down and
// re-created (cudaDeviceReset), the module is loaded again and the array may
// live elsewhere, so a new id repeats the look-up.
struct ScratchAddr {
    float *addr = nullptr;
    unsigned long long ctx = 0;
};
std::mutex g_scratch_mu;
ScratchAddr g_scratch_addr[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context, or 0 when no context is
// current or the driver offers no way to ask (the caller then looks the
// address up again).
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) ==
                cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) ==
                cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(a);
            get_id = reinterpret_cast<CtxGetIdFn>(b);
        }
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx &&
        get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

int scratch_on_current_device(float **out) {
    int dev = -1;
    BLR_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return BLR_EINVAL;
    // id 0: no context is current on this thread yet (or the driver cannot say);
    // the look-up below makes the device's primary context current
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchAddr &e = g_scratch_addr[dev];
    if (!e.addr || ctx == 0 || ctx != e.ctx) {
        void *addr = nullptr;
        if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) {
            cudaGetLastError();
            return BLR_ECUDA;
        }
        e.addr = static_cast<float *>(addr);
        e.ctx = current_context_id();
    }
    *out = e.addr;
    return BLR_OK;
}

size_t chunk(size_t floats) { return (floats + 63) & ~(size_t)63; }   // 256-byte pieces

}  // namespace

extern "C" int blr_expand_noalloc(const int n[3], const int band[3], const float *vt,
                                  float *v, blr_stream_t stream) {
    if (!n || !band || !vt || !v) return BLR_EINVAL;
    for (int d = 0; d < 3; ++d)
        if (n[d] < 1 || band[d] < 2 || (band[d] & 1) || band[d] > n[d]) return BLR_EINVAL;
    if (band[2] > 64) return BLR_EINVAL;
    const size_t N1 = n[0], N2 = n[1], N3 = n[2], B1 = band[0], B2 = band[1], B3 = band[2];
    const size_t need = chunk(2 * B1 * N1) + 2 * chunk(B2 * N2) + 2 * chunk(B3 * N3) +
                        chunk(B1 * B2 * B3) + chunk(6 * B1 * B2 * N3) + chunk(6 * B1 * N2 * N3);
    if (need > BLR_NOALLOC_SCRATCH_FLOATS) return BLR_EINVAL;
    float *base = nullptr;
    int rc = scratch_on_current_device(&base);
    if (rc) return rc;

    // A plan-shaped view of the scratch array for the shared launchers.  Every
    // element the launchers read is written earlier in the same call, so nothing
    // needs clearing and nothing carries over from the previous call.
    blr_plan P{};
    P.N1 = n[0];
    P.N2 = n[1];
    P.N3 = n[2];
    P.B1 = band[0];
    P.B2 = band[1];
    P.B3 = band[2];
    P.V = (long long)N1 * N2 * N3;
    P.nb = (long long)B1 * B2 * B3;
    P.nf1 = P.nfloat = 6 * P.nb;
    P.nvel = 1;
    P.p.alpha = 0.0;   // the regulariser table is filled but unused by iota
    P.p.gamma = 1.0;
    P.p.s = 0;
    P.dstatus = nullptr;   // only the displacement mode latches flags
    float *q = base;
    P.W1 = q;         q += chunk(2 * B1 * N1);
    P.T2c = q;        q += chunk(B2 * N2);
    P.T2s = q;        q += chunk(B2 * N2);
    P.T3c = q;        q += chunk(B3 * N3);
    P.T3s = q;        q += chunk(B3 * N3);
    P.A = q;          q += chunk(B1 * B2 * B3);
    P.dft_small = q;  q += chunk(6 * B1 * B2 * N3);
    P.dft_big = q;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = dft_init_tables(&P, s))) return rc;
    return dft_expand(&P, vt, v, 0, s);
}
