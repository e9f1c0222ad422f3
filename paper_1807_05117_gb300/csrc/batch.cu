// Batching form: many independent registration pairs (each with its own grid,
// band and images, common number of time steps) advanced together.
//
// * Sweeps: one persistent launch per time step serves every pair; blocks pop
//   (pair, tile) items from an atomic work queue (k_sweep_batch in sweeps.cu).
// * DFT stages and PCG vector kernels are per pair, spread over side streams
//   (fork / join with events) so small pairs run concurrently.
// * One PCG iteration of all pairs (HVP, <p, Hp>, update, new direction) is
//   captured once as a CUDA graph and replayed; per-pair device flags freeze
//   pairs whose PCG has converged.
// * The x1 chunk of the sweep tiles is chosen by timing candidate shapes on the
//   batch itself (batch_autotune).
// Each pair's arithmetic is exactly that of a single plan, so batched results
// are bit-identical to running the pairs one by one.
#include <string.h>

#include <new>
#include <vector>

#include "blr_internal.cuh"

namespace {

constexpr int KINDS = 3;   // 0 state, 1 adjoint, 2 incremental state

struct Batch {
    int npairs = 0, nt = 0, device = 0, grid = 0;
    std::vector<blr_plan_t> plans;
    SweepPair *d_desc = nullptr;              // [KINDS][nt][npairs]
    long long *d_starts = nullptr;            // [KINDS][npairs + 1]
    unsigned long long *d_counters = nullptr; // [KINDS][nt]
    int *d_active = nullptr;                  // [npairs]
    std::vector<int> h_active;                // pageable: cudaMemcpyAsync stages it before returning
    cudaStream_t s = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    cudaGraphExec_t pcg_exec = nullptr;
    unsigned long long pcg_launches = 0;      // kernel nodes per replay
    double *h_sc = nullptr;                   // pinned [npairs][SC_COUNT]
    int *h_flags = nullptr;                   // pinned [npairs]
    bool wide = false;                        // every pair runs the wide-copy sweep tiles
};

Batch *as_batch(blr_batch_t b) { return reinterpret_cast<Batch *>(b); }

int fill_descriptors(Batch *B) {
    const int np = B->npairs, nt = B->nt;
    std::vector<SweepPair> h((size_t)KINDS * nt * np);
    std::vector<long long> starts((size_t)KINDS * (np + 1), 0);
    for (int p = 0; p < np; ++p) {
        blr_plan *P = B->plans[p];
        int tiles[KINDS][3];
        for (int kind = 0; kind < KINDS; ++kind) {
            sweep_tiles(P, kind, B->wide, &tiles[kind][0], &tiles[kind][1], &tiles[kind][2]);
            long long *st = starts.data() + (size_t)kind * (np + 1);
            st[p + 1] = st[p] + (long long)tiles[kind][0] * tiles[kind][1] * tiles[kind][2];
        }
        const float lam_scale = (float)(-2.0 / (P->p.sigma * P->p.sigma));
        auto base_for = [&](int kind) {
            SweepPair b{};
            b.g = P->grid;
            b.chunk = sweep_chunk(P, kind);
            b.tk = tiles[kind][0];
            b.tj = tiles[kind][1];
            b.ti = tiles[kind][2];
            b.d = P->d;
            b.d4 = P->d4;
            b.dt = P->dt;
            b.scale = lam_scale;
            b.active = B->d_active + p;
            return b;
        };
        for (int n = 0; n < nt; ++n) {
            // state step n: m^n -> m^{n+1}; the last step also writes lambda^nt
            SweepPair st = base_for(0);
            st.in0 = state_slot(P, n);
            st.out0 = state_slot(P, n + 1);
            if (n == nt - 1) {
                st.aux = P->I1;
                st.out1 = P->lam[0];
                st.partials = P->partials;
            }
            h[((size_t)0 * nt + n) * np + p] = st;
            // adjoint step n: lambda ping-pong starts in lam[0] at n = nt - 1
            SweepPair ad = base_for(1);
            const int ca = (nt - 1 - n) & 1;
            ad.in0 = P->lam[ca];
            ad.m = state_slot(P, n);
            ad.out0 = P->lam[1 - ca];
            ad.out1 = P->b;
            h[((size_t)1 * nt + n) * np + p] = ad;
            // incremental state step n: dm ping-pong, dlambda^nt into lam[0]
            SweepPair in = base_for(2);
            const int ci = n & 1;
            in.in0 = P->dm[ci];
            in.m = state_slot(P, n);
            in.aux = P->dv;
            in.out0 = (n == nt - 1) ? P->lam[0] : P->dm[1 - ci];
            h[((size_t)2 * nt + n) * np + p] = in;
        }
    }
    BLR_CK(cudaMemcpy(B->d_desc, h.data(), h.size() * sizeof(SweepPair), cudaMemcpyHostToDevice));
    BLR_CK(cudaMemcpy(B->d_starts, starts.data(), starts.size() * sizeof(long long),
                      cudaMemcpyHostToDevice));
    return BLR_OK;
}

int launch_sweep(Batch *B, int kind, int n, cudaStream_t s) {
    const int nt = B->nt;
    bool f1, f2;
    if (kind == 0) {
        f1 = n == nt - 1;
        f2 = false;
    } else if (kind == 1) {
        f1 = n == nt - 1;
        f2 = n > 0;
    } else {
        f1 = n == 0;
        f2 = n == nt - 1;
    }
    return sweep_batch_launch(kind, f1, f2, B->wide, B->d_desc + ((size_t)kind * nt + n) * B->npairs,
                              B->d_starts + (size_t)kind * (B->npairs + 1), B->npairs,
                              B->d_counters + (size_t)kind * nt + n,
                              sweep_blocks_per_sm(kind, B->wide) * B->grid, s);
}

int reset_counters(Batch *B, cudaStream_t s) {
    BLR_CK(cudaMemsetAsync(B->d_counters, 0, (size_t)KINDS * B->nt * sizeof(unsigned long long), s));
    return BLR_OK;
}

int fork(Batch *B) {
    BLR_CK(cudaEventRecord(B->ev_fork, B->s));
    for (cudaStream_t t : B->side) BLR_CK(cudaStreamWaitEvent(t, B->ev_fork, 0));
    return BLR_OK;
}

int join(Batch *B) {
    for (size_t i = 0; i < B->side.size(); ++i) {
        BLR_CK(cudaEventRecord(B->ev_join[i], B->side[i]));
        BLR_CK(cudaStreamWaitEvent(B->s, B->ev_join[i], 0));
    }
    return BLR_OK;
}

cudaStream_t lane_of(Batch *B, int p) { return B->side[p % B->side.size()]; }

int upload_active(Batch *B, const std::vector<int> &sel) {
    B->h_active.assign(sel.begin(), sel.end());
    BLR_CK(cudaMemcpyAsync(B->d_active, B->h_active.data(), B->npairs * sizeof(int),
                           cudaMemcpyHostToDevice, B->s));
    return BLR_OK;
}

int flag_status(int flags) {
    if (flags & BLR_FLAG_TIMEOUT) return BLR_ETIMEOUT;
    if (flags & BLR_FLAG_NAN) return BLR_ENAN;
    if (flags & BLR_FLAG_CFL) return BLR_ECFL;
    return BLR_OK;
}

// Forward solves at vt[p] (device) for the selected pairs; energies in each dsc.
int batch_state(Batch *B, const std::vector<int> &sel, const std::vector<const float *> &vt) {
    int rc;
    if ((rc = upload_active(B, sel)) || (rc = reset_counters(B, B->s)) || (rc = fork(B))) return rc;
    for (int p = 0; p < B->npairs; ++p) {
        if (!sel[p]) continue;
        blr_plan *P = B->plans[p];
        cudaStream_t t = lane_of(B, p);
        if (vt[p] != P->vt)
            BLR_CK(cudaMemcpyAsync(P->vt, vt[p], P->nfloat * sizeof(float), cudaMemcpyDefault, t));
        if ((rc = dft_expand(P, P->vt, P->d, 1, t))) return rc;
    }
    if ((rc = join(B))) return rc;
    for (int n = 0; n < B->nt; ++n)
        if ((rc = launch_sweep(B, 0, n, B->s))) return rc;
    if ((rc = fork(B))) return rc;
    for (int p = 0; p < B->npairs; ++p) {
        if (!sel[p]) continue;
        blr_plan *P = B->plans[p];
        if ((rc = energy_finalize(P, P->vt, nullptr, (int)sweep_blocks(P), lane_of(B, p)))) return rc;
        P->have_state = true;
        P->seg_valid = 0;
    }
    return join(B);
}

// Gradients of the selected pairs at their current points into g[p].
int batch_gradient_here(Batch *B, const std::vector<int> &sel, const std::vector<float *> &g) {
    int rc;
    if ((rc = upload_active(B, sel)) || (rc = reset_counters(B, B->s))) return rc;
    for (int n = B->nt - 1; n >= 0; --n)
        if ((rc = launch_sweep(B, 1, n, B->s))) return rc;
    if ((rc = fork(B))) return rc;
    for (int p = 0; p < B->npairs; ++p) {
        if (!sel[p]) continue;
        blr_plan *P = B->plans[p];
        if ((rc = dft_project(P, P->b, g[p], P->vt, lane_of(B, p)))) return rc;
    }
    return join(B);
}

// Gauss-Newton HVPs of all pairs (flags decide which pairs' sweeps run).
int batch_hessvec_all(Batch *B, const std::vector<const float *> &dvt,
                      const std::vector<float *> &hdv) {
    int rc;
    if ((rc = reset_counters(B, B->s)) || (rc = fork(B))) return rc;
    for (int p = 0; p < B->npairs; ++p)
        if ((rc = dft_expand(B->plans[p], dvt[p], B->plans[p]->dv, 0, lane_of(B, p)))) return rc;
    if ((rc = join(B))) return rc;
    for (int n = 0; n < B->nt; ++n)
        if ((rc = launch_sweep(B, 2, n, B->s))) return rc;
    for (int n = B->nt - 1; n >= 0; --n)
        if ((rc = launch_sweep(B, 1, n, B->s))) return rc;
    if ((rc = fork(B))) return rc;
    for (int p = 0; p < B->npairs; ++p)
        if ((rc = dft_project(B->plans[p], B->plans[p]->b, hdv[p], dvt[p], lane_of(B, p)))) return rc;
    return join(B);
}

// One PCG iteration of every pair (HVP, <p, q>, update of x = step, r and the
// next direction), captured once as a graph.
int capture_pcg(Batch *B) {
    if (B->pcg_exec) return BLR_OK;
    std::vector<const float *> in(B->npairs);
    std::vector<float *> out(B->npairs);
    for (int p = 0; p < B->npairs; ++p) {
        in[p] = B->plans[p]->pv;
        out[p] = B->plans[p]->q;
    }
    const unsigned long long l0 = blr_kernel_launches();
    BLR_CK(cudaStreamBeginCapture(B->s, cudaStreamCaptureModeThreadLocal));
    int rc = batch_hessvec_all(B, in, out);
    if (!rc) rc = fork(B);
    for (int p = 0; p < B->npairs && !rc; ++p) {
        blr_plan *P = B->plans[p];
        cudaStream_t t = lane_of(B, p);
        if ((rc = vec_dot(P, P->pv, P->q, nullptr, P->dsc + SC_PQ, t))) break;
        if ((rc = pcg_update(P, P->step, t))) break;
        rc = pcg_direction(P, t);
    }
    if (!rc) rc = join(B);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(B->s, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return BLR_ECUDA;
    B->pcg_launches = blr_kernel_launches() - l0;
    e = cudaGraphInstantiate(&B->pcg_exec, graph, 0);
    cudaGraphDestroy(graph);
    return e == cudaSuccess ? BLR_OK : BLR_ECUDA;
}

int fetch_all(Batch *B, bool flags) {
    for (int p = 0; p < B->npairs; ++p) {
        BLR_CK(cudaMemcpyAsync(B->h_sc + (size_t)p * SC_COUNT, B->plans[p]->dsc,
                               SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, B->s));
        if (flags) {
            BLR_CK(cudaMemcpyAsync(B->h_flags + p, B->plans[p]->dstatus, sizeof(int),
                                   cudaMemcpyDeviceToHost, B->s));
            BLR_CK(cudaMemsetAsync(B->plans[p]->dstatus, 0, sizeof(int), B->s));
        }
    }
    BLR_CK(cudaStreamSynchronize(B->s));
    return BLR_OK;
}

double sc(Batch *B, int p, int slot) { return B->h_sc[(size_t)p * SC_COUNT + slot]; }

// For the adjoint and the incremental-state sweeps, time one interior batched
// step for candidate x1 chunks (each plan's own autotuned chunk, or 4, 8, 16, 32
// planes for every pair) and keep the best; the state sweep shares the
// incremental-state chunk.
int batch_autotune(Batch *B) {
    const int cands[5] = {0, 4, 8, 16, 32};   // 0: each plan's own chunk
    cudaEvent_t e0, e1;
    BLR_CK(cudaEventCreate(&e0));
    BLR_CK(cudaEventCreate(&e1));
    std::vector<int> all(B->npairs, 1);
    int rc = upload_active(B, all);
    const int n = B->nt > 2 ? 1 : 0;
    for (int kind = 1; kind <= 2 && !rc; ++kind) {
        std::vector<int> own(B->npairs);
        for (int p = 0; p < B->npairs; ++p) own[p] = sweep_chunk(B->plans[p], kind);
        auto apply = [&](int c) {
            for (int p = 0; p < B->npairs; ++p) {
                blr_plan *P = B->plans[p];
                sweep_set_chunk(P, kind, cands[c] ? (cands[c] < P->N1 ? cands[c] : P->N1) : own[p]);
            }
        };
        float best = 1e30f;
        int best_c = 0;
        for (int c = 0; c < 5 && !rc; ++c) {
            apply(c);
            if ((rc = fill_descriptors(B))) break;
            float tot = 0.f;
            for (int rep = 0; rep < 3 && !rc; ++rep) {
                if ((rc = reset_counters(B, B->s))) break;
                if (cudaEventRecord(e0, B->s) != cudaSuccess) rc = BLR_ECUDA;
                if (!rc) rc = launch_sweep(B, kind, n, B->s);
                if (!rc && (cudaEventRecord(e1, B->s) != cudaSuccess ||
                            cudaEventSynchronize(e1) != cudaSuccess))
                    rc = BLR_ECUDA;
                float ms = 0.f;
                if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = BLR_ECUDA;
                if (rep) tot += ms;
            }
            if (tot < best) {
                best = tot;
                best_c = c;
            }
        }
        apply(best_c);
    }
    if (!rc) rc = fill_descriptors(B);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

void free_batch(Batch *B) {
    if (!B) return;
    if (B->pcg_exec) cudaGraphExecDestroy(B->pcg_exec);
    for (cudaStream_t t : B->side) cudaStreamDestroy(t);
    for (cudaEvent_t e : B->ev_join) cudaEventDestroy(e);
    if (B->ev_fork) cudaEventDestroy(B->ev_fork);
    if (B->s) cudaStreamDestroy(B->s);
    cudaFree(B->d_desc);
    cudaFree(B->d_starts);
    cudaFree(B->d_counters);
    cudaFree(B->d_active);
    cudaFreeHost(B->h_sc);
    cudaFreeHost(B->h_flags);
    for (blr_plan_t P : B->plans) blr_plan_destroy(P);
    delete B;
}

}  // namespace

extern "C" {

int blr_batch_create(const blr_params *params, int npairs, blr_batch_t *out) {
    if (!out || !params || npairs < 1) return BLR_EINVAL;
    *out = nullptr;
    for (int p = 0; p < npairs; ++p)
        if (params[p].nt != params[0].nt || params[p].ckpt_every != 0 ||
            params[p].precision != BLR_FP32 || params[p].incompressible != 0 ||
            params[p].hessian != BLR_GAUSS_NEWTON || params[p].nonstationary != 0 ||
            params[p].state_equation != BLR_STATE_IMAGE)
            return BLR_EINVAL;
    Batch *B = new (std::nothrow) Batch();
    if (!B) return BLR_ENOMEM;
    B->npairs = npairs;
    B->nt = params[0].nt;
    int rc = BLR_OK;
    if (cudaGetDevice(&B->device) != cudaSuccess) rc = BLR_ECUDA;
    for (int p = 0; p < npairs && !rc; ++p) {
        blr_plan_t P = nullptr;
        rc = plan_create(&params[p], false, &P);
        if (!rc) B->plans.push_back(P);
    }
    int sms = 0;
    if (!rc && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device) != cudaSuccess)
        rc = BLR_ECUDA;
    B->grid = sms > 0 ? sms : 148;   // SMs; persistent grids are blocks-per-SM multiples
    B->wide = !rc;
    for (int p = 0; p < npairs && !rc; ++p) B->wide = B->wide && B->plans[p]->sweep_wide;
    const int nside = npairs < 8 ? npairs : 8;
    if (!rc &&
        (cudaMalloc(&B->d_desc, sizeof(SweepPair) * KINDS * B->nt * npairs) != cudaSuccess ||
         cudaMalloc(&B->d_starts, sizeof(long long) * KINDS * (npairs + 1)) != cudaSuccess ||
         cudaMalloc(&B->d_counters, sizeof(unsigned long long) * KINDS * B->nt) != cudaSuccess ||
         cudaMalloc(&B->d_active, sizeof(int) * npairs) != cudaSuccess ||
         cudaMallocHost(&B->h_sc, sizeof(double) * SC_COUNT * npairs) != cudaSuccess ||
         cudaMallocHost(&B->h_flags, sizeof(int) * npairs) != cudaSuccess))
        rc = BLR_ENOMEM;
    if (!rc && (cudaStreamCreateWithFlags(&B->s, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) != cudaSuccess))
        rc = BLR_ECUDA;
    for (int i = 0; i < nside && !rc; ++i) {
        cudaStream_t t;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            rc = BLR_ECUDA;
            break;
        }
        B->side.push_back(t);
        B->ev_join.push_back(e);
    }
    for (int p = 0; p < npairs && !rc; ++p) B->plans[p]->active = B->d_active + p;
    if (!rc) rc = batch_autotune(B);
    if (!rc && cudaStreamSynchronize(B->s) != cudaSuccess) rc = BLR_ECUDA;
    if (rc) {
        free_batch(B);
        return rc;
    }
    *out = reinterpret_cast<blr_batch_t>(B);
    return BLR_OK;
}

int blr_batch_destroy(blr_batch_t b) {
    if (!b) return BLR_OK;
    cudaDeviceSynchronize();
    free_batch(as_batch(b));
    return BLR_OK;
}

int blr_batch_set_images(blr_batch_t b, int pair, const float *I0, const float *I1,
                         blr_stream_t stream) {
    Batch *B = as_batch(b);
    if (!B || pair < 0 || pair >= B->npairs) return BLR_EINVAL;
    return blr_set_images(B->plans[pair], I0, I1, stream);
}

int blr_batch_gradient(blr_batch_t b, const float *const *vt, float *const *g, blr_stream_t stream) {
    Batch *B = as_batch(b);
    if (!B || !vt || !g) return BLR_EINVAL;
    BLR_CK(cudaStreamSynchronize((cudaStream_t)stream));
    std::vector<int> all(B->npairs, 1);
    std::vector<const float *> v(vt, vt + B->npairs);
    std::vector<float *> gg(g, g + B->npairs);
    int rc = batch_state(B, all, v);
    if (!rc) rc = batch_gradient_here(B, all, gg);
    BLR_CK(cudaStreamSynchronize(B->s));
    return rc;
}

int blr_batch_hessvec(blr_batch_t b, const float *const *dvt, float *const *hdv,
                      blr_stream_t stream) {
    Batch *B = as_batch(b);
    if (!B || !dvt || !hdv) return BLR_EINVAL;
    for (blr_plan_t P : B->plans)
        if (!P->have_state) return BLR_ESTATE;
    BLR_CK(cudaStreamSynchronize((cudaStream_t)stream));
    std::vector<int> all(B->npairs, 1);
    int rc = upload_active(B, all);
    if (!rc) rc = batch_hessvec_all(B, std::vector<const float *>(dvt, dvt + B->npairs),
                                    std::vector<float *>(hdv, hdv + B->npairs));
    BLR_CK(cudaStreamSynchronize(B->s));
    return rc;
}

int blr_batch_newton(blr_batch_t b, float *const *vt, int max_newton, int max_pcg, double gtol,
                     double forcing, blr_report *reps, blr_stream_t stream) {
    Batch *B = as_batch(b);
    if (!B || !vt || max_newton < 0 || max_pcg < 0) return BLR_EINVAL;
    BLR_CK(cudaStreamSynchronize((cudaStream_t)stream));
    const int np = B->npairs;
    int rc = capture_pcg(B);
    if (rc) return rc;
    std::vector<blr_report> R(np);
    memset(R.data(), 0, sizeof(blr_report) * np);
    std::vector<int> all(np, 1), live(np, 1);
    std::vector<double> E(np), g0inf(np), g0n(np), ginf(np), gn(np);
    std::vector<const float *> cur(np), tri(np);
    std::vector<float *> gptr(np);
    for (int p = 0; p < np; ++p) {
        blr_plan *P = B->plans[p];
        BLR_CK(cudaMemcpyAsync(P->vtmp, vt[p], P->nfloat * sizeof(float), cudaMemcpyDefault, B->s));
        cur[p] = P->vtmp;
        tri[p] = P->trial;
        gptr[p] = P->g;
    }
    if ((rc = batch_state(B, all, cur)) || (rc = batch_gradient_here(B, all, gptr))) return rc;
    for (int p = 0; p < np; ++p) {
        blr_plan *P = B->plans[p];
        if ((rc = vec_maxabs(P, P->g, P->dsc + SC_GINF, B->s)) ||
            (rc = vec_dot(P, P->g, P->g, nullptr, P->dsc + SC_DOT, B->s)))
            return rc;
    }
    if ((rc = fetch_all(B, true))) return rc;
    for (int p = 0; p < np; ++p) {
        R[p].n_state = 1;
        if ((R[p].status = flag_status(B->h_flags[p]))) live[p] = 0;
        E[p] = sc(B, p, SC_E);
        R[p].energy0 = E[p];
        g0inf[p] = ginf[p] = sc(B, p, SC_GINF);
        g0n[p] = gn[p] = sqrt(sc(B, p, SC_DOT));
    }
    const double c1 = 1e-4;
    for (int it = 0; it < max_newton; ++it) {
        std::vector<int> go(np, 0);
        std::vector<double> eta(np, 0.0);
        int any = 0;
        for (int p = 0; p < np; ++p) {
            if (!live[p] || !(g0inf[p] > 0) || ginf[p] / g0inf[p] < gtol) continue;
            go[p] = 1;
            any = 1;
            eta[p] = forcing >= 0 ? forcing : fmin(0.5, sqrt(gn[p] / g0n[p]));
        }
        if (!any) break;
        // PCG on H p = -g from 0 for the pairs in `go`
        for (int p = 0; p < np; ++p) {
            if (!go[p]) continue;
            blr_plan *P = B->plans[p];
            if ((rc = vec_axpy(P, P->trial, P->g, P->g, -2.0, B->s)) ||
                (rc = pcg_init(P, P->trial, P->step, B->s)))
                return rc;
        }
        if ((rc = fetch_all(B, false))) return rc;
        std::vector<int> pcg_on(np, 0);
        std::vector<double> rr0(np, 0.0);
        for (int p = 0; p < np; ++p) {
            rr0[p] = sc(B, p, SC_RR0);
            pcg_on[p] = go[p] && rr0[p] > 0;
        }
        for (int j = 0; j < max_pcg; ++j) {
            int on = 0;
            for (int p = 0; p < np; ++p) on |= pcg_on[p];
            if (!on) break;
            if ((rc = upload_active(B, pcg_on))) return rc;
            BLR_CK(cudaGraphLaunch(B->pcg_exec, B->s));
            __atomic_fetch_add(&g_blr_launches, B->pcg_launches, __ATOMIC_RELAXED);
            if ((rc = fetch_all(B, false))) return rc;
            for (int p = 0; p < np; ++p) {
                if (!pcg_on[p]) continue;
                R[p].n_hessvec++;
                R[p].pcg_iters++;
                const double pq = sc(B, p, SC_PQ);
                if (!(pq > 0)) {
                    R[p].status = isfinite(pq) ? BLR_ECURV : BLR_ENAN;
                    pcg_on[p] = 0;
                    go[p] = 0;
                    live[p] = 0;
                    continue;
                }
                if (sqrt(sc(B, p, SC_RR) / rr0[p]) <= eta[p]) pcg_on[p] = 0;
            }
        }
        // Armijo backtracking for every pair still going
        std::vector<double> slope(np), eps(np, 1.0);
        for (int p = 0; p < np; ++p)
            if (go[p] && (rc = vec_dot(B->plans[p], B->plans[p]->g, B->plans[p]->step, nullptr,
                                       B->plans[p]->dsc + SC_DOT, B->s)))
                return rc;
        if ((rc = fetch_all(B, false))) return rc;
        for (int p = 0; p < np; ++p) slope[p] = sc(B, p, SC_DOT);
        std::vector<int> search = go, accepted(np, 0);
        for (int h = 0; h <= 10; ++h) {
            int on = 0;
            for (int p = 0; p < np; ++p) {
                if (!search[p]) continue;
                on = 1;
                blr_plan *P = B->plans[p];
                if ((rc = vec_axpy(P, P->trial, P->vtmp, P->step, eps[p], B->s))) return rc;
            }
            if (!on) break;
            if ((rc = batch_state(B, search, tri)) || (rc = fetch_all(B, true))) return rc;
            for (int p = 0; p < np; ++p) {
                if (!search[p]) continue;
                R[p].n_state++;
                const double Et = sc(B, p, SC_E);
                if (B->h_flags[p] == 0 && isfinite(Et) && Et <= E[p] + c1 * eps[p] * slope[p]) {
                    accepted[p] = 1;
                    search[p] = 0;
                    E[p] = Et;
                } else {
                    eps[p] *= 0.5;
                    R[p].n_halvings++;
                }
            }
        }
        std::vector<int> restore(np, 0);
        int any_restore = 0;
        for (int p = 0; p < np; ++p)
            if (go[p] && !accepted[p]) {
                restore[p] = 1;
                any_restore = 1;
                live[p] = 0;
            }
        if (any_restore) {
            if ((rc = batch_state(B, restore, cur))) return rc;
            for (int p = 0; p < np; ++p) R[p].n_state += restore[p];
        }
        int any_acc = 0;
        for (int p = 0; p < np; ++p) {
            if (!accepted[p]) continue;
            any_acc = 1;
            blr_plan *P = B->plans[p];
            BLR_CK(cudaMemcpyAsync(P->vtmp, P->trial, P->nfloat * sizeof(float),
                                   cudaMemcpyDeviceToDevice, B->s));
            R[p].newton_iters++;
        }
        if (!any_acc) break;
        if ((rc = batch_gradient_here(B, accepted, gptr))) return rc;
        for (int p = 0; p < np; ++p) {
            if (!accepted[p]) continue;
            blr_plan *P = B->plans[p];
            if ((rc = vec_maxabs(P, P->g, P->dsc + SC_GINF, B->s)) ||
                (rc = vec_dot(P, P->g, P->g, nullptr, P->dsc + SC_DOT, B->s)))
                return rc;
        }
        if ((rc = fetch_all(B, false))) return rc;
        for (int p = 0; p < np; ++p)
            if (accepted[p]) {
                ginf[p] = sc(B, p, SC_GINF);
                gn[p] = sqrt(sc(B, p, SC_DOT));
            }
    }
    for (int p = 0; p < np; ++p) {
        BLR_CK(cudaMemcpyAsync(vt[p], B->plans[p]->vtmp, B->plans[p]->nfloat * sizeof(float),
                               cudaMemcpyDefault, B->s));
        R[p].energy = E[p];
        R[p].grad_inf_rel = g0inf[p] > 0 ? ginf[p] / g0inf[p] : 0.0;
    }
    BLR_CK(cudaStreamSynchronize(B->s));
    if (reps) memcpy(reps, R.data(), sizeof(blr_report) * np);
    return BLR_OK;
}

}  // extern "C"
