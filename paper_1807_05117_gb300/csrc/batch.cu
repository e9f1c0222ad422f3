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
// * The x1 chunk of the sweep tiles, and whether the batched sweeps keep the
//   state gradients, are chosen by timing candidates on the batch itself
//   (batch_autotune).
// * A pair of at least solo_min voxels (2^19 by default) runs "solo": it skips
//   the work queue and runs its own plan's autotuned kernels (balanced grids, the
//   split or two-step adjoint, the gather form of the incremental state) on one
//   of three side lanes, concurrently with other solo pairs and with the queued
//   pairs' launches; its PCG iteration is a graph of its own, replayed while the
//   pair is active.
// Each pair's arithmetic is exactly that of a single plan, so batched results
// are bit-identical to running the pairs one by one.
#include <string.h>

#include <new>
#include <vector>

#include "blr_internal.cuh"

namespace {

constexpr int KINDS = 3;   // 0 state, 1 adjoint, 2 incremental state
constexpr int SOLO_LANES = 3;   // side streams that run solo pairs concurrently

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
    bool gm = false;                          // every pair keeps its state gradients
    bool useg = false;                        // the batched sweeps write / read them (autotuned)
    bool inc_gather = false;                  // with useg: incremental steps in the gather form
    std::vector<int> own_chunk[3];            // [kind][pair]: each plan's own x1 chunk
    int chunk_choice[3] = {0, 0, 0};          // [kind]: 0 = own chunks, else planes for all
    long long solo_min = 1LL << 19;           // voxels from which a pair runs solo (0: none)
    std::vector<char> solo;                   // [pair]
    int nbatched = 0;                         // pairs in the work queue
    std::vector<cudaGraphExec_t> solo_exec;   // [pair]: PCG iteration of a solo pair
    std::vector<unsigned long long> solo_launches;
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
            st[p + 1] = st[p] + (B->solo[p] ? 0LL
                                            : (long long)tiles[kind][0] * tiles[kind][1] * tiles[kind][2]);
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
            st.Gout = B->useg ? grad_slot(P, n) : nullptr;
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
            ad.G = B->useg ? grad_slot(P, n) : nullptr;
            h[((size_t)1 * nt + n) * np + p] = ad;
            // incremental state step n: dm ping-pong, dlambda^nt into lam[0]
            SweepPair in = base_for(2);
            const int ci = n & 1;
            in.in0 = P->dm[ci];
            in.m = state_slot(P, n);
            in.aux = P->dv;
            in.out0 = (n == nt - 1) ? P->lam[0] : P->dm[1 - ci];
            in.G = B->useg ? grad_slot(P, n) : nullptr;
            h[((size_t)2 * nt + n) * np + p] = in;
        }
    }
    B->nbatched = 0;
    for (int p = 0; p < np; ++p) B->nbatched += B->solo[p] ? 0 : 1;
    BLR_CK(cudaMemcpy(B->d_desc, h.data(), h.size() * sizeof(SweepPair), cudaMemcpyHostToDevice));
    BLR_CK(cudaMemcpy(B->d_starts, starts.data(), starts.size() * sizeof(long long),
                      cudaMemcpyHostToDevice));
    return BLR_OK;
}

int launch_sweep(Batch *B, int kind, int n, cudaStream_t s) {
    if (B->nbatched == 0) return BLR_OK;   // every pair runs solo
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
    // the gather form runs on the incremental-state (kind 2) items and descriptors
    const int launch_kind = (kind == 2 && B->useg && B->inc_gather) ? 3 : kind;
    return sweep_batch_launch(launch_kind, f1, f2, B->wide, B->useg,
                              B->d_desc + ((size_t)kind * nt + n) * B->npairs,
                              B->d_starts + (size_t)kind * (B->npairs + 1), B->npairs,
                              B->d_counters + (size_t)kind * nt + n,
                              sweep_blocks_per_sm(launch_kind, B->wide) * B->grid, s);
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

// Lane of the k-th solo pair of a pass.
cudaStream_t solo_lane(Batch *B, int k) {
    const int n = (int)B->side.size() < SOLO_LANES ? (int)B->side.size() : SOLO_LANES;
    return B->side[k % n];
}

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
        if (!sel[p] || B->solo[p]) continue;
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
        if (!sel[p] || B->solo[p]) continue;
        blr_plan *P = B->plans[p];
        if ((rc = energy_finalize(P, P->vt, nullptr, (int)sweep_blocks(P), lane_of(B, p)))) return rc;
        P->have_state = true;
        P->seg_valid = 0;
    }
    int k = 0;
    for (int p = 0; p < B->npairs; ++p)
        if (sel[p] && B->solo[p] && (rc = state_at(B->plans[p], vt[p], nullptr, solo_lane(B, k++))))
            return rc;
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
        if (!sel[p] || B->solo[p]) continue;
        blr_plan *P = B->plans[p];
        if ((rc = dft_project(P, P->b, g[p], P->vt, lane_of(B, p)))) return rc;
    }
    int k = 0;
    for (int p = 0; p < B->npairs; ++p)
        if (sel[p] && B->solo[p] && (rc = gradient_here(B->plans[p], g[p], solo_lane(B, k++))))
            return rc;
    return join(B);
}

// Gauss-Newton HVPs of all pairs (flags decide which queued pairs' sweeps run);
// with_solo: the solo pairs' products too.
int batch_hessvec_all(Batch *B, const std::vector<const float *> &dvt,
                      const std::vector<float *> &hdv, bool with_solo) {
    int rc;
    if ((rc = reset_counters(B, B->s)) || (rc = fork(B))) return rc;
    for (int p = 0; p < B->npairs; ++p)
        if (!B->solo[p] && (rc = dft_expand(B->plans[p], dvt[p], B->plans[p]->dv, 0, lane_of(B, p))))
            return rc;
    if ((rc = join(B))) return rc;
    for (int n = 0; n < B->nt; ++n)
        if ((rc = launch_sweep(B, 2, n, B->s))) return rc;
    for (int n = B->nt - 1; n >= 0; --n)
        if ((rc = launch_sweep(B, 1, n, B->s))) return rc;
    if ((rc = fork(B))) return rc;
    for (int p = 0; p < B->npairs; ++p)
        if (!B->solo[p] &&
            (rc = dft_project(B->plans[p], B->plans[p]->b, hdv[p], dvt[p], lane_of(B, p))))
            return rc;
    if ((rc = join(B))) return rc;
    for (int p = 0; p < B->npairs && with_solo; ++p)
        if (B->solo[p] && (rc = hessvec_here(B->plans[p], dvt[p], hdv[p], B->s))) return rc;
    return BLR_OK;
}

// Capture what `body` queues on the batch stream as a graph (instantiated into
// *exec; *launches: kernel nodes per replay).
template <typename F>
int capture_graph(Batch *B, F &&body, cudaGraphExec_t *exec, unsigned long long *launches) {
    const unsigned long long l0 = blr_kernel_launches();
    BLR_CK(cudaStreamBeginCapture(B->s, cudaStreamCaptureModeThreadLocal));
    int rc = body();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(B->s, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return BLR_ECUDA;
    *launches = blr_kernel_launches() - l0;
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    return e == cudaSuccess ? BLR_OK : BLR_ECUDA;
}

void drop_graphs(Batch *B) {
    if (B->pcg_exec) cudaGraphExecDestroy(B->pcg_exec);
    B->pcg_exec = nullptr;
    for (cudaGraphExec_t &g : B->solo_exec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// One PCG iteration (HVP, <p, q>, update of x = step, r and the next direction)
// captured once as graphs: one for every queued pair, one per solo pair.
int capture_pcg(Batch *B) {
    int rc = BLR_OK;
    if (B->nbatched > 0 && !B->pcg_exec) {
        std::vector<const float *> in(B->npairs);
        std::vector<float *> out(B->npairs);
        for (int p = 0; p < B->npairs; ++p) {
            in[p] = B->plans[p]->pv;
            out[p] = B->plans[p]->q;
        }
        rc = capture_graph(B, [&]() {
            int r = batch_hessvec_all(B, in, out, false);
            if (!r) r = fork(B);
            for (int p = 0; p < B->npairs && !r; ++p) {
                if (B->solo[p]) continue;
                blr_plan *P = B->plans[p];
                cudaStream_t t = lane_of(B, p);
                if ((r = vec_dot(P, P->pv, P->q, nullptr, P->dsc + SC_PQ, t))) break;
                if ((r = pcg_update(P, P->step, t))) break;
                r = pcg_direction(P, t);
            }
            if (!r) r = join(B);
            return r;
        }, &B->pcg_exec, &B->pcg_launches);
    }
    for (int p = 0; p < B->npairs && !rc; ++p) {
        if (!B->solo[p] || B->solo_exec[p]) continue;
        blr_plan *P = B->plans[p];
        // A member keeps every state (no checkpoints), so whenever the graph is
        // replayed a forward solve has left the one segment valid.  Capture with
        // that state, or the product would capture a recomputation of the segment
        // (the segment flag of a plan that has not run yet) and repeat it on
        // every replay.
        const int seg_was = P->seg_valid;
        if (P->nseg == 1) P->seg_valid = 0;
        rc = capture_graph(B, [&]() {
            int r = hessvec_here(P, P->pv, P->q, B->s);
            if (!r) r = vec_dot(P, P->pv, P->q, nullptr, P->dsc + SC_PQ, B->s);
            if (!r) r = pcg_update(P, P->step, B->s);
            if (!r) r = pcg_direction(P, B->s);
            return r;
        }, &B->solo_exec[p], &B->solo_launches[p]);
        P->seg_valid = seg_was;
    }
    return rc;
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

// x1 chunk of every pair for a sweep kind (1 adjoint, 2 incremental and state):
// each plan's own (0) or `planes` for all pairs (at most N1).
void apply_chunk(Batch *B, int kind, int planes) {
    for (int p = 0; p < B->npairs; ++p) {
        blr_plan *P = B->plans[p];
        sweep_set_chunk(P, kind, planes ? (planes < P->N1 ? planes : P->N1) : B->own_chunk[kind][p]);
    }
    B->chunk_choice[kind] = planes;
}

// For the adjoint and the incremental-state sweeps, time one interior batched
// step for candidate x1 chunks (each plan's own autotuned chunk, or 4, 8, 16, 32
// planes for every pair) and keep the best; the state sweep shares the
// incremental-state chunk.  When every pair keeps its state gradients, both
// kinds are tuned with and without reading them, and the faster sum is kept.
// Only the queued pairs take part (solo pairs have no items).
int batch_autotune(Batch *B) {
    const int cands[5] = {0, 4, 8, 16, 32};   // 0: each plan's own chunk
    for (int kind = 1; kind <= 2; ++kind) {
        B->own_chunk[kind].resize(B->npairs);
        for (int p = 0; p < B->npairs; ++p) B->own_chunk[kind][p] = sweep_chunk(B->plans[p], kind);
    }
    int rc = fill_descriptors(B);
    if (rc || B->nbatched == 0) return rc;
    cudaEvent_t e0, e1;
    BLR_CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return BLR_ECUDA;
    }
    std::vector<int> all(B->npairs, 1);
    rc = upload_active(B, all);
    const int n = B->nt > 2 ? 1 : 0;
    const int nu = B->gm ? 2 : 1;
    float total[2] = {0.f, 0.f};
    int best_c[2][3] = {{0, 0, 0}, {0, 0, 0}};
    bool gather[2] = {false, false};
    for (int u = 0; u < nu && !rc; ++u) {
        B->useg = u == 1;
        B->inc_gather = false;
        for (int kind = 1; kind <= 2 && !rc; ++kind) {
            float best = 1e30f;
            for (int c = 0; c < 5 && !rc; ++c) {
                apply_chunk(B, kind, cands[c]);
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
                    best_c[u][kind] = cands[c];
                }
            }
            apply_chunk(B, kind, best_c[u][kind]);
            if (kind == 2 && B->useg && !rc) {   // the gather form at that chunk
                if ((rc = fill_descriptors(B))) break;
                B->inc_gather = true;
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
                B->inc_gather = tot < best;
                gather[u] = B->inc_gather;
                if (tot < best) best = tot;
            }
            total[u] += best;
        }
    }
    const int u = (nu == 2 && total[1] < total[0]) ? 1 : 0;
    B->useg = u == 1;
    B->inc_gather = gather[u];
    apply_chunk(B, 1, best_c[u][1]);
    apply_chunk(B, 2, best_c[u][2]);
    if (!rc) rc = fill_descriptors(B);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

void free_batch(Batch *B) {
    if (!B) return;
    drop_graphs(B);
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
        // kept state gradients (3 nt V floats) when they fit, else the pair
        // interpolates grad m^n in every adjoint and incremental-state step
        blr_plan_t P = nullptr;
        rc = plan_create(&params[p], true, &P);
        if (rc == BLR_ENOMEM) rc = plan_create(&params[p], false, &P);
        if (!rc) B->plans.push_back(P);
    }
    int sms = 0;
    if (!rc && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device) != cudaSuccess)
        rc = BLR_ECUDA;
    B->grid = sms > 0 ? sms : 148;   // SMs; persistent grids are blocks-per-SM multiples
    B->wide = !rc;
    for (int p = 0; p < npairs && !rc; ++p) B->wide = B->wide && B->plans[p]->sweep_wide;
    B->gm = B->wide;
    for (int p = 0; p < npairs && !rc; ++p) B->gm = B->gm && B->plans[p]->Gm != nullptr;
    B->solo.assign(npairs, 0);
    for (int p = 0; p < npairs && !rc; ++p)
        B->solo[p] = B->solo_min > 0 && B->plans[p]->V >= B->solo_min;
    B->solo_exec.assign(npairs, nullptr);
    B->solo_launches.assign(npairs, 0);
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
        if (cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess) {
            rc = BLR_ECUDA;
            break;
        }
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaStreamDestroy(t);
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

int blr_batch_tuning(blr_batch_t b, int *vals, int n) {
    Batch *B = as_batch(b);
    if (!B || !vals || n < 0) return BLR_EINVAL;
    int nsolo = 0;
    for (char c : B->solo) nsolo += c;
    const long long smin = B->solo_min < 0x7fffffffLL ? B->solo_min : 0x7fffffffLL;
    const int v[7] = {B->gm ? 1 : 0, B->useg ? 1 : 0, B->chunk_choice[1], B->chunk_choice[2],
                      (int)smin, nsolo, B->inc_gather ? 1 : 0};
    for (int i = 0; i < n && i < 7; ++i) vals[i] = v[i];
    return BLR_OK;
}

int blr_batch_set_tuning(blr_batch_t b, const int *vals, int n) {
    Batch *B = as_batch(b);
    if (!B || !vals || n < 5) return BLR_EINVAL;
    if (vals[0] != (B->gm ? 1 : 0) || vals[1] < 0 || vals[1] > vals[0] || vals[4] < 0) return BLR_EINVAL;
    for (int k = 2; k < 4; ++k)
        if (vals[k] != 0 && (vals[k] < 2 || vals[k] > 1024)) return BLR_EINVAL;
    const bool gather = n >= 7 ? vals[6] != 0 : (B->inc_gather && vals[1] != 0);
    if (n >= 7 && (vals[6] < 0 || vals[6] > vals[1])) return BLR_EINVAL;
    BLR_CK(cudaDeviceSynchronize());
    drop_graphs(B);   // the captured iterations hold the old launches
    bool moved = (vals[1] != 0) != B->useg;
    B->useg = vals[1] != 0;
    B->solo_min = vals[4];
    for (int p = 0; p < B->npairs; ++p) {
        const char solo = B->solo_min > 0 && B->plans[p]->V >= B->solo_min;
        moved = moved || solo != B->solo[p];
        B->solo[p] = solo;
    }
    // the current points' kept gradients and final adjoint states were written
    // (or not) for the old path: every pair needs a new forward solve
    if (moved)
        for (blr_plan_t P : B->plans) P->have_state = false;
    B->inc_gather = gather;
    apply_chunk(B, 1, vals[2]);
    apply_chunk(B, 2, vals[3]);
    return fill_descriptors(B);
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
                                    std::vector<float *>(hdv, hdv + B->npairs), true);
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
            bool queued = false;
            for (int p = 0; p < np; ++p) queued = queued || (pcg_on[p] && !B->solo[p]);
            // the solo pairs' iterations on SOLO_LANES side lanes in turn, so that one
            // pair's launch tails and transform stages overlap another's sweeps
            if ((rc = fork(B))) return rc;
            if (queued) {
                BLR_CK(cudaGraphLaunch(B->pcg_exec, B->s));
                __atomic_fetch_add(&g_blr_launches, B->pcg_launches, __ATOMIC_RELAXED);
            }
            int k = 0;
            for (int p = 0; p < np; ++p) {
                if (!pcg_on[p] || !B->solo[p]) continue;
                cudaStream_t t = solo_lane(B, k++);
                BLR_CK(cudaGraphLaunch(B->solo_exec[p], t));
                __atomic_fetch_add(&g_blr_launches, B->solo_launches[p], __ATOMIC_RELAXED);
            }
            if ((rc = join(B))) return rc;
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
