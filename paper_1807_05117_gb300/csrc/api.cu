// C-ABI entry points of libblr (declared and documented in include/blr.h).
//
// Host-side control only: every arithmetic step of the hot path runs in the
// kernels of dft.cu, sweeps.cu and reduce.cu.  The Newton and PCG drivers read
// FP64 scalars back from the device to take their stop / accept decisions.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>

#include "blr_internal.cuh"

unsigned long long g_blr_launches = 0;

namespace {

// The context's persisting-L2 set-aside is a per-process limit shared with every
// other library in the process.  Plans that may keep their displacement copy in
// persisting lines raise it; the first of them records the limit as it was, and
// the last one destroyed releases the persisting lines (only if some plan used
// them) and puts the old limit back.
struct L2Share {
    int plans = 0;        // live plans counted here
    bool raised = false;  // a plan raised the limit above `prev`
    bool used = false;    // a plan kept lines in the set-aside
    size_t prev = 0;      // the limit before the first counted plan
};
constexpr int kL2Devices = 64;
std::mutex g_l2_mu;
L2Share g_l2[kL2Devices];

// Raise the set-aside to `aside` bytes for plan P (its device current).
bool l2_acquire(blr_plan *P, size_t aside) {
    if (P->device < 0 || P->device >= kL2Devices) return false;
    std::lock_guard<std::mutex> lock(g_l2_mu);
    L2Share &u = g_l2[P->device];
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) return false;
    if (u.plans == 0) {
        u.prev = cur;
        u.raised = false;
        u.used = false;
    }
    if (cur < aside) {
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, aside) != cudaSuccess) return false;
        u.raised = true;
        cur = aside;
    }
    ++u.plans;
    P->l2_counted = 1;
    P->l2_hit = (float)((double)cur / (double)P->l2_win_bytes);
    if (P->l2_hit > 1.f) P->l2_hit = 1.f;
    return true;
}

// Plan P is going away (its device current).
void l2_release(blr_plan *P) {
    if (!P->l2_counted) return;
    std::lock_guard<std::mutex> lock(g_l2_mu);
    L2Share &u = g_l2[P->device];
    if (P->l2_persist) u.used = true;
    if (--u.plans > 0) return;
    if (u.used) cudaCtxResetPersistingL2Cache();
    if (u.raised) cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, u.prev);
    cudaGetLastError();
    u = L2Share();
}

int validate(const blr_params *p) {
    if (!p) return BLR_EINVAL;
    for (int d = 0; d < 3; ++d) {
        if (p->n[d] < 1 || p->band[d] < 2 || (p->band[d] & 1) || p->band[d] > p->n[d])
            return BLR_EINVAL;
    }
    if (p->band[2] > 64) return BLR_EINVAL;      // stage A' keeps <= 64 frequencies per lane pair
    if (p->nt < 1 || !(p->sigma > 0) || !(p->gamma > 0) || !(p->alpha >= 0)) return BLR_EINVAL;
    if (!(p->s >= 0 && p->s <= 32) || 2.0 * p->s != floor(2.0 * p->s)) return BLR_EINVAL;
    if (p->incompressible != 0 && p->incompressible != 1) return BLR_EINVAL;
    if (p->hessian != BLR_GAUSS_NEWTON && p->hessian != BLR_NEWTON) return BLR_EINVAL;
    if (p->nonstationary != 0 && p->nonstationary != 1) return BLR_EINVAL;
    // the full Hessian is built for stationary velocities
    if (p->nonstationary && p->hessian == BLR_NEWTON) return BLR_EINVAL;
    if (p->state_equation != BLR_STATE_IMAGE && p->state_equation != BLR_STATE_DEFORMATION)
        return BLR_EINVAL;
    // the deformation variant: stationary velocity, every state kept
    if (p->state_equation == BLR_STATE_DEFORMATION &&
        (p->nonstationary || (p->ckpt_every > 0 && p->ckpt_every < p->nt)))
        return BLR_EINVAL;
    // the full Hessian keeps every adjoint and incremental state: no checkpoints
    if (p->hessian == BLR_NEWTON && p->ckpt_every > 0 && p->ckpt_every < p->nt) return BLR_EINVAL;
    if (p->precision != BLR_FP32 && p->precision != BLR_MIXED) return BLR_EINVAL;
    if (p->ckpt_every < 0) return BLR_EINVAL;
    long long V = (long long)p->n[0] * p->n[1] * p->n[2];
    if (V > (1LL << 31)) return BLR_EINVAL;
    if (p->n[0] > 65535) return BLR_EINVAL;   // one grid row of blocks per x1 plane
    return BLR_OK;
}

struct Arena {
    char *base = nullptr;
    size_t used = 0;
    template <typename T>
    T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
        T *r = reinterpret_cast<T *>(base + used);
        used += bytes;
        return r;
    }
};

// Lay out (or, with base == nullptr, size) every device buffer of the plan.
size_t layout(blr_plan *P, char *base) {
    Arena a;
    a.base = base;
    const long long V = P->V;
    P->m = a.take<float>((size_t)(P->nseg + P->ck) * V);
    P->I0 = P->m;                        // m^0 = I0 lives in the first slot
    P->I1 = a.take<float>(V);
    P->d = P->d_base = a.take<float>((size_t)3 * P->nvel * V);
    P->d4 = P->d4_base = P->sweep_wide ? a.take<float4>((size_t)P->nvel * V) : nullptr;
    P->lam[0] = a.take<float>(V);
    P->lam[1] = a.take<float>(V);
    const bool def = P->p.state_equation == BLR_STATE_DEFORMATION;
    P->rho_all = P->du_all = nullptr;
    if (P->p.hessian == BLR_NEWTON) {
        const int nt = P->p.nt;
        if (def) {   // the vector adjoint and incremental states instead of lambda, dm
            P->lam_all = P->dm_all = nullptr;
            P->lam_nt = a.take<float>(V);
            P->rho_all = a.take<float>((size_t)3 * nt * V);
            P->du_all = nt > 1 ? a.take<float>((size_t)3 * (nt - 1) * V) : nullptr;
        } else {
            P->lam_all = a.take<float>((size_t)nt * V);
            P->lam_nt = P->lam_all + (size_t)(nt - 1) * V;
            P->dm_all = nt > 1 ? a.take<float>((size_t)(nt - 1) * V) : nullptr;
        }
        P->nt_kap = a.take<float>((size_t)27 * V);
    } else {
        P->lam_all = P->dm_all = P->nt_kap = nullptr;
        P->lam_nt = a.take<float>(V);
    }
    if (def) {
        P->U = a.take<float>((size_t)3 * (P->p.nt + 1) * V);
        P->rho_nt = P->rho_all ? P->rho_all + (size_t)3 * (P->p.nt - 1) * V : a.take<float>(3 * V);
        P->rho[0] = a.take<float>(3 * V);
        P->rho[1] = a.take<float>(3 * V);
        P->du[0] = a.take<float>(3 * V);
        P->du[1] = a.take<float>(3 * V);
        P->Gw = a.take<float>(3 * V);
    } else {
        P->U = P->rho_nt = P->rho[0] = P->rho[1] = P->du[0] = P->du[1] = P->Gw = nullptr;
    }
    // kept state gradients: [nt][3][V] (image), [nt][3 components][3][V] (deformation)
    const size_t gm_fields = P->p.state_equation == BLR_STATE_DEFORMATION ? 9 : 3;
    P->Gm = P->use_gm ? a.take<float>(gm_fields * P->p.nt * V) : nullptr;
    P->lam_keep = (P->use_gm && P->nvel == 1 && P->p.nt > 1 && P->p.hessian != BLR_NEWTON &&
                   P->p.state_equation == BLR_STATE_IMAGE)
                      ? a.take<float>((size_t)(P->p.nt - 1) * V)
                      : nullptr;
    P->rho_keep = (P->use_gm && P->p.nt > 1 && P->p.state_equation == BLR_STATE_DEFORMATION &&
                   P->p.hessian != BLR_NEWTON)
                      ? a.take<float>((size_t)3 * (P->p.nt - 1) * V)
                      : nullptr;
    P->b = a.take<float>(3 * V);
    P->dv = a.take<float>(3 * V);
    P->dm[0] = a.take<float>(V);
    P->dm[1] = a.take<float>(V);
    P->W1 = a.take<float>((size_t)2 * P->B1 * P->N1);
    P->T2c = a.take<float>((size_t)P->B2 * P->N2);
    P->T2s = a.take<float>((size_t)P->B2 * P->N2);
    P->T3c = a.take<float>((size_t)P->B3 * P->N3);
    P->T3s = a.take<float>((size_t)P->B3 * P->N3);
    P->T2e = P->T2p = P->W1t = P->T3e = nullptr;
    if (P->p.precision == BLR_FP32) {
        P->T3e = a.take<float>((size_t)4 * P->B3 * P->N3);
        P->W1t = a.take<float>((size_t)2 * P->B1 * P->N1);
        P->T2e = a.take<float>((size_t)4 * P->B2 * P->N2);
        P->T2p = a.take<float>((size_t)4 * P->B2 * P->N2);
    }
    P->A = a.take<float>(P->nb);
    // the FP32 stages' intermediates (for every step's velocity at once when non-stationary)
    const size_t dft_vel = (P->p.precision == BLR_FP32 && P->nvel > 1) ? (size_t)P->nvel : 1;
    P->dft_big = a.take<float>(dft_vel * 3 * P->B1 * P->N2 * P->N3 * 2);
    P->dft_small = a.take<float>(dft_vel * 3 * P->B1 * P->B2 * P->N3 * 2);
    for (int k = 0; k < 4; ++k) P->fz_tab[k] = nullptr;
    P->fz_buf = nullptr;
    P->dv_all = P->b_all = nullptr;
    if (P->p.precision == BLR_MIXED && fz_supported(P)) {
        for (int k = 0; k < 4; ++k) P->fz_tab[k] = a.take<uint8_t>(fz_table_bytes(P, k));
        P->fz_buf = a.take<float>(fz_buffer_floats(P));
        if (P->nvel > 1) {   // every step's velocity in one fused transform
            P->dv_all = a.take<float>((size_t)3 * P->nvel * V);
            P->b_all = a.take<float>((size_t)3 * P->nvel * V);
        }
        P->tc_tab_expand = P->tc_tab_project = nullptr;
        P->tc_tab2_expand = P->tc_tab2_project = nullptr;
    } else if (P->p.precision == BLR_MIXED) {
        P->tc_tab_expand = a.take<uint8_t>(tc_table_bytes(P, 0));
        P->tc_tab_project = a.take<uint8_t>(tc_table_bytes(P, 1));
        if (tc_axis2_supported(P)) {
            P->tc_tab2_expand = a.take<uint8_t>(tc_table_bytes(P, 2));
            P->tc_tab2_project = a.take<uint8_t>(tc_table_bytes(P, 3));
        } else {
            P->tc_tab2_expand = P->tc_tab2_project = nullptr;
        }
    } else {
        P->tc_tab_expand = P->tc_tab_project = nullptr;
        P->tc_tab2_expand = P->tc_tab2_project = nullptr;
        if (P->p.precision == BLR_FP32 && P->nvel > 1) {   // every step in one GEMM pass
            P->dv_all = a.take<float>((size_t)3 * P->nvel * V);
            P->b_all = a.take<float>((size_t)3 * P->nvel * V);
        }
    }
    float **vecs[] = {&P->vt, &P->g, &P->r, &P->pv, &P->q, &P->x, &P->trial, &P->step, &P->vtmp};
    for (float **v : vecs) *v = a.take<float>(P->nfloat);
    P->vproj = P->p.incompressible ? a.take<float>(P->nfloat) : nullptr;
    P->dsc = a.take<double>(SC_COUNT);
    P->dstatus = a.take<int>(1);
    P->pcg_live = a.take<int>(4);
    P->ticket = a.take<unsigned int>(1);
    P->partials = a.take<double>(P->npart);
    P->partials2 = a.take<double>(reduce_partials_needed());
    P->active = nullptr;
    return a.used;
}

char *arena_base(blr_plan *P) { return reinterpret_cast<char *>(P->m); }

// Copy the device scalars and the latched flags to the host and wait.
int fetch_scalars(blr_plan *P, cudaStream_t s, int *flags) {
    BLR_CK(cudaMemcpyAsync(P->hsc, P->dsc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (flags) {
        BLR_CK(cudaMemcpyAsync(P->hsc + SC_COUNT, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
        BLR_CK(cudaMemsetAsync(P->dstatus, 0, sizeof(int), s));
    }
    BLR_CK(cudaStreamSynchronize(s));
    if (flags) memcpy(flags, P->hsc + SC_COUNT, sizeof(int));
    return BLR_OK;
}

int flags_to_status(int flags) {
    if (flags & BLR_FLAG_TIMEOUT) return BLR_ETIMEOUT;
    if (flags & BLR_FLAG_NAN) return BLR_ENAN;
    if (flags & BLR_FLAG_CFL) return BLR_ECFL;
    return BLR_OK;
}

}  // namespace

// Forward solve at vt (device) -> current point; energy into dsc (and energy_out).
// Incompressible plans keep P vt as the current velocity.
int state_at(blr_plan *P, const float *vt, double *energy_out, cudaStream_t s) {
    int rc;
    if (P->p.incompressible) {
        if ((rc = vec_leray(P, P->vt, vt, s))) return rc;
    } else if (vt != P->vt) {
        BLR_CK(cudaMemcpyAsync(P->vt, vt, P->nfloat * sizeof(float), cudaMemcpyDefault, s));
    }
    P->have_lams = false;
    if (P->nvel > 1 && P->dv_all) {   // every step's displacement in one transform
        if ((rc = dft_expand_nc(P, P->vt, P->d_base, 1, s, 3 * P->nvel))) return rc;
        for (int n = 0; n < P->nvel; ++n) {
            use_step(P, n);
            if ((rc = sweep_pack_d4(P, s))) return rc;
        }
    } else {
        for (int n = 0; n < P->nvel; ++n) {   // every step's displacement (one when stationary)
            use_step(P, n);
            if ((rc = dft_expand(P, P->vt + (size_t)n * P->nf1, P->d, 1, s))) return rc;
        }
    }
    if (P->p.state_equation == BLR_STATE_DEFORMATION) {
        if ((rc = sweep_state_def(P, s))) return rc;
        if ((rc = energy_finalize(P, P->vt, energy_out, def_final_blocks(P), s))) return rc;
    } else {
        if ((rc = sweep_state(P, s))) return rc;
        if ((rc = energy_finalize(P, P->vt, energy_out, (int)sweep_blocks(P), s))) return rc;
    }
    P->have_state = true;
    return BLR_OK;
}

// g = A v~ + pi(b) at the current point (incompressible: P applied to it).
// Non-stationary: g^n = dt A v~^n + pi(b^n) per step.
int gradient_here(blr_plan *P, float *g, cudaStream_t s) {
    int rc;
    if (P->nvel > 1) {
        if ((rc = sweep_adjoint_steps(P, P->lam_nt, g, P->vt, nullptr, nullptr, s))) return rc;
    } else if (P->p.state_equation == BLR_STATE_DEFORMATION) {
        if ((rc = sweep_adjoint_def(P, P->rho_nt, P->b, s))) return rc;
        if ((rc = dft_project(P, P->b, g, P->vt, s))) return rc;
    } else {
        if ((rc = sweep_adjoint(P, P->b, nullptr, P->lam_nt, s))) return rc;
        if ((rc = dft_project(P, P->b, g, P->vt, s))) return rc;
    }
    return P->p.incompressible ? vec_leray(P, g, g, s) : BLR_OK;
}

// H dv~ = A dv~ + pi(db) (incompressible: P H P dv~).  Gauss-Newton, or the full
// Hessian, which needs the gradient's adjoint states (computed here when the
// current point has none yet).
int hessvec_here(blr_plan *P, const float *dvt, float *hdv, cudaStream_t s) {
    int rc;
    const bool full = P->p.hessian == BLR_NEWTON;
    if (full && !P->have_lams && P->p.state_equation == BLR_STATE_IMAGE &&
        (rc = sweep_adjoint(P, P->b, nullptr, P->lam_nt, s)))
        return rc;
    if (P->p.incompressible) {
        if ((rc = vec_leray(P, P->vproj, dvt, s))) return rc;
        dvt = P->vproj;
    }
    if (P->p.state_equation == BLR_STATE_DEFORMATION) {
        if (full && !P->have_lams && (rc = sweep_adjoint_def(P, P->rho_nt, P->b, s))) return rc;
        if ((rc = dft_expand(P, dvt, P->dv, 0, s))) return rc;
        if ((rc = sweep_incremental_def(P, s))) return rc;
        if (full && (rc = newton_prep(P, s))) return rc;
        rc = full ? sweep_adjoint_def_newton(P, P->b, s) : sweep_adjoint_def(P, P->rho[0], P->b, s);
        if (rc) return rc;
        if ((rc = dft_project(P, P->b, hdv, dvt, s))) return rc;
        return P->p.incompressible ? vec_leray(P, hdv, hdv, s) : BLR_OK;
    }
    if (P->nvel > 1) {   // non-stationary: each step expands its own direction
        if ((rc = sweep_incremental(P, s, dvt))) return rc;
        if ((rc = sweep_adjoint_steps(P, P->lam[0], hdv, dvt, nullptr, nullptr, s))) return rc;
        return P->p.incompressible ? vec_leray(P, hdv, hdv, s) : BLR_OK;
    }
    if ((rc = dft_expand(P, dvt, P->dv, 0, s))) return rc;
    if ((rc = sweep_incremental(P, s))) return rc;
    if (full && (rc = newton_prep(P, s))) return rc;
    rc = full ? sweep_adjoint_newton(P, P->b, s) : sweep_adjoint(P, P->b, nullptr, P->lam[0], s);
    if (rc) return rc;
    if ((rc = dft_project(P, P->b, hdv, dvt, s))) return rc;
    return P->p.incompressible ? vec_leray(P, hdv, hdv, s) : BLR_OK;
}

namespace {

// PCG (Eq. 55).  The stopping test runs on the device (k_pcg_update), so the
// host queues iteration j + 1 before it looks at iteration j - 1's flag: the GPU
// always has an iteration queued and no iteration waits for a host round trip.
// When the solve stops, the one iteration queued past the stop does nothing
// but a Hessian-vector product into scratch (its update and direction see the
// flag).  Kernels, order and stopping rule are those of the loop written with a
// host test after every update, so the iterates are identical.
// truncate: non-positive curvature ends the solve with the iterate so far (or the
// first direction K~ rhs when no update was made) instead of BLR_ECURV: the
// truncated Newton-CG rule for the full Hessian, which can be indefinite away
// from a minimum (Section 3.4).
int pcg_run(blr_plan *P, const float *rhs, float *x, int maxit, double eta, int *iters,
            double *relres, int *n_hv, cudaStream_t s, bool truncate = false) {
    int rc = pcg_init(P, rhs, x, s);
    if (rc) return rc;
    if ((rc = fetch_scalars(P, s, nullptr))) return rc;
    const double rr0 = P->hsc[SC_RR0];
    if (!(rr0 > 0) || maxit <= 0) {
        if (iters) *iters = 0;
        if (relres) *relres = rr0 > 0 ? 1.0 : 0.0;
        return BLR_OK;
    }
    int *start = P->hlive + 8;   // running, no stop code, no updates
    start[0] = 1;
    start[1] = PCG_RUN;
    start[2] = 0;
    start[3] = 0;
    BLR_CK(cudaMemcpyAsync(P->pcg_live, start, 4 * sizeof(int), cudaMemcpyHostToDevice, s));
    cudaEvent_t ev[2];
    BLR_CK(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    if (cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return BLR_ECUDA;
    }
    for (int j = 0; j < maxit && !rc; ++j) {
        if ((rc = hessvec_here(P, P->pv, P->q, s))) break;
        if ((rc = vec_dot(P, P->pv, P->q, nullptr, P->dsc + SC_PQ, s))) break;
        if ((rc = pcg_update(P, x, s, P->pcg_live, eta))) break;
        if ((rc = pcg_direction(P, s, P->pcg_live))) break;
        if (cudaMemcpyAsync(P->hlive + 4 * (j & 1), P->pcg_live, 4 * sizeof(int),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaEventRecord(ev[j & 1], s) != cudaSuccess) {
            rc = BLR_ECUDA;
            break;
        }
        if (j >= 1) {
            if (cudaEventSynchronize(ev[(j - 1) & 1]) != cudaSuccess) {
                rc = BLR_ECUDA;
                break;
            }
            if (P->hlive[4 * ((j - 1) & 1)] == 0) break;   // stopped by iteration j - 1
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc) return rc;
    BLR_CK(cudaMemcpyAsync(P->hlive, P->pcg_live, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    if ((rc = fetch_scalars(P, s, nullptr))) return rc;   // also waits for the copy above
    const int code = P->hlive[1], it = P->hlive[2];
    if (n_hv) *n_hv += it + ((code == PCG_CURV || code == PCG_NAN_PQ) ? 1 : 0);
    if (iters) *iters = it;
    if (relres) *relres = it > 0 ? P->hsc[SC_REL] : 1.0;
    if (code == PCG_CURV && truncate) {
        if (it == 0)   // p_0 = K~ rhs, untouched since the stop
            BLR_CK(cudaMemcpyAsync(x, P->pv, P->nfloat * sizeof(float), cudaMemcpyDeviceToDevice, s));
        return BLR_OK;
    }
    if (code == PCG_CURV) return BLR_ECURV;
    if (code != PCG_RUN) return BLR_ENAN;
    return BLR_OK;
}

int check_plan(blr_plan_t P) { return P ? BLR_OK : BLR_EINVAL; }

}  // namespace

extern "C" {

int blr_plan_create(const blr_params *p, blr_plan_t *out) { return plan_create(p, true, out); }

}  // extern "C"

int plan_create(const blr_params *p, bool grad_cache, blr_plan **out) {
    if (!out) return BLR_EINVAL;
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    blr_plan *P = new (std::nothrow) blr_plan();
    if (!P) return BLR_ENOMEM;
    P->p = *p;
    P->N1 = p->n[0];
    P->N2 = p->n[1];
    P->N3 = p->n[2];
    P->B1 = p->band[0];
    P->B2 = p->band[1];
    P->B3 = p->band[2];
    P->V = (long long)P->N1 * P->N2 * P->N3;
    P->nb = (long long)P->B1 * P->B2 * P->B3;
    P->nf1 = 6 * P->nb;
    P->nvel = p->nonstationary ? p->nt : 1;
    P->nfloat = P->nvel * P->nf1;
    P->dt = (float)(1.0 / p->nt);
    P->ck = (p->ckpt_every > 0 && p->ckpt_every < p->nt) ? p->ckpt_every : p->nt;
    P->nseg = (int)ceil_div_ll(p->nt, P->ck);
    P->seg_valid = -1;
    P->grid = Grid3{P->N1, P->N2, P->N3, P->V};
    if (cudaGetDevice(&P->device) != cudaSuccess) {
        delete P;
        return BLR_ECUDA;
    }
    sweep_setup(P);   // SM count and sweep shapes (the tensor-core tile shapes use the SM count)
    if (p->precision == BLR_MIXED && !fz_supported(P) && !tc_supported(P)) {
        delete P;
        return BLR_EINVAL;
    }
    P->use_gm = grad_cache && P->sweep_wide && P->ck == p->nt &&
                (p->state_equation == BLR_STATE_IMAGE || !p->nonstationary);
    // L2 persistence for the displacement copy d4 (the autotuner decides whether the
    // sweeps use it): the window covers one step's d4, and the context's
    // persisting set-aside is raised to hold it when the device allows
    P->l2_persist = 0;
    P->l2_win_bytes = 0;
    P->l2_hit = 0.f;
    P->l2_counted = 0;
    if (P->sweep_wide) {
        int max_persist = 0, max_window = 0;
        if (cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, P->device) ==
                cudaSuccess &&
            cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, P->device) ==
                cudaSuccess &&
            max_persist > 0 && max_window > 0) {
            size_t win = (size_t)P->V * sizeof(float4);
            if (win > (size_t)max_window) win = (size_t)max_window;
            size_t aside = win < (size_t)max_persist ? win : (size_t)max_persist;
            P->l2_win_bytes = win;
            if (!l2_acquire(P, aside)) P->l2_win_bytes = 0;
        }
        cudaGetLastError();
    }
    long long nsweep = sweep_blocks(P);
    long long nred = reduce_partials_needed();
    P->npart = (int)(nsweep > nred ? nsweep : nred);
    size_t bytes = layout(P, nullptr);
    char *base = nullptr;
    if (cudaMalloc(&base, bytes) != cudaSuccess) {
        cudaGetLastError();
        l2_release(P);
        delete P;
        return BLR_ENOMEM;
    }
    layout(P, base);
    if (cudaMallocHost(&P->hsc, (SC_COUNT + 1) * sizeof(double)) != cudaSuccess) {
        cudaFree(base);
        l2_release(P);
        delete P;
        return BLR_ENOMEM;
    }
    if (cudaMallocHost(&P->hlive, 12 * sizeof(int)) != cudaSuccess) {
        cudaFreeHost(P->hsc);
        cudaFree(base);
        l2_release(P);
        delete P;
        return BLR_ENOMEM;
    }
    if (cudaMemset(base, 0, bytes) != cudaSuccess ||
        dft_init_tables(P, 0) != BLR_OK || dft_autotune(P, 0) != BLR_OK ||
        (p->precision == BLR_MIXED && tc_init_tables(P, 0) != BLR_OK) ||
        (P->fz_tab[0] && fz_init_tables(P, 0) != BLR_OK) ||
        sweep_autotune(P, 0) != BLR_OK || cudaDeviceSynchronize() != cudaSuccess) {
        cudaFreeHost(P->hlive);
        cudaFreeHost(P->hsc);
        cudaFree(base);
        l2_release(P);
        delete P;
        return BLR_ECUDA;
    }
    *out = P;
    return BLR_OK;
}

extern "C" {

int blr_plan_tuning(blr_plan_t P, int *vals, int n) {
    if (!P || !vals) return BLR_EINVAL;
    int tiles = 0;
    for (int st = 0; st < 5; ++st) tiles |= P->gemm_tile[st] << (3 * st);
    const int v[13] = {P->sweep_wide ? 1 : 0, P->Gm ? 1 : 0, P->bal_adj, P->adj_useg,
                       P->inc_mode, P->bal_inc, P->bal_sweep, P->chunk, P->chunk_adj,
                       P->l2_persist, P->adj2, P->adj_split, tiles};
    for (int i = 0; i < n && i < 13; ++i) vals[i] = v[i];
    return BLR_OK;
}

int blr_plan_set_tuning(blr_plan_t P, const int *vals, int n) {
    if (!P || !vals || n < 11) return BLR_EINVAL;
    // the first two entries describe the plan's buffers and must be unchanged
    if (vals[0] != (P->sweep_wide ? 1 : 0) || vals[1] != (P->Gm ? 1 : 0)) return BLR_EINVAL;
    const int bal_adj = vals[2], useg = vals[3], inc = vals[4], bal_inc = vals[5];
    const int bal_sweep = vals[6], chunk = vals[7], chunk_adj = vals[8], l2 = vals[9], adj2 = vals[10];
    const bool gm = P->Gm != nullptr;
    if (bal_adj < 0 || bal_adj > 4 || (P->sweep_wide && bal_adj < 1)) return BLR_EINVAL;
    if ((useg != 0 && useg != 1) || (useg && !gm)) return BLR_EINVAL;
    if (inc < 0 || inc > 2 || (inc > 0 && !gm)) return BLR_EINVAL;
    if (bal_inc < 0 || bal_inc > 4 || bal_sweep < 0 || bal_sweep > 4) return BLR_EINVAL;
    if (chunk < 1 || chunk > P->N1 || chunk_adj < 1 || chunk_adj > P->N1) return BLR_EINVAL;
    if ((l2 != 0 && l2 != 1) || (l2 && !P->l2_win_bytes)) return BLR_EINVAL;
    if (adj2 < 0 || adj2 > 2 || (adj2 && (!gm || !P->d4 || P->nvel != 1))) return BLR_EINVAL;
    const int split = n >= 12 ? vals[11] : P->adj_split;
    if ((split != 0 && split != 1) || (split && ((!P->lam_keep && !P->rho_keep) || !P->d4 || adj2)))
        return BLR_EINVAL;
    int tiles[5];
    for (int st = 0; st < 5; ++st) tiles[st] = P->gemm_tile[st];
    if (n >= 13) {
        if (vals[12] < 0 || vals[12] >= (1 << 15)) return BLR_EINVAL;
        for (int st = 0; st < 5; ++st) {
            tiles[st] = (vals[12] >> (3 * st)) & 7;
            if (tiles[st] > SG_CANDS) return BLR_EINVAL;
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return BLR_ECUDA;
    P->bal_adj = bal_adj;
    P->adj_useg = useg;
    P->inc_mode = inc;
    P->bal_inc = bal_inc;
    P->bal_sweep = bal_sweep;
    sweep_set_chunk(P, 2, chunk);
    sweep_set_chunk(P, 1, chunk_adj);
    P->l2_persist = l2;
    P->adj2 = adj2;
    P->adj_split = split;
    for (int st = 0; st < 5; ++st) P->gemm_tile[st] = tiles[st];
    return BLR_OK;
}

int blr_plan_destroy(blr_plan_t P) {
    if (!P) return BLR_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(P->device);
    cudaError_t e1 = cudaFree(arena_base(P));
    l2_release(P);   // the last such plan releases the lines and restores the limit
    cudaError_t e2 = cudaFreeHost(P->hsc);
    if (cudaFreeHost(P->hlive) != cudaSuccess) e2 = cudaErrorInvalidValue;
    if (prev >= 0) cudaSetDevice(prev);
    delete P;
    return (e1 == cudaSuccess && e2 == cudaSuccess) ? BLR_OK : BLR_ECUDA;
}

int blr_set_images(blr_plan_t P, const float *I0, const float *I1, blr_stream_t stream) {
    if (check_plan(P) || !I0 || !I1) return BLR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    BLR_CK(cudaMemcpyAsync(P->I0, I0, P->V * sizeof(float), cudaMemcpyDefault, s));
    BLR_CK(cudaMemcpyAsync(P->I1, I1, P->V * sizeof(float), cudaMemcpyDefault, s));
    P->have_state = false;
    P->seg_valid = -1;
    return BLR_OK;
}

int blr_expand(blr_plan_t P, const float *vt, float *v, blr_stream_t stream) {
    if (check_plan(P) || !vt || !v) return BLR_EINVAL;
    return dft_expand(P, vt, v, 0, (cudaStream_t)stream);
}

int blr_project(blr_plan_t P, const float *f, float *ft, blr_stream_t stream) {
    if (check_plan(P) || !f || !ft) return BLR_EINVAL;
    return dft_project(P, f, ft, nullptr, (cudaStream_t)stream);
}

int blr_state(blr_plan_t P, const float *vt, float *m1, double *energy, blr_stream_t stream) {
    if (check_plan(P) || !vt) return BLR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = state_at(P, vt, energy, s);
    if (rc) return rc;
    if (m1)
        BLR_CK(cudaMemcpyAsync(m1, state_slot(P, P->p.nt), P->V * sizeof(float),
                               cudaMemcpyDeviceToDevice, s));
    return BLR_OK;
}

int blr_adjoint(blr_plan_t P, float *b, float *lambda0, blr_stream_t stream) {
    if (check_plan(P) || !b) return BLR_EINVAL;
    if (!P->have_state) return BLR_ESTATE;
    if (P->p.state_equation == BLR_STATE_DEFORMATION)   // rho is a vector: no lambda^0
        return lambda0 ? BLR_EINVAL : sweep_adjoint_def(P, P->rho_nt, b, (cudaStream_t)stream);
    if (P->nvel > 1)   // one body force per step: b holds nt * 3V floats
        return sweep_adjoint_steps(P, P->lam_nt, nullptr, nullptr, b, lambda0, (cudaStream_t)stream);
    return sweep_adjoint(P, b, lambda0, P->lam_nt, (cudaStream_t)stream);
}

int blr_gradient(blr_plan_t P, const float *vt, float *g, double *energy, blr_stream_t stream) {
    if (check_plan(P) || !vt || !g) return BLR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = state_at(P, vt, energy, s);
    if (rc) return rc;
    return gradient_here(P, g, s);
}

int blr_gradient_at_state(blr_plan_t P, float *g, blr_stream_t stream) {
    if (check_plan(P) || !g) return BLR_EINVAL;
    if (!P->have_state) return BLR_ESTATE;
    return gradient_here(P, g, (cudaStream_t)stream);
}

int blr_hessvec(blr_plan_t P, const float *dvt, float *hdv, blr_stream_t stream) {
    if (check_plan(P) || !dvt || !hdv) return BLR_EINVAL;
    if (!P->have_state) return BLR_ESTATE;
    return hessvec_here(P, dvt, hdv, (cudaStream_t)stream);
}

int blr_pcg(blr_plan_t P, const float *rhs, float *x, int maxit, double eta, int *iters,
            double *relres, blr_stream_t stream) {
    if (check_plan(P) || !rhs || !x || maxit < 0) return BLR_EINVAL;
    if (!P->have_state) return BLR_ESTATE;
    return pcg_run(P, rhs, x, maxit, eta, iters, relres, nullptr, (cudaStream_t)stream);
}

int blr_newton(blr_plan_t P, float *vt, int max_newton, int max_pcg, double gtol,
               double forcing, blr_report *rep, blr_stream_t stream) {
    if (check_plan(P) || !vt || max_newton < 0 || max_pcg < 0) return BLR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    blr_report R;
    memset(&R, 0, sizeof(R));
    const size_t vbytes = P->nfloat * sizeof(float);
    int flags = 0, rc;
    // a failure before the first update still reports (status, counts)
    auto fail = [&](int code) {
        R.status = code;
        if (rep) *rep = R;
        return code;
    };
    if (cudaMemsetAsync(P->dstatus, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemcpyAsync(P->vtmp, vt, vbytes, cudaMemcpyDefault, s) != cudaSuccess)
        return fail(BLR_ECUDA);
    if (P->p.incompressible && (rc = vec_leray(P, P->vtmp, P->vtmp, s))) return fail(rc);
    if ((rc = state_at(P, P->vtmp, nullptr, s))) return fail(rc);
    R.n_state = 1;
    if ((rc = gradient_here(P, P->g, s))) return fail(rc);
    if ((rc = vec_maxabs(P, P->g, P->dsc + SC_GINF, s))) return fail(rc);
    if ((rc = vec_dot(P, P->g, P->g, nullptr, P->dsc + SC_DOT, s))) return fail(rc);
    if ((rc = fetch_scalars(P, s, &flags))) return fail(rc);
    if ((rc = flags_to_status(flags))) {
        R.energy0 = R.energy = P->hsc[SC_E];
        return fail(rc);
    }
    double E = P->hsc[SC_E];
    const double g0inf = P->hsc[SC_GINF], g0n = sqrt(P->hsc[SC_DOT]);
    double ginf = g0inf, gn = g0n;
    R.energy0 = E;
    const double c1 = 1e-4;
    for (int it = 0; it < max_newton; ++it) {
        if (!(g0inf > 0) || ginf / g0inf < gtol) break;
        const double eta = forcing >= 0 ? forcing : fmin(0.5, sqrt(gn / g0n));
        // rhs = -g (exact: g + (-2) g)
        if ((rc = vec_axpy(P, P->trial, P->g, P->g, -2.0, s))) break;
        int its = 0;
        double relres = 0;
        rc = pcg_run(P, P->trial, P->step, max_pcg, eta, &its, &relres, &R.n_hessvec, s,
                     P->p.hessian == BLR_NEWTON);
        R.pcg_iters += its;
        if (rc) break;
        if ((rc = vec_dot(P, P->g, P->step, nullptr, P->dsc + SC_DOT, s))) break;
        if ((rc = fetch_scalars(P, s, nullptr))) break;
        const double slope = P->hsc[SC_DOT];
        double eps = 1.0;
        bool accepted = false;
        for (int h = 0; h <= 10; ++h) {
            if ((rc = vec_axpy(P, P->trial, P->vtmp, P->step, eps, s))) break;
            if ((rc = state_at(P, P->trial, nullptr, s))) break;
            ++R.n_state;
            if ((rc = fetch_scalars(P, s, &flags))) break;
            const double Et = P->hsc[SC_E];
            if (flags == 0 && isfinite(Et) && Et <= E + c1 * eps * slope) {
                accepted = true;
                E = Et;
                break;
            }
            eps *= 0.5;
            ++R.n_halvings;
        }
        if (rc) break;
        if (!accepted) {
            // restore the last accepted point as the plan's current point
            if ((rc = state_at(P, P->vtmp, nullptr, s))) break;
            ++R.n_state;
            break;
        }
        if (cudaMemcpyAsync(P->vtmp, P->trial, vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            rc = BLR_ECUDA;
            break;
        }
        ++R.newton_iters;
        if ((rc = gradient_here(P, P->g, s))) break;
        if ((rc = vec_maxabs(P, P->g, P->dsc + SC_GINF, s))) break;
        if ((rc = vec_dot(P, P->g, P->g, nullptr, P->dsc + SC_DOT, s))) break;
        if ((rc = fetch_scalars(P, s, nullptr))) break;
        ginf = P->hsc[SC_GINF];
        gn = sqrt(P->hsc[SC_DOT]);
    }
    if ((cudaMemcpyAsync(vt, P->vtmp, vbytes, cudaMemcpyDefault, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess) && !rc)
        rc = BLR_ECUDA;
    R.energy = E;
    R.grad_inf_rel = g0inf > 0 ? ginf / g0inf : 0.0;
    R.status = rc;
    if (rep) *rep = R;
    return rc;
}

int blr_status(blr_plan_t P, blr_stream_t stream) {
    if (check_plan(P)) return BLR_EINVAL;
    int flags = 0;
    int rc = fetch_scalars(P, (cudaStream_t)stream, &flags);
    if (rc) return rc;
    return flags_to_status(flags);
}

unsigned long long blr_kernel_launches(void) {
    return __atomic_load_n(&g_blr_launches, __ATOMIC_RELAXED);
}

const char *blr_strerror(int code) {
    switch (code) {
        case BLR_OK: return "ok";
        case BLR_EINVAL: return "invalid argument, shape or call order";
        case BLR_ENOMEM: return "device allocation failed";
        case BLR_ECUDA: return "CUDA runtime error";
        case BLR_ECFL: return "displacement per time step reached one voxel (CFL bound)";
        case BLR_ENAN: return "non-finite value";
        case BLR_ESTATE: return "no forward solve at the current point (call blr_state first)";
        case BLR_ECURV: return "PCG met non-positive curvature";
        case BLR_ETIMEOUT: return "a bounded device wait expired (tensor-core stage)";
        default: return "unknown status";
    }
}

}  // extern "C"
