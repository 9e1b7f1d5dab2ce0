// kg_api.cu -- the extern "C" boundary of libkrylovgf (include/krylovgf.h).
// Argument checks and defaults live here; every numerical step runs in the
// kernels of kg_sector.cu, kg_hpsi.cu, kg_krylov.cu and kg_green.cu.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kg_internal.h"

namespace kg {

int propagate(kg_sector* s, double2* x, double dt, int n_steps, const kg_opts* o) {
    if (!x || n_steps < 0) {
        set_error("NULL vector or negative step count");
        return KG_EINVAL;
    }
    if (o->M < 1 || o->M > kMaxM || o->reorth < 0 || o->reorth > 2 || o->schedule < 0 || o->schedule > 7) {
        set_error("bad M or reorth");
        return KG_EINVAL;
    }
    if (n_steps == 0) return KG_OK;
    cudaStream_t st = pick_stream(s, o);
    const int d = (int)s->d;
    Krylov K;
    StepRunner R;
    int rc = krylov_alloc(K, {s}, std::min(o->M, d), s->nsm, o->schedule);
    if (rc == KG_OK) {
        K.hdesc[0].tau = dt;
        rc = krylov_upload(K, st);
    }
    if (rc == KG_OK)
        rc = cudaMemcpyAsync(K.vec(0, 0), x, sizeof(double2) * d, cudaMemcpyDeviceToDevice, st) == cudaSuccess
                 ? KG_OK
                 : KG_ECUDA;
    if (rc == KG_OK) rc = R.init(K, o->reorth, st, o->use_graphs != 0 && n_steps > 1);
    for (int n = 0; rc == KG_OK && n < n_steps; ++n) rc = R.run(st);
    ColScalars h;
    if (rc == KG_OK)
        rc = cudaMemcpyAsync(x, K.vec(0, 0), sizeof(double2) * d, cudaMemcpyDeviceToDevice, st) == cudaSuccess
                 ? KG_OK
                 : KG_ECUDA;
    if (rc == KG_OK)
        rc = cudaMemcpyAsync(&h, K.cs, sizeof(ColScalars), cudaMemcpyDeviceToHost, st) == cudaSuccess ? KG_OK : KG_ECUDA;
    if (rc == KG_OK)
        rc = cudaStreamSynchronize(st) == cudaSuccess ? KG_OK : cuda_fail(cudaGetLastError(), "propagate", __FILE__, __LINE__);
    if (rc == KG_OK && h.status == KG_ENUMERIC) {
        set_error("non-finite value during propagation");
        rc = KG_ENUMERIC;
    }
    R.release();
    krylov_free(K);
    return rc;
}

}  // namespace kg

using namespace kg;

extern "C" {

void kg_opts_default(kg_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->M = 20;
    o->M_gs = 100;
    o->max_restarts = 200;
    o->tol_resid = 1e-12;
    o->reorth = 1;
    o->mem_budget_mb = 0;
    o->schedule = 0;
    o->use_graphs = 1;
    o->dt_internal = 0.0;
    o->seed = 1234ULL;
    o->stream = nullptr;
}

static const kg_opts* opts_or_default(const kg_opts* o, kg_opts* tmp) {
    if (o) return o;
    kg_opts_default(tmp);
    return tmp;
}

int kg_build_sector(int L, int n_up, int n_dn, const double* h_re, const double* h_im, const double* eps,
                    const double* U, kg_sector** out) {
    return sector_build(L, n_up, n_dn, h_re, h_im, eps, U, out);
}

void kg_free_sector(kg_sector* s) {
    if (s && !s->is_child) sector_free(s);
}

int kg_sector_dims(const kg_sector* s, long long* dim, long long* D_up, long long* D_dn) {
    if (!s) {
        set_error("NULL sector");
        return KG_EINVAL;
    }
    if (dim) *dim = s->d;
    if (D_up) *D_up = s->Du;
    if (D_dn) *D_dn = s->Dd;
    return KG_OK;
}

int kg_sector_strings(const kg_sector* s, unsigned int* up_host, unsigned int* dn_host) {
    if (!s) {
        set_error("NULL sector");
        return KG_EINVAL;
    }
    if (up_host) KG_CUDA(cudaMemcpy(up_host, s->up.bits, sizeof(unsigned) * s->Du, cudaMemcpyDeviceToHost));
    if (dn_host) KG_CUDA(cudaMemcpy(dn_host, s->dn.bits, sizeof(unsigned) * s->Dd, cudaMemcpyDeviceToHost));
    return KG_OK;
}

int kg_hpsi(kg_sector* s, const double* x_dev, double* y_dev, void* stream) {
    if (!s || !x_dev || !y_dev || x_dev == y_dev) {
        set_error("NULL or aliased argument");
        return KG_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;  // NULL: the legacy default stream
    return launch_hpsi(s, reinterpret_cast<const double2*>(x_dev), reinterpret_cast<double2*>(y_dev), st);
}

int kg_neighbour_dim(kg_sector* s, int spin, int dagger, long long* dim) {
    if (!s || !dim) {
        set_error("NULL argument");
        return KG_EINVAL;
    }
    kg_sector* n = nullptr;
    KG_TRY(neighbour(s, spin, dagger, &n));
    *dim = n->d;
    return KG_OK;
}

int kg_apply_cop(kg_sector* s, int site, int spin, int dagger, const double* x_dev, double* y_dev, void* stream) {
    if (!s || !x_dev || !y_dev || site < 0 || site >= s->L) {
        set_error("bad argument to kg_apply_cop");
        return KG_EINVAL;
    }
    kg_sector* n = nullptr;
    KG_TRY(neighbour(s, spin, dagger, &n));
    cudaStream_t st = (cudaStream_t)stream;  // NULL: the legacy default stream
    return launch_cop(s, n, site, spin, dagger ? 1 : 0, reinterpret_cast<const double2*>(x_dev),
                      reinterpret_cast<double2*>(y_dev), st);
}

int kg_ground_state(kg_sector* s, const kg_opts* o, double* E0, double* resid, double* gap) {
    if (!s) {
        set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    const int rc = ground_state(s, opts_or_default(o, &tmp));
    if (E0) *E0 = s->E0;
    if (resid) *resid = s->resid;
    if (gap) *gap = s->gap;
    return rc;
}

int kg_copy_ground_state(kg_sector* s, double* psi, int to_host) {
    if (!s || !psi || !s->has_gs) {
        set_error("no ground state cached (call kg_ground_state first)");
        return KG_EINVAL;
    }
    KG_CUDA(cudaMemcpy(psi, s->gs, sizeof(double2) * s->d, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice));
    return KG_OK;
}

int kg_propagate(kg_sector* s, double* x_dev, double dt, int n_steps, const kg_opts* o) {
    if (!s) {
        set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    return propagate(s, reinterpret_cast<double2*>(x_dev), dt, n_steps, opts_or_default(o, &tmp));
}

int kg_green_equilibrium(kg_sector* s, const int* orb, int n_orb, double dt, int n_steps, const kg_opts* o,
                         double* G_gtr, double* G_les) {
    if (!s) {
        set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    return green_equilibrium(s, orb, n_orb, dt, n_steps, opts_or_default(o, &tmp), G_gtr, G_les);
}

int kg_green_equilibrium_batched(kg_sector* const* s, int n_inst, const int* orb, int n_orb, double dt, int n_steps,
                                 const kg_opts* o, double* G_gtr, double* G_les, int* status) {
    kg_opts tmp;
    return green_equilibrium_batched(s, n_inst, orb, n_orb, dt, n_steps, opts_or_default(o, &tmp), G_gtr, G_les,
                                     status);
}

int kg_green_keldysh(kg_sector* H_ini, kg_sector* H_fin, const int* orb, int n_orb, double dt, int n_t,
                     const kg_opts* o, double* G_les, double* G_gtr) {
    if (!H_ini || !H_fin) {
        set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    return green_keldysh(H_ini, H_fin, orb, n_orb, dt, n_t, opts_or_default(o, &tmp), G_les, G_gtr);
}

int kg_green_keldysh_td(kg_sector* H_ini, kg_sector* H_fin, const int* orb, int n_orb, double dt, int n_t,
                        const double* dparams, const kg_opts* o, double* G_les, double* G_gtr) {
    if (!H_ini || !H_fin || (!dparams && n_t > 1)) {
        set_error("NULL sector or drive");
        return KG_EINVAL;
    }
    kg_opts tmp;
    return green_keldysh(H_ini, H_fin, orb, n_orb, dt, n_t, opts_or_default(o, &tmp), G_les, G_gtr,
                         n_t > 1 ? dparams : nullptr);
}

int kg_keldysh_create_td(kg_sector* H_ini, kg_sector* H_fin, const int* orb, int n_orb, double dt, int n_t,
                         const double* dparams, const kg_opts* o, kg_keldysh** out) {
    if (!H_ini || !H_fin || !out || (!dparams && n_t > 1)) {
        set_error("NULL argument");
        return KG_EINVAL;
    }
    kg_opts tmp;
    return keldysh_create(H_ini, H_fin, orb, n_orb, dt, n_t, opts_or_default(o, &tmp), out,
                          n_t > 1 ? dparams : nullptr);
}

int kg_green_four_time(kg_sector* H_ini, kg_sector* H_fin, const int* ops, double dt, int n_t, const kg_opts* o,
                       double* G) {
    if (!H_ini || !H_fin) {
        set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    return green_four_time(H_ini, H_fin, ops, dt, n_t, opts_or_default(o, &tmp), G);
}

int kg_keldysh_create(kg_sector* H_ini, kg_sector* H_fin, const int* orb, int n_orb, double dt, int n_t,
                      const kg_opts* o, kg_keldysh** out) {
    if (!H_ini || !H_fin || !out) {
        set_error("NULL argument");
        return KG_EINVAL;
    }
    kg_opts tmp;
    return keldysh_create(H_ini, H_fin, orb, n_orb, dt, n_t, opts_or_default(o, &tmp), out);
}

int kg_keldysh_row(kg_keldysh* K, int k, double* G_les_kk, double* G_gtr_kk) {
    if (!K) {
        set_error("NULL handle");
        return KG_EINVAL;
    }
    return keldysh_row(K, k, G_les_kk, G_gtr_kk);
}

int kg_keldysh_gram(kg_keldysh* K, double* G_les, double* G_gtr) {
    if (!K) {
        set_error("NULL handle");
        return KG_EINVAL;
    }
    return keldysh_gram(K, G_les, G_gtr);
}

int kg_keldysh_plan(const kg_keldysh* K, int* phi_on_host, int* stores_kept, int* planes, long long* budget) {
    if (!K) {
        set_error("NULL Keldysh handle");
        return KG_EINVAL;
    }
    return keldysh_plan(K, phi_on_host, stores_kept, planes, budget);
}

int kg_keldysh_get_phi(kg_keldysh* K, int k, double* phi_host) {
    if (!K || !phi_host) {
        set_error("NULL argument");
        return KG_EINVAL;
    }
    return keldysh_phi(K, k, phi_host, nullptr);
}

int kg_keldysh_set_phi(kg_keldysh* K, int k, const double* phi_host) {
    if (!K || !phi_host) {
        set_error("NULL argument");
        return KG_EINVAL;
    }
    return keldysh_phi(K, k, nullptr, phi_host);
}

void kg_keldysh_free(kg_keldysh* K) { keldysh_free(K); }

const char* kg_strerror(int code) {
    switch (code) {
        case KG_OK: return "success";
        case KG_EINVAL: return "invalid argument";
        case KG_ENOMEM: return "out of memory";
        case KG_ENOCONV: return "ground state not converged";
        case KG_EDEGEN: return "ground state degenerate";
        case KG_EBREAKDOWN: return "Krylov breakdown (invariant subspace)";
        case KG_ENUMERIC: return "non-finite value";
        case KG_ETIMEOUT: return "device wait timed out";
        case KG_ECUDA: return "CUDA error";
        default: return "unknown status";
    }
}

const char* kg_last_error(void) { return last_error(); }

unsigned long long kg_launch_count(void) { return launch_count(); }

}  // extern "C"
