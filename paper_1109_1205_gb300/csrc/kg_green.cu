// kg_green.cu -- the Green's-function drivers.
//
// Equilibrium (Section 3, Eqs. (psit), (psigreen), eta = 0; hole part after
// Eq. (gomega)):  the columns c^dag_a'|0> (particle) and c_a|0> (hole) are
// propagated together, one batched Krylov step per time step, and their
// overlaps with the fixed vectors c^dag_a|0> / c_a'|0> are fused into the
// combination pass of every step.  The batched form runs the columns of many
// instances (different sectors and dimensions) in the same launches.
//
// Nonequilibrium (Section 4, steps (i)-(iv)): Phi(t_k) = e^{-iHt_k}|0> is
// stored for every grid time; row k of step (iii) starts the columns
// c_a Phi(t_k) (or c^dag_a Phi(t_k)) and propagates them backward by t_k;
// step (iv) is a Hermitian Gram matrix over all stored columns.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "kg_internal.h"

namespace kg {

int StepRunner::init(Krylov& k, int reorth_mode, cudaStream_t st, bool use_graph) {
    release();
    K = &k;
    reorth = reorth_mode;
    KG_TRY(prepare_step(k, reorth));
    if (!use_graph || profiling()) return KG_OK;
    cudaGraph_t g = nullptr;
    KG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    const int rc = enqueue_step(*K, reorth, st);
    set_capturing(false);
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc != KG_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    cudaGraphGetNodes(g, nullptr, &nodes);
    const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate", __FILE__, __LINE__);
    graph = true;
    return KG_OK;
}

int StepRunner::run(cudaStream_t st) {
    if (!graph || profiling()) return enqueue_step(*K, reorth, st);
    KG_CUDA(cudaGraphLaunch(exec, st));
    count_launch(nodes);
    return KG_OK;
}

void StepRunner::release() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    graph = false;
}

static int ensure_gs(kg_sector* s, const kg_opts* o) {
    if (s->has_gs) return KG_OK;
    return ground_state(s, o);
}

static void groups(const int* orb, int n_orb, std::vector<int> idx[2]) {
    idx[0].clear();
    idx[1].clear();
    for (int a = 0; a < n_orb; ++a) idx[orb[2 * a + 1]].push_back(a);
}

static int check_orbitals(const kg_sector* s, const int* orb, int n_orb) {
    if (!orb || n_orb < 1) {
        set_error("empty orbital list");
        return KG_EINVAL;
    }
    for (int a = 0; a < n_orb; ++a)
        if (orb[2 * a] < 0 || orb[2 * a] >= s->L || (orb[2 * a + 1] != 0 && orb[2 * a + 1] != 1)) {
            set_error("orbital %d = (%d,%d) out of range", a, orb[2 * a], orb[2 * a + 1]);
            return KG_EINVAL;
        }
    std::vector<int> idx[2];
    groups(orb, n_orb, idx);
    if ((int)idx[0].size() > kMaxOv || (int)idx[1].size() > kMaxOv) {
        set_error("at most %d orbitals per spin", kMaxOv);
        return KG_EINVAL;
    }
    return KG_OK;
}

static int check_opts(const kg_opts* o) {
    if (o->M < 1 || o->M > kMaxM) {
        set_error("M must be in [1, %d]", kMaxM);
        return KG_EINVAL;
    }
    if (o->reorth < 0 || o->reorth > 2) {
        set_error("reorth must be 0, 1 or 2");
        return KG_EINVAL;
    }
    if (o->schedule < 0 || o->schedule > 7) {
        set_error("schedule must be in [0, 7]");
        return KG_EINVAL;
    }
    return KG_OK;
}

// ------------------------------------------------------------ equilibrium
// One (instance, spin, kind) group of columns: the na start vectors
// c^dag_p|0> (kind 1, forward in time) or c_p|0> (kind 0, backward) in the
// neighbour sector, which are also the overlap partners of every step.
struct EqGroup {
    int inst = 0, spin = 0, dagger = 0;
    std::vector<int> idx;      // orbital indices of this spin
    kg_sector* nb = nullptr;
    double2* chi = nullptr;    // [na][dn]
    int col0 = 0;              // first column of the group in the batch
    size_t ov0 = 0;            // first overlap entry of the group
};

static void eq_groups(std::vector<EqGroup>& out, std::vector<const kg_sector*>& cols, kg_sector* s, int inst,
                      const int* orb, int n_orb) {
    std::vector<int> idx[2];
    groups(orb, n_orb, idx);
    for (int spin = 0; spin < 2; ++spin) {
        if (idx[spin].empty()) continue;
        for (int dagger = 1; dagger >= 0; --dagger) {
            kg_sector* nb = nullptr;
            if (neighbour(s, spin, dagger, &nb) != KG_OK) continue;  // empty/full band: that part is zero
            EqGroup g;
            g.inst = inst;
            g.spin = spin;
            g.dagger = dagger;
            g.idx = idx[spin];
            g.nb = nb;
            g.col0 = (int)cols.size();
            for (size_t a = 0; a < g.idx.size(); ++a) cols.push_back(nb);
            out.push_back(g);
        }
    }
}

// Builds the start vectors, propagates every column of the batch n_steps
// times and leaves the raw overlaps in ov: group g's column a has its rows
// [rows][na] at g.ov0 + a*rows*na.  With `tune`, the work-list scale is first
// chosen by timing two steps per candidate (the autotuner).
static int eq_run(std::vector<EqGroup>& G, const std::vector<kg_sector*>& inst, const int* orb, Krylov& K,
                  double2* ov, int rows, double dt, int n_steps, const kg_opts* o, bool tune, cudaStream_t st) {
    size_t off = 0;
    for (auto& g : G) {
        const int na = (int)g.idx.size(), dn = (int)g.nb->d;
        kg_sector* s = inst[g.inst];
        for (int a = 0; a < na; ++a)
            KG_TRY(launch_cop(s, g.nb, orb[2 * g.idx[a]], g.spin, g.dagger, s->gs, g.chi + (size_t)a * dn, st));
        g.ov0 = off;
        for (int a = 0; a < na; ++a) {
            ColDesc& D = K.hdesc[g.col0 + a];
            D.tau = g.dagger ? dt : -dt;  // particle: e^{-iHt}; hole: e^{+iHt}
            D.ov = g.chi;
            D.n_ov = na;
            D.ov_stride = dn;
            D.ov_out = ov + off;
            D.ov_rows = rows;
            off += (size_t)rows * na;
        }
    }
    KG_TRY(krylov_upload(K, st));
    // row 0 (t = 0): <chi_a | chi_b> of every group
    for (auto& g : G) {
        const int na = (int)g.idx.size(), dn = (int)g.nb->d;
        KG_TRY(launch_inner_lib(g.chi, na, g.chi, na, dn, ov + g.ov0, rows * na, st));
    }
    auto load_start = [&]() -> int {
        for (auto& g : G) {
            const int na = (int)g.idx.size(), dn = (int)g.nb->d;
            for (int a = 0; a < na; ++a)
                KG_CUDA(cudaMemcpyAsync(K.vec(g.col0 + a, 0), g.chi + (size_t)a * dn, sizeof(double2) * dn,
                                        cudaMemcpyDeviceToDevice, st));
        }
        return launch_set_slots(K, 1, st);
    };
    if (n_steps == 0) return KG_OK;
    StepRunner R;
    const bool graphs = o->use_graphs != 0;
    if (tune && n_steps > 4 && graphs && !profiling()) {
        // autotuner: work-list size relative to one wave, timed on two steps
        const double cands[3] = {0.5, 1.0, 2.0};
        double best_t = 1e300, best = 1.0;
        cudaEvent_t e0, e1;
        KG_CUDA(cudaEventCreate(&e0));
        KG_CUDA(cudaEventCreate(&e1));
        for (double c : cands) {
            K.wave_scale = c;
            KG_TRY(load_start());
            KG_TRY(R.init(K, o->reorth, st, true));
            KG_TRY(R.run(st));
            cudaEventRecord(e0, st);
            KG_TRY(R.run(st));
            KG_TRY(R.run(st));
            cudaEventRecord(e1, st);
            KG_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_t) {
                best_t = ms;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        K.wave_scale = best;
    }
    KG_TRY(load_start());
    int rc = R.init(K, o->reorth, st, graphs);
    for (int k = 1; rc == KG_OK && k <= n_steps; ++k) rc = R.run(st);
    R.release();
    return rc;
}

// Fine output grid (Section 3: Eq. (udelta) evaluated at several times from
// one Krylov space).  Each Krylov space, built from psi(t) with step `fine`
// dt, serves the times t + q dt, q = 1..fine: psi(t + q dt) = sum_k c^(q)_k V_k
// with c^(q) = beta0 e^{-iT q dt} e_1 (one multi-time step exponential), so
// the overlaps with the start vectors are the small products
// sum_k c^(q)_k <chi_a | V_k> -- the <chi_a | V_k> are one overlap launch per
// step.  Fills ov exactly as eq_run does.
static int eq_run_fine(std::vector<EqGroup>& G, const std::vector<kg_sector*>& inst, const int* orb, Krylov& K,
                       double2* ov, int rows, double dt, int n_steps, int fine, const kg_opts* o, cudaStream_t st) {
    const int B = K.B, MK = K.M + 1;
    size_t off = 0;
    int na_max = 1;
    for (auto& g : G) {
        const int na = (int)g.idx.size(), dn = (int)g.nb->d;
        na_max = std::max(na_max, na);
        kg_sector* s = inst[g.inst];
        for (int a = 0; a < na; ++a)
            KG_TRY(launch_cop(s, g.nb, orb[2 * g.idx[a]], g.spin, g.dagger, s->gs, g.chi + (size_t)a * dn, st));
        g.ov0 = off;
        off += (size_t)na * rows * na;
        KG_TRY(launch_inner_lib(g.chi, na, g.chi, na, dn, ov + g.ov0, rows * na, st));  // row 0
        for (int a = 0; a < na; ++a)
            KG_CUDA(cudaMemcpyAsync(K.vec(g.col0 + a, 0), g.chi + (size_t)a * dn, sizeof(double2) * dn,
                                    cudaMemcpyDeviceToDevice, st));
    }
    if (n_steps == 0) return KG_OK;
    double2 *P = nullptr, *cq = nullptr;
    double* taus = nullptr;
    auto release = [&](int rc) {
        cudaFree(P);
        cudaFree(cq);
        cudaFree(taus);
        return rc;
    };
    if (cudaMalloc(&P, sizeof(double2) * (size_t)B * MK * na_max) != cudaSuccess ||
        cudaMalloc(&cq, sizeof(double2) * (size_t)B * fine * K.M) != cudaSuccess ||
        cudaMalloc(&taus, sizeof(double) * (size_t)B * fine) != cudaSuccess) {
        set_error("fine-grid workspace allocation failed");
        return release(KG_ENOMEM);
    }
    std::vector<double2> hP((size_t)B * MK * na_max), hc((size_t)B * fine * K.M), hov(off);
    KG_CUDA(cudaMemcpyAsync(hov.data(), ov, sizeof(double2) * off, cudaMemcpyDeviceToHost, st));  // row 0
    std::vector<ColScalars> hcs(B);
    std::vector<double> ht((size_t)B * fine);
    int nq_prev = -1;
    for (int k0 = 0; k0 < n_steps; k0 += fine) {
        const int nq = std::min(fine, n_steps - k0);
        if (nq != nq_prev) {
            for (auto& g : G)
                for (size_t a = 0; a < g.idx.size(); ++a)
                    for (int q = 0; q < nq; ++q)
                        ht[(size_t)(g.col0 + a) * nq + q] = (g.dagger ? dt : -dt) * (q + 1);
            if (cudaMemcpyAsync(taus, ht.data(), sizeof(double) * B * nq, cudaMemcpyHostToDevice, st) != cudaSuccess)
                return release(KG_ECUDA);
            nq_prev = nq;
        }
        int rc = build_space(K, o->reorth, st);
        // <chi_a | V_k> of every column, then c^(q) for every column and time
        for (auto& g : G) {
            const int na = (int)g.idx.size(), dn = (int)g.nb->d;
            for (int a = 0; rc == KG_OK && a < na; ++a)
                rc = launch_inner_lib(g.chi, na, K.vec(g.col0 + a, 0), MK, dn, P + (size_t)(g.col0 + a) * MK * na_max,
                                      na_max, st);
        }
        if (rc == KG_OK) rc = launch_tridiag_multi(K, taus, nq, cq, st);
        if (rc != KG_OK) return release(rc);
        if (cudaMemcpyAsync(hP.data(), P, sizeof(double2) * hP.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hc.data(), cq, sizeof(double2) * (size_t)B * nq * K.M, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(hcs.data(), K.cs, sizeof(ColScalars) * B, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return release(cuda_fail(cudaGetLastError(), "fine-grid readback", __FILE__, __LINE__));
        for (auto& g : G) {
            const int na = (int)g.idx.size();
            for (int bcol = 0; bcol < na; ++bcol) {
                const int b = g.col0 + bcol, m = hcs[b].m_eff;
                for (int q = 0; q < nq; ++q)
                    for (int a = 0; a < na; ++a) {
                        std::complex<double> acc(0.0, 0.0);
                        for (int k = 0; k < m; ++k) {
                            const double2 c = hc[((size_t)b * nq + q) * K.M + k];
                            const double2 pv = hP[((size_t)b * MK + k) * na_max + a];
                            acc += std::complex<double>(c.x, c.y) * std::complex<double>(pv.x, pv.y);
                        }
                        hov[g.ov0 + ((size_t)bcol * rows + k0 + 1 + q) * na + a] = make_double2(acc.real(), acc.imag());
                    }
            }
        }
        // psi(t + nq dt) = V c^(nq) becomes the next start vector
        if (cudaMemcpy2DAsync(reinterpret_cast<char*>(K.cs) + offsetof(ColScalars, c), sizeof(ColScalars),
                              cq + (size_t)(nq - 1) * K.M, sizeof(double2) * nq * K.M, sizeof(double2) * K.M, B,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return release(KG_ECUDA);
        rc = launch_combine(K, st);
        if (rc != KG_OK) return release(rc);
    }
    if (cudaMemcpyAsync(ov, hov.data(), sizeof(double2) * off, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return release(KG_ECUDA);
    return release(KG_OK);
}

// G entries of one instance from the raw overlaps (host): ov[b][k][a] =
// <vec_a | propagated vec_b at t_k>; particle gives G^>_{a b}, hole G^<_{b a}.
static void eq_assemble(const EqGroup& g, const std::vector<double2>& hov, int rows, double dt, double E0, int n_orb,
                        double* G_gtr, double* G_les) {
    const int na = (int)g.idx.size();
    for (int k = 0; k < rows; ++k) {
        const double t = dt * k;
        const std::complex<double> ph = g.dagger ? std::complex<double>(0.0, -1.0) * std::exp(std::complex<double>(0.0, E0 * t))
                                                 : std::complex<double>(0.0, 1.0) * std::exp(std::complex<double>(0.0, -E0 * t));
        for (int bcol = 0; bcol < na; ++bcol)
            for (int a = 0; a < na; ++a) {
                const double2 v = hov[g.ov0 + ((size_t)bcol * rows + k) * na + a];
                const std::complex<double> val = ph * std::complex<double>(v.x, v.y);
                const int r = g.dagger ? g.idx[a] : g.idx[bcol];
                const int c = g.dagger ? g.idx[bcol] : g.idx[a];
                double* G = g.dagger ? G_gtr : G_les;
                G[((size_t)k * n_orb * n_orb + (size_t)r * n_orb + c) * 2] = val.real();
                G[((size_t)k * n_orb * n_orb + (size_t)r * n_orb + c) * 2 + 1] = val.imag();
            }
    }
}

// Equilibrium G of n_inst sectors (one instance when n_inst = 1), every
// column of every instance in one batch.  status[i] receives the ground-state
// status of instance i (its G stays zero unless KG_OK).
static int green_eq_batch(kg_sector* const* sv, int n_inst, const int* orb, int n_orb, double dt, int n_steps,
                          const kg_opts* o, double* G_gtr, double* G_les, int* status, bool tune, int fine = 0) {
    KG_TRY(check_opts(o));
    if (n_steps < 0 || !G_gtr || !G_les || n_inst < 1) {
        set_error("bad n_steps, n_inst or NULL output");
        return KG_EINVAL;
    }
    for (int i = 0; i < n_inst; ++i) {
        if (!sv[i]) {
            set_error("NULL sector %d", i);
            return KG_EINVAL;
        }
        KG_TRY(check_orbitals(sv[i], orb, n_orb));
    }
    const int rows = n_steps + 1;
    const size_t per_inst = (size_t)rows * n_orb * n_orb * 2;
    std::memset(G_gtr, 0, sizeof(double) * per_inst * n_inst);
    std::memset(G_les, 0, sizeof(double) * per_inst * n_inst);
    std::vector<kg_sector*> inst(sv, sv + n_inst);
    std::vector<EqGroup> G;
    std::vector<const kg_sector*> cols;
    int first_err = KG_OK;
    for (int i = 0; i < n_inst; ++i) {
        const int r = ensure_gs(inst[i], o);
        if (status) status[i] = r;
        if (r != KG_OK) {
            if (first_err == KG_OK) first_err = r;
            continue;
        }
        eq_groups(G, cols, inst[i], i, orb, n_orb);
    }
    if (n_inst == 1 && first_err != KG_OK) return first_err;
    if (cols.empty()) return n_inst == 1 ? KG_OK : first_err;
    cudaStream_t st = pick_stream(inst[0], o);
    // every column keeps M; a sector smaller than M ends its space by a happy
    // breakdown (the recursion is exact once it spans the sector)
    const int Mb = o->M;
    Krylov K;
    int rc = krylov_alloc(K, cols, Mb, inst[0]->nsm, o->schedule);
    size_t n_ov = 0;
    for (auto& g : G) {
        const size_t na = g.idx.size();
        n_ov += na * rows * na;
        if (rc == KG_OK && cudaMalloc(&g.chi, sizeof(double2) * na * g.nb->d) != cudaSuccess) rc = KG_ENOMEM;
    }
    double2* ov = nullptr;
    if (rc == KG_OK && cudaMalloc(&ov, sizeof(double2) * std::max<size_t>(1, n_ov)) != cudaSuccess) rc = KG_ENOMEM;
    if (rc == KG_OK)
        rc = fine > 0 ? eq_run_fine(G, inst, orb, K, ov, rows, dt, n_steps, fine, o, st)
                      : eq_run(G, inst, orb, K, ov, rows, dt, n_steps, o, tune, st);
    std::vector<double2> hov(n_ov);
    if (rc == KG_OK &&
        (cudaMemcpyAsync(hov.data(), ov, sizeof(double2) * n_ov, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
        rc = cuda_fail(cudaGetLastError(), "overlap readback", __FILE__, __LINE__);
    std::vector<ColScalars> hcs;
    if (rc == KG_OK) {
        hcs.resize(K.B);
        if (cudaMemcpy(hcs.data(), K.cs, sizeof(ColScalars) * K.B, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = KG_ECUDA;
    }
    if (rc == KG_OK) {
        for (auto& g : G) {
            bool bad = false;
            for (size_t a = 0; a < g.idx.size(); ++a) bad |= hcs[g.col0 + a].status == KG_ENUMERIC;
            if (bad) {
                if (status) status[g.inst] = KG_ENUMERIC;
                if (n_inst == 1) {
                    set_error("non-finite value during propagation");
                    rc = KG_ENUMERIC;
                }
                continue;
            }
            eq_assemble(g, hov, rows, dt, inst[g.inst]->E0, n_orb, G_gtr + per_inst * g.inst,
                        G_les + per_inst * g.inst);
        }
    }
    for (auto& g : G) cudaFree(g.chi);
    cudaFree(ov);
    krylov_free(K);
    return rc;
}

int green_equilibrium(kg_sector* s, const int* orb, int n_orb, double dt, int n_steps, const kg_opts* o,
                      double* G_gtr, double* G_les) {
    return green_eq_batch(&s, 1, orb, n_orb, dt, n_steps, o, G_gtr, G_les, nullptr, false);
}

int green_equilibrium_batched(kg_sector* const* s, int n_inst, const int* orb, int n_orb, double dt, int n_steps,
                              const kg_opts* o, double* G_gtr, double* G_les, int* status) {
    if (!s || n_inst < 1) {
        set_error("no instances");
        return KG_EINVAL;
    }
    return green_eq_batch(s, n_inst, orb, n_orb, dt, n_steps, o, G_gtr, G_les, status, true);
}

// --------------------------------------------------- Gram, step (iv)
// G[p][q] = <X_p | X_q> for the upper-triangle tiles (p tile <= q tile) of a
// set of nv vectors of dimension d, FP64 on the CUDA cores.  32 x 32 output
// tile per block, 2 x 2 complex outputs per thread, 16-element slabs of the
// vectors staged in shared memory, split over d by gridDim.z (partials).
constexpr int kGT = 32, kGK = 16;

__global__ void __launch_bounds__(256) k_gram(const double2* __restrict__ X, int nv, int d, int ntile,
                                              const int2* __restrict__ tiles, double2* __restrict__ part) {
    __shared__ double2 As[kGT][kGK + 1];
    __shared__ double2 Bs[kGK][kGT + 1];
    const int2 tl = tiles[blockIdx.x];
    const int p0 = tl.x * kGT, q0 = tl.y * kGT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int z = blockIdx.y, nz = gridDim.y;
    const int slab = (d + nz - 1) / nz;
    const int i_begin = z * slab, i_end = min(d, i_begin + slab);
    double2 acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc[a][b] = make_double2(0.0, 0.0);
    for (int i0 = i_begin; i0 < i_end; i0 += kGK) {
        // 32 rows x 16 elements of each operand: 2 loads per thread
        for (int t = threadIdx.x; t < kGT * kGK; t += 256) {
            const int r = t / kGK, c = t % kGK;
            const int i = i0 + c;
            const int p = p0 + r, q = q0 + r;
            As[r][c] = (p < nv && i < i_end) ? X[(size_t)p * d + i] : make_double2(0.0, 0.0);
            Bs[c][r] = (q < nv && i < i_end) ? X[(size_t)q * d + i] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kGK; ++c) {
            const double2 a0 = As[ty][c], a1 = As[ty + 16][c];
            const double2 b0 = Bs[c][tx], b1 = Bs[c][tx + 16];
            acc[0][0].x = fma(a0.x, b0.x, fma(a0.y, b0.y, acc[0][0].x));
            acc[0][0].y = fma(a0.x, b0.y, fma(-a0.y, b0.x, acc[0][0].y));
            acc[0][1].x = fma(a0.x, b1.x, fma(a0.y, b1.y, acc[0][1].x));
            acc[0][1].y = fma(a0.x, b1.y, fma(-a0.y, b1.x, acc[0][1].y));
            acc[1][0].x = fma(a1.x, b0.x, fma(a1.y, b0.y, acc[1][0].x));
            acc[1][0].y = fma(a1.x, b0.y, fma(-a1.y, b0.x, acc[1][0].y));
            acc[1][1].x = fma(a1.x, b1.x, fma(a1.y, b1.y, acc[1][1].x));
            acc[1][1].y = fma(a1.x, b1.y, fma(-a1.y, b1.x, acc[1][1].y));
        }
        __syncthreads();
    }
    double2* out = part + (size_t)z * ntile * kGT * kGT + (size_t)blockIdx.x * kGT * kGT;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) out[(ty + 16 * a) * kGT + tx + 16 * b] = acc[a][b];
}

__global__ void k_gram_reduce(const double2* part, int nz, int ntile, const int2* tiles, int nv, double2* G) {
    const int t = blockIdx.x, e = threadIdx.x + blockDim.x * blockIdx.y;
    if (e >= kGT * kGT) return;
    double2 s = make_double2(0.0, 0.0);
    for (int z = 0; z < nz; ++z) {
        const double2 v = part[((size_t)z * ntile + t) * kGT * kGT + e];
        s.x += v.x;
        s.y += v.y;
    }
    const int2 tl = tiles[t];
    const int p = tl.x * kGT + e / kGT, q = tl.y * kGT + e % kGT;
    if (p < nv && q < nv) G[(size_t)p * nv + q] = s;
}

// Full Hermitian Gram matrix (host, nv x nv complex) of the nv vectors X.
int gram(const double2* X, int nv, int d, int nsm, std::vector<std::complex<double>>& G, cudaStream_t st) {
    const int nt = (nv + kGT - 1) / kGT;
    std::vector<int2> tiles;
    for (int a = 0; a < nt; ++a)
        for (int b = a; b < nt; ++b) tiles.push_back(make_int2(a, b));
    const int ntile = (int)tiles.size();
    int nz = std::max(1, std::min((nsm * 2 + ntile - 1) / ntile, (d + 4095) / 4096));
    int2* dt = nullptr;
    double2 *part = nullptr, *dG = nullptr;
    int rc = KG_OK;
    if (cudaMalloc(&dt, sizeof(int2) * ntile) != cudaSuccess ||
        cudaMalloc(&part, sizeof(double2) * (size_t)nz * ntile * kGT * kGT) != cudaSuccess ||
        cudaMalloc(&dG, sizeof(double2) * (size_t)nv * nv) != cudaSuccess)
        rc = KG_ENOMEM;
    if (rc == KG_OK) {
        cudaMemcpyAsync(dt, tiles.data(), sizeof(int2) * ntile, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(dG, 0, sizeof(double2) * (size_t)nv * nv, st);
        ProfScope ps("gram", st);
        k_gram<<<dim3(ntile, nz), 256, 0, st>>>(X, nv, d, ntile, dt, part);
        count_launch();
        k_gram_reduce<<<dim3(ntile, (kGT * kGT + 255) / 256), 256, 0, st>>>(part, nz, ntile, dt, nv, dG);
        count_launch();
        std::vector<double2> h((size_t)nv * nv);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(h.data(), dG, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), "gram", __FILE__, __LINE__);
        G.assign((size_t)nv * nv, 0.0);
        for (int p = 0; p < nv; ++p)
            for (int q = p; q < nv; ++q) {
                const double2 v = h[(size_t)p * nv + q];
                G[(size_t)p * nv + q] = std::complex<double>(v.x, v.y);
                G[(size_t)q * nv + p] = std::complex<double>(v.x, -v.y);
            }
    }
    cudaFree(dt);
    cudaFree(part);
    cudaFree(dG);
    return rc;
}

// ---------------------------- time-dependent Lanczos with f restarts
// Eigen-decomposition of a real symmetric tridiagonal matrix by the implicit
// QL method with Wilkinson-type shifts, eigenvectors accumulated by the
// Givens rotations (Golub and Van Loan, Section 8.3).  d[0..m): diagonal,
// e[0..m): e[k] couples k and k+1 (e[m-1] unused).  On return d holds the
// eigenvalues and Z[k * m + j] the k-th component of eigenvector j.
static void tql_eigen(std::vector<double>& d, std::vector<double>& e, int m, std::vector<double>& Z) {
    Z.assign((size_t)m * m, 0.0);
    for (int k = 0; k < m; ++k) Z[(size_t)k * m + k] = 1.0;
    if (m > 0) e[m - 1] = 0.0;
    const double eps = 2.220446049250313e-16;
    for (int l = 0; l < m; ++l) {
        for (int iter = 0; iter < 64; ++iter) {
            int mm = l;
            for (; mm < m - 1; ++mm)
                if (std::fabs(e[mm]) <= eps * (std::fabs(d[mm]) + std::fabs(d[mm + 1]))) break;
            if (mm == l) break;
            // shift from the leading 2x2 block
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[mm] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = mm - 1;
            bool early = false;
            for (; i >= l; --i) {
                const double ff = s * e[i], b = c * e[i];
                r = std::hypot(ff, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    e[mm] = 0.0;
                    early = true;
                    break;
                }
                s = ff / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                for (int k = 0; k < m; ++k) {
                    double* row = Z.data() + (size_t)k * m;
                    const double zf = row[i + 1];
                    row[i + 1] = s * row[i] + c * zf;
                    row[i] = c * row[i] - s * zf;
                }
            }
            if (early) continue;
            d[l] -= p;
            e[l] = g;
            e[mm] = 0.0;
        }
    }
}

// Section 3, Fig. 1 and Eqs. (newstate), (udelta): the equilibrium G(t) on
// t_k = k dt, k = 0..f q, with one Krylov space of dimension n per restart
// interval Delta t = q dt.  Within an interval the space built from psi(t_r)
// gives psi(t_r + tau) = ||psi|| V Z e^{-i Theta tau} Z^T e_1 (Eq. (udelta),
// the eigen-decomposition T = Z Theta Z^T by implicit QL on the host) at
// every output time, and psi(t_r + Delta t) starts the next space.  f = 1 is
// the conventional Lanczos Green's function in the time domain (Eq. (res));
// the paper's Fig. 1 compares f = 1, 100 and 1000 at n = 100.
static int green_restarted(kg_sector* s, const int* orb, int n_orb, int n, int f, int q, double dt,
                           const kg_opts* o, double* G_gtr, double* G_les) {
    if (n < 1 || n > kMaxMgs - 1 || f < 1 || q < 1 || !(dt > 0.0) || !std::isfinite(dt) || !G_gtr || !G_les ||
        (long long)f * q > (1ll << 28) || o->reorth < 0 || o->reorth > 2 || o->schedule < 0 || o->schedule > 7) {
        set_error("kg_green_restarted: need 1 <= n <= %d, f, q >= 1, f q <= 2^28, finite dt > 0, outputs",
                  kMaxMgs - 1);
        return KG_EINVAL;
    }
    KG_TRY(check_orbitals(s, orb, n_orb));
    const int rows = f * q + 1;
    const size_t per = (size_t)rows * n_orb * n_orb * 2;
    std::memset(G_gtr, 0, sizeof(double) * per);
    std::memset(G_les, 0, sizeof(double) * per);
    KG_TRY(ensure_gs(s, o));
    std::vector<EqGroup> G;
    std::vector<const kg_sector*> cols;
    eq_groups(G, cols, s, 0, orb, n_orb);
    if (cols.empty()) return KG_OK;
    cudaStream_t st = pick_stream(s, o);
    Krylov K;
    double2 *P = nullptr, *cq = nullptr, *ov0 = nullptr;
    auto release = [&](int rc) {
        for (auto& g : G) cudaFree(g.chi);
        cudaFree(P);
        cudaFree(cq);
        cudaFree(ov0);
        krylov_free(K);
        return rc;
    };
    int rc = krylov_alloc(K, cols, n, s->nsm, o->schedule);
    if (rc != KG_OK) return release(rc);
    const int B = K.B, MK = K.M + 1;
    int na_max = 1;
    size_t off = 0;
    for (auto& g : G) {
        const size_t na = g.idx.size();
        na_max = std::max(na_max, (int)na);
        g.ov0 = off;
        off += na * rows * na;
        if (cudaMalloc(&g.chi, sizeof(double2) * na * g.nb->d) != cudaSuccess) {
            set_error("restarted-Lanczos workspace allocation failed");
            return release(KG_ENOMEM);
        }
    }
    if (cudaMalloc(&P, sizeof(double2) * (size_t)B * MK * na_max) != cudaSuccess ||
        cudaMalloc(&cq, sizeof(double2) * (size_t)B * K.M) != cudaSuccess ||
        cudaMalloc(&ov0, sizeof(double2) * (size_t)na_max * na_max) != cudaSuccess) {
        set_error("restarted-Lanczos workspace allocation failed");
        return release(KG_ENOMEM);
    }
    std::vector<double2> hov(off), h0((size_t)na_max * na_max);
    for (auto& g : G) {
        const int na = (int)g.idx.size(), dn = (int)g.nb->d;
        for (int a = 0; a < na && rc == KG_OK; ++a) {
            rc = launch_cop(s, g.nb, orb[2 * g.idx[a]], g.spin, g.dagger, s->gs, g.chi + (size_t)a * dn, st);
            if (rc == KG_OK &&
                cudaMemcpyAsync(K.vec(g.col0 + a, 0), g.chi + (size_t)a * dn, sizeof(double2) * dn,
                                cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                rc = KG_ECUDA;
        }
        if (rc == KG_OK) rc = launch_inner_lib(g.chi, na, g.chi, na, dn, ov0, na, st);  // t = 0
        if (rc == KG_OK &&
            (cudaMemcpyAsync(h0.data(), ov0, sizeof(double2) * na * na, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess))
            rc = cuda_fail(cudaGetLastError(), "restarted Lanczos, t = 0", __FILE__, __LINE__);
        if (rc != KG_OK) return release(rc);
        for (int bcol = 0; bcol < na; ++bcol)
            for (int a = 0; a < na; ++a) hov[g.ov0 + (size_t)bcol * rows * na + a] = h0[(size_t)bcol * na + a];
    }
    std::vector<double2> hP((size_t)B * MK * na_max), hc((size_t)B * K.M);
    std::vector<ColScalars> hcs(B);
    std::vector<double> dd, ee, Z;
    std::vector<std::complex<double>> W, ph, step;
    for (int r = 0; r < f; ++r) {
        rc = build_space(K, o->reorth, st);
        for (auto& g : G) {
            const int na = (int)g.idx.size(), dn = (int)g.nb->d;
            for (int a = 0; rc == KG_OK && a < na; ++a)
                rc = launch_inner_lib(g.chi, na, K.vec(g.col0 + a, 0), MK, dn, P + (size_t)(g.col0 + a) * MK * na_max,
                                      na_max, st);
        }
        if (rc == KG_OK &&
            (cudaMemcpyAsync(hP.data(), P, sizeof(double2) * hP.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaMemcpyAsync(hcs.data(), K.cs, sizeof(ColScalars) * B, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess))
            rc = cuda_fail(cudaGetLastError(), "restarted-Lanczos readback", __FILE__, __LINE__);
        if (rc != KG_OK) return release(rc);
        for (auto& g : G) {
            const int na = (int)g.idx.size();
            const double sgn = g.dagger ? 1.0 : -1.0;  // particle columns forward, hole columns backward in t
            for (int bcol = 0; bcol < na; ++bcol) {
                const int b = g.col0 + bcol;
                const ColScalars& c = hcs[b];
                if (c.status == KG_ENUMERIC) {
                    set_error("non-finite value in the restarted Lanczos run");
                    return release(KG_ENUMERIC);
                }
                const int m = c.m_eff;
                double2* cnext = hc.data() + (size_t)b * K.M;
                for (int k = 0; k < K.M; ++k) cnext[k] = make_double2(0.0, 0.0);
                if (m == 0) continue;  // the column vanished: G stays zero from here
                dd.assign(c.alpha, c.alpha + m);
                ee.assign(m, 0.0);
                for (int k = 0; k + 1 < m; ++k) ee[k] = c.beta[k + 1];
                tql_eigen(dd, ee, m, Z);
                // G value of orbital a at tau: sum_m W[a][m] e^{-i theta_m sgn tau},
                // W[a][m] = beta0 (sum_k <chi_a | V_k> s_k Z_km) Z_0m
                W.assign((size_t)na * m, 0.0);
                for (int a = 0; a < na; ++a)
                    for (int mm = 0; mm < m; ++mm) {
                        std::complex<double> acc(0.0, 0.0);
                        for (int k = 0; k < m; ++k) {
                            const double2 pv = hP[((size_t)b * MK + k) * na_max + a];
                            acc += std::complex<double>(pv.x, pv.y) * (c.scale[k] * Z[(size_t)k * m + mm]);
                        }
                        W[(size_t)a * m + mm] = acc * (c.beta0 * Z[mm]);
                    }
                // output times t_r + i dt, i = 1..q: phases by repeated multiplication,
                // re-anchored on exact values every 256 times
                ph.assign(m, 1.0);
                step.resize(m);
                for (int mm = 0; mm < m; ++mm) step[mm] = std::polar(1.0, -dd[mm] * sgn * dt);
                for (int i = 1; i <= q; ++i) {
                    if ((i & 255) == 0)
                        for (int mm = 0; mm < m; ++mm) ph[mm] = std::polar(1.0, -dd[mm] * sgn * dt * i);
                    else
                        for (int mm = 0; mm < m; ++mm) ph[mm] *= step[mm];
                    const size_t row = (size_t)r * q + i;
                    for (int a = 0; a < na; ++a) {
                        std::complex<double> acc(0.0, 0.0);
                        for (int mm = 0; mm < m; ++mm) acc += W[(size_t)a * m + mm] * ph[mm];
                        hov[g.ov0 + ((size_t)bcol * rows + row) * na + a] = make_double2(acc.real(), acc.imag());
                    }
                }
                // psi(t_r + Delta t) = V c, c_k = beta0 s_k sum_m Z_km e^{-i theta_m sgn q dt} Z_0m
                for (int k = 0; k < m; ++k) {
                    std::complex<double> acc(0.0, 0.0);
                    for (int mm = 0; mm < m; ++mm)
                        acc += Z[(size_t)k * m + mm] * std::polar(1.0, -dd[mm] * sgn * dt * q) * Z[mm];
                    acc *= c.beta0 * c.scale[k];
                    cnext[k] = make_double2(acc.real(), acc.imag());
                }
            }
        }
        if (r + 1 == f) break;
        if (cudaMemcpyAsync(cq, hc.data(), sizeof(double2) * hc.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpy2DAsync(reinterpret_cast<char*>(K.cs) + offsetof(ColScalars, c), sizeof(ColScalars), cq,
                              sizeof(double2) * K.M, sizeof(double2) * K.M, B, cudaMemcpyDeviceToDevice,
                              st) != cudaSuccess)
            return release(cuda_fail(cudaGetLastError(), "restarted-Lanczos coefficients", __FILE__, __LINE__));
        rc = launch_combine(K, st);
        if (rc != KG_OK) return release(rc);
    }
    for (auto& g : G) eq_assemble(g, hov, rows, dt, s->E0, n_orb, G_gtr, G_les);
    return release(KG_OK);
}

// ------------------------------------------ Matsubara function on a tau grid
// Section 4, after step (iv): the zero-temperature Matsubara function of H for
// every orbital pair of one spin on tau_k = k dtau, by imaginary-time Krylov
// steps.  Each column's vector (c^dag_b|0> for the particle part, c_b|0> for
// the hole part) goes from tau to tau + dtau by the step of Eq. (udelta) with
// the imaginary-time exponential, psi' = ||psi|| V e^{-(T - s) dtau} e_1,
// s = E0 + mu (particle) or E0 - mu (hole).  The Krylov spaces, the overlaps
// <vec_a | V_k> and the combination run on the GPU (the kernels of the fine
// output grid); the m-dimensional exponential is a Taylor series on the host
// (substeps with ||T - s||_inf h <= 1/2, 18 terms).

// Coefficients on the stored (unnormalised) basis: out[k] = beta0 scale_k
// [e^{-(T - s) dtau} e_1]_k for k < m_eff, zero up to M.  Returns the usual
// a-posteriori estimate of the step's relative error, b_m dtau
// |[e^{-(T - s) dtau} e_1]_{m-1}| (zero when the space is invariant).
static double imag_step_coefficients(const ColScalars& c, double shift, double dtau, int M, double2* out) {
    const int m = c.m_eff;
    for (int k = 0; k < M; ++k) out[k] = make_double2(0.0, 0.0);
    if (m == 0) return 0.0;
    std::vector<double> v(m, 0.0), term(m), y(m), sum(m);
    v[0] = 1.0;
    double g = 0.0;
    for (int k = 0; k < m; ++k) {
        const double bl = k >= 1 ? c.beta[k] : 0.0, br = k + 1 < m ? c.beta[k + 1] : 0.0;
        g = std::max(g, std::fabs(c.alpha[k] - shift) + std::fabs(bl) + std::fabs(br));
    }
    const int nsub = std::max(1, (int)std::ceil(2.0 * g * dtau));
    const double h = dtau / nsub;
    for (int sub = 0; sub < nsub; ++sub) {
        term = v;
        sum = v;
        for (int n = 1; n <= 18; ++n) {
            for (int k = 0; k < m; ++k) {
                double t = (c.alpha[k] - shift) * term[k];
                if (k >= 1) t += c.beta[k] * term[k - 1];
                if (k + 1 < m) t += c.beta[k + 1] * term[k + 1];
                y[k] = t;
            }
            for (int k = 0; k < m; ++k) {
                term[k] = -(h / n) * y[k];
                sum[k] += term[k];
            }
        }
        v = sum;
    }
    for (int k = 0; k < m; ++k) out[k] = make_double2(c.beta0 * c.scale[k] * v[k], 0.0);
    if (m < M) return 0.0;  // happy breakdown: the Krylov space is invariant
    double nv = 0.0;
    for (int k = 0; k < m; ++k) nv += v[k] * v[k];
    return c.beta[m] * dtau * std::fabs(v[m - 1]) / std::max(std::sqrt(nv), 1e-300);
}

// Largest accepted a-posteriori error of one imaginary-time Krylov step.
constexpr double kImagStepTol = 1e-11;

static int imag_step_error(double err, double dtau, int M) {
    if (err <= kImagStepTol) return KG_OK;
    set_error("imaginary-time Krylov step error estimate %.2e above %.0e: dtau = %g is too large for M = %d "
              "(reduce dtau or raise M)", err, kImagStepTol, dtau, M);
    return KG_ENOCONV;
}

int green_matsubara_steps(kg_sector* s, const int* orb, int n_orb, double mu, double dtau, int n_steps,
                          const kg_opts* o, double* G_plus, double* G_minus) {
    KG_TRY(check_opts(o));
    if (n_steps < 0 || !(dtau > 0.0) || !std::isfinite(dtau) || !std::isfinite(mu) || !G_plus || !G_minus) {
        set_error("kg_green_matsubara_steps: need n_steps >= 0, finite dtau > 0, finite mu and output buffers");
        return KG_EINVAL;
    }
    KG_TRY(check_orbitals(s, orb, n_orb));
    const int rows = n_steps + 1;
    const size_t per = (size_t)rows * n_orb * n_orb * 2;
    std::memset(G_plus, 0, sizeof(double) * per);
    std::memset(G_minus, 0, sizeof(double) * per);
    KG_TRY(ensure_gs(s, o));
    std::vector<EqGroup> G;
    std::vector<const kg_sector*> cols;
    eq_groups(G, cols, s, 0, orb, n_orb);
    if (cols.empty()) return KG_OK;
    cudaStream_t st = pick_stream(s, o);
    Krylov K;
    double2 *ov0 = nullptr, *P = nullptr, *cq = nullptr;
    auto release = [&](int rc) {
        for (auto& g : G) cudaFree(g.chi);
        cudaFree(ov0);
        cudaFree(P);
        cudaFree(cq);
        krylov_free(K);
        return rc;
    };
    const int rc_alloc = krylov_alloc(K, cols, o->M, s->nsm, o->schedule);
    if (rc_alloc != KG_OK) return release(rc_alloc);
    const int B = K.B, MK = K.M + 1;
    size_t off = 0;
    int na_max = 1;
    for (auto& g : G) {
        const size_t na = g.idx.size();
        na_max = std::max(na_max, (int)na);
        g.ov0 = off;
        off += na * rows * na;
        if (cudaMalloc(&g.chi, sizeof(double2) * na * g.nb->d) != cudaSuccess) {
            set_error("Matsubara workspace allocation failed");
            return release(KG_ENOMEM);
        }
    }
    if (cudaMalloc(&ov0, sizeof(double2) * (size_t)na_max * na_max * G.size()) != cudaSuccess ||
        cudaMalloc(&P, sizeof(double2) * (size_t)B * MK * na_max) != cudaSuccess ||
        cudaMalloc(&cq, sizeof(double2) * (size_t)B * K.M) != cudaSuccess) {
        set_error("Matsubara workspace allocation failed");
        return release(KG_ENOMEM);
    }
    // start vectors and row 0 (tau = 0): <vec_a | vec_b>
    std::vector<double2> hov(off), h0((size_t)na_max * na_max * G.size());
    for (size_t gi = 0; gi < G.size(); ++gi) {
        const EqGroup& g = G[gi];
        const int na = (int)g.idx.size(), dn = (int)g.nb->d;
        for (int a = 0; a < na; ++a) {
            int rc = launch_cop(s, g.nb, orb[2 * g.idx[a]], g.spin, g.dagger, s->gs, g.chi + (size_t)a * dn, st);
            if (rc != KG_OK) return release(rc);
            if (cudaMemcpyAsync(K.vec(g.col0 + a, 0), g.chi + (size_t)a * dn, sizeof(double2) * dn,
                                cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return release(cuda_fail(cudaGetLastError(), "Matsubara start vectors", __FILE__, __LINE__));
        }
        const int rc = launch_inner_lib(g.chi, na, g.chi, na, dn, ov0 + gi * na_max * na_max, na, st);
        if (rc != KG_OK) return release(rc);
    }
    if (cudaMemcpyAsync(h0.data(), ov0, sizeof(double2) * h0.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return release(cuda_fail(cudaGetLastError(), "Matsubara row 0", __FILE__, __LINE__));
    for (size_t gi = 0; gi < G.size(); ++gi) {
        const EqGroup& g = G[gi];
        const int na = (int)g.idx.size();
        for (int bcol = 0; bcol < na; ++bcol)
            for (int a = 0; a < na; ++a)
                hov[g.ov0 + (size_t)bcol * rows * na + a] = h0[gi * na_max * na_max + (size_t)bcol * na + a];
    }
    std::vector<double2> hP((size_t)B * MK * na_max), hc((size_t)B * K.M);
    std::vector<ColScalars> hcs(B);
    for (int k = 1; k <= n_steps; ++k) {
        int rc = build_space(K, o->reorth, st);
        for (auto& g : G) {
            const int na = (int)g.idx.size(), dn = (int)g.nb->d;
            for (int a = 0; rc == KG_OK && a < na; ++a)
                rc = launch_inner_lib(g.chi, na, K.vec(g.col0 + a, 0), MK, dn, P + (size_t)(g.col0 + a) * MK * na_max,
                                      na_max, st);
        }
        if (rc != KG_OK) return release(rc);
        if (cudaMemcpyAsync(hP.data(), P, sizeof(double2) * hP.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hcs.data(), K.cs, sizeof(ColScalars) * B, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return release(cuda_fail(cudaGetLastError(), "Matsubara readback", __FILE__, __LINE__));
        for (auto& g : G) {
            const int na = (int)g.idx.size();
            const double shift = g.dagger ? s->E0 + mu : s->E0 - mu;
            for (int bcol = 0; bcol < na; ++bcol) {
                const int b = g.col0 + bcol, m = hcs[b].m_eff;
                if (hcs[b].status == KG_ENUMERIC) {
                    set_error("non-finite value during the imaginary-time steps");
                    return release(KG_ENUMERIC);
                }
                double2* c = hc.data() + (size_t)b * K.M;
                const int erc = imag_step_error(imag_step_coefficients(hcs[b], shift, dtau, K.M, c), dtau, K.M);
                if (erc != KG_OK) return release(erc);
                for (int a = 0; a < na; ++a) {
                    std::complex<double> acc(0.0, 0.0);
                    for (int kk = 0; kk < m; ++kk) {
                        const double2 pv = hP[((size_t)b * MK + kk) * na_max + a];
                        acc += c[kk].x * std::complex<double>(pv.x, pv.y);
                    }
                    hov[g.ov0 + ((size_t)bcol * rows + k) * na + a] = make_double2(acc.real(), acc.imag());
                }
            }
        }
        // psi(tau + dtau) = V c becomes the next start vector
        if (cudaMemcpyAsync(cq, hc.data(), sizeof(double2) * hc.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpy2DAsync(reinterpret_cast<char*>(K.cs) + offsetof(ColScalars, c), sizeof(ColScalars), cq,
                              sizeof(double2) * K.M, sizeof(double2) * K.M, B, cudaMemcpyDeviceToDevice,
                              st) != cudaSuccess)
            return release(cuda_fail(cudaGetLastError(), "Matsubara coefficients", __FILE__, __LINE__));
        rc = launch_combine(K, st);
        if (rc != KG_OK) return release(rc);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return release(cuda_fail(cudaGetLastError(), "Matsubara steps", __FILE__, __LINE__));
    // G_plus[k][a][b] = -<c^dag_a 0 | psi_b>; G_minus[k][b][a] = <c_a 0 | psi_b>
    for (auto& g : G) {
        const int na = (int)g.idx.size();
        for (int k = 0; k < rows; ++k)
            for (int bcol = 0; bcol < na; ++bcol)
                for (int a = 0; a < na; ++a) {
                    const double2 v = hov[g.ov0 + ((size_t)bcol * rows + k) * na + a];
                    const int r = g.dagger ? g.idx[a] : g.idx[bcol];
                    const int c = g.dagger ? g.idx[bcol] : g.idx[a];
                    const double sg = g.dagger ? -1.0 : 1.0;
                    double* out =
                        (g.dagger ? G_plus : G_minus) + ((size_t)k * n_orb * n_orb + (size_t)r * n_orb + c) * 2;
                    out[0] = sg * v.x;
                    out[1] = sg * v.y;
                }
    }
    return release(KG_OK);
}

// The imaginary-time vectors of one (spin, kind) group of orbitals on
// tau_j = j dtau, j = 0..n_steps: e^{-(H - s) tau_j} c_a|0> (dagger = 0,
// s = E0 - mu) or e^{-(H - s) tau_j} c^dag_a|0> (dagger = 1, s = E0 + mu) in
// the neighbour sector of H, by the imaginary-time Krylov steps of
// green_matsubara_steps, each row copied to store[j][a][:].
int imag_time_vectors(kg_sector* s, const int* orb, const std::vector<int>& idx, int spin, int dagger, double mu,
                      double dtau, int n_steps, const kg_opts* o, double2* store, cudaStream_t st) {
    kg_sector* nb = nullptr;
    KG_TRY(neighbour(s, spin, dagger, &nb));
    const int na = (int)idx.size(), dn = (int)nb->d;
    std::vector<const kg_sector*> cols(na, nb);
    Krylov K;
    double2* cq = nullptr;
    auto release = [&](int rc) {
        cudaFree(cq);
        krylov_free(K);
        return rc;
    };
    const int rc_alloc = krylov_alloc(K, cols, std::min(o->M, dn), s->nsm, o->schedule);
    if (rc_alloc != KG_OK) return release(rc_alloc);
    if (cudaMalloc(&cq, sizeof(double2) * (size_t)na * K.M) != cudaSuccess) {
        set_error("imaginary-time workspace allocation failed");
        return release(KG_ENOMEM);
    }
    auto keep_row = [&](int j) -> int {
        const cudaError_t e = cudaMemcpy2DAsync(store + (size_t)j * na * dn, (size_t)dn * sizeof(double2), K.vec(0, 0),
                                                (size_t)(K.M + 1) * dn * sizeof(double2),
                                                (size_t)dn * sizeof(double2), na, cudaMemcpyDeviceToDevice, st);
        return e == cudaSuccess ? KG_OK : cuda_fail(e, "imaginary-time store", __FILE__, __LINE__);
    };
    for (int a = 0; a < na; ++a) {
        const int rc = launch_cop(s, nb, orb[2 * idx[a]], spin, dagger, s->gs, K.vec(a, 0), st);
        if (rc != KG_OK) return release(rc);
    }
    int rc = keep_row(0);
    const double shift = dagger ? s->E0 + mu : s->E0 - mu;
    std::vector<double2> hc((size_t)na * K.M);
    std::vector<ColScalars> hcs(na);
    for (int j = 1; rc == KG_OK && j <= n_steps; ++j) {
        rc = build_space(K, o->reorth, st);
        if (rc == KG_OK &&
            (cudaMemcpyAsync(hcs.data(), K.cs, sizeof(ColScalars) * na, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess))
            rc = cuda_fail(cudaGetLastError(), "imaginary-time readback", __FILE__, __LINE__);
        for (int a = 0; rc == KG_OK && a < na; ++a) {
            if (hcs[a].status == KG_ENUMERIC) {
                set_error("non-finite value during the imaginary-time steps");
                rc = KG_ENUMERIC;
                break;
            }
            rc = imag_step_error(imag_step_coefficients(hcs[a], shift, dtau, K.M, hc.data() + (size_t)a * K.M), dtau,
                                 K.M);
        }
        if (rc == KG_OK &&
            (cudaMemcpyAsync(cq, hc.data(), sizeof(double2) * hc.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
             cudaMemcpy2DAsync(reinterpret_cast<char*>(K.cs) + offsetof(ColScalars, c), sizeof(ColScalars), cq,
                               sizeof(double2) * K.M, sizeof(double2) * K.M, na, cudaMemcpyDeviceToDevice,
                               st) != cudaSuccess))
            rc = cuda_fail(cudaGetLastError(), "imaginary-time coefficients", __FILE__, __LINE__);
        if (rc == KG_OK) rc = launch_combine(K, st);
        if (rc == KG_OK) rc = keep_row(j);
    }
    if (rc == KG_OK && cudaStreamSynchronize(st) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "imaginary-time steps", __FILE__, __LINE__);
    return release(rc);
}

}  // namespace kg

// ------------------------------------------------------------- Keldysh
// Memory plan.  The vectors of the four-step method can exceed the device:
// for the 16-site chain of the local-excitation quench (d = 130.9M) Phi(t_k)
// for 50 times is 105 GB, one (spin, kind) block of stored columns up to
// 118 GB and one column's Krylov workspace 106 GB (57 GB without the
// Gram-Schmidt planes).  keldysh_create therefore plans against a budget (the
// free device memory, or opts.mem_budget_mb):
//   * Phi(t_k) for all k stays on the device when it fits beside the blocks'
//     needs, else in host memory (pinned when the host allows), one time
//     staged onto the device per row;
//   * every block keeps its Krylov workspace between rows when all fit, else
//     each block's workspace lives only for its part of a row;
//   * the staged API keeps every block's columns for step (iv) when they fit
//     together; otherwise rows return their time-diagonal blocks only and
//     the whole grid comes from kg_green_keldysh, which runs one block at a
//     time (its columns and its workspace, with the planes when they fit).
struct KBlock {
    int spin = 0, dagger = 0;
    std::vector<int> idx;
    kg_sector* nb = nullptr;
    double2* store = nullptr;  // [slots][na][d_nb]: every row, or only the current one
    int slots = 0;
    double2* ovbuf = nullptr;  // [na][na]
    kg::Krylov K;
    kg::StepRunner R;
    bool ready = false;
    double* dwork = nullptr;   // driven H(t): diagonal of the current exponential + tables
};

struct kg_keldysh {
    kg_sector* ini = nullptr;
    kg_sector* fin = nullptr;
    std::vector<int> orb;
    int n_orb = 0, n_t = 0, n_sub = 1;
    double dt = 0.0;
    kg_opts o;
    double2* phi = nullptr;       // [n_t][d] on the device, or
    double2* phi_host = nullptr;  // [n_t][d] in host memory
    bool phi_pinned = false;
    double2* phi_stage = nullptr; // [d] device copy of one Phi(t_k) (host placement)
    int staged = -1;              // which k phi_stage holds
    bool keep_stores = true;      // staged API: all blocks' columns kept for step (iv)
    bool keep_krylov = true;      // staged API: workspaces kept between rows
    bool planes = true;           // staged API: Gram-Schmidt planes in the workspaces
    size_t budget = 0;
    std::vector<KBlock> blocks;
    std::vector<char> row_done;
    // driven H(t): per internal step the on-site offsets of its two
    // exponentials, [(n_t - 1) n_sub][2][3L] on the device (null: a quench)
    double* drive = nullptr;
};

namespace kg {

static void block_release_krylov(KBlock& B) {
    B.R.release();
    krylov_free(B.K);
    B.ready = false;
}

static void block_release(KBlock& B) {
    block_release_krylov(B);
    cudaFree(B.store);
    cudaFree(B.ovbuf);
    cudaFree(B.dwork);
    B.store = nullptr;
    B.ovbuf = nullptr;
    B.dwork = nullptr;
    B.slots = 0;
}

// ------------------------------------------------------- driven H(t)
// Section 6 proposes commutator-free exponential propagators for a
// Hamiltonian with a general time dependence after t = 0.  The library takes
// the fourth-order one with two exponentials: with A_1, A_2 the Hamiltonian
// at the two Gauss-Legendre nodes t + (1/2 -+ sqrt(3)/6) h of a step,
//   U(t + h, t) = exp(-i h (a1 A_1 + a2 A_2)) exp(-i h (a2 A_1 + a1 A_2)),
// a1 = (3 - 2 sqrt(3)) / 12, a2 = (3 + 2 sqrt(3)) / 12, the right factor
// applied first.  The time dependence is an offset of the on-site energies
// and U; H is linear in them and a1 + a2 = 1/2, so each exponential is
// exp(-i (h/2) H(fin + o)) with o = 2 (a2 d_1 + a1 d_2) (first) or
// 2 (a1 d_1 + a2 d_2) (second), d_1, d_2 the offsets at the nodes: a Krylov
// step of tau = h/2 on a diagonal rebuilt before it.
static const double kCF4_A1 = (3.0 - 2.0 * 1.7320508075688772) / 12.0;
static const double kCF4_A2 = (3.0 + 2.0 * 1.7320508075688772) / 12.0;

static size_t drive_bytes(const kg_keldysh* X, const kg_sector* s) {
    return X->drive ? drive_work_doubles(s) * sizeof(double) : 0;
}

// Internal step `step` of the driven H(t) on every column of R (all in sector
// s, whose diagonal the runner's columns read from `work`): forward
// U = e^{-i h/2 H_2} e^{-i h/2 H_1}, or backward U^dag = e^{+i h/2 H_1}
// e^{+i h/2 H_2}, the runner's tau being +h/2 or -h/2.
static int driven_step(const kg_keldysh* X, const kg_sector* s, double* work, StepRunner& R, int step,
                       bool backward, cudaStream_t st) {
    const size_t L3 = 3 * (size_t)X->fin->L;
    const double* first = X->drive + (size_t)step * 2 * L3;
    const double* second = first + L3;
    const SecView S = s->view();
    KG_TRY(launch_drive_diag(S, backward ? second : first, work, st));
    KG_TRY(R.run(st));
    KG_TRY(launch_drive_diag(S, backward ? first : second, work, st));
    return R.run(st);
}

// The exponentials' offsets from the offsets at the Gauss nodes (host
// dparams [n_steps][2][3L]), uploaded to X->drive.
static int drive_upload(kg_keldysh* X, const double* dparams, int n_steps) {
    const size_t L3 = 3 * (size_t)X->fin->L;
    std::vector<double> ex((size_t)n_steps * 2 * L3);
    for (int s = 0; s < n_steps; ++s)
        for (size_t p = 0; p < L3; ++p) {
            const double d1 = dparams[((size_t)s * 2 + 0) * L3 + p], d2 = dparams[((size_t)s * 2 + 1) * L3 + p];
            if (!std::isfinite(d1) || !std::isfinite(d2)) {
                set_error("non-finite drive offset at step %d", s);
                return KG_EINVAL;
            }
            ex[((size_t)s * 2 + 0) * L3 + p] = 2.0 * (kCF4_A2 * d1 + kCF4_A1 * d2);
            ex[((size_t)s * 2 + 1) * L3 + p] = 2.0 * (kCF4_A1 * d1 + kCF4_A2 * d2);
        }
    if (ex.empty()) return KG_OK;
    KG_CUDA(cudaMalloc(&X->drive, sizeof(double) * ex.size()));
    KG_CUDA(cudaMemcpy(X->drive, ex.data(), sizeof(double) * ex.size(), cudaMemcpyHostToDevice));
    return KG_OK;
}

static std::vector<const kg_sector*> block_cols(const KBlock& B) {
    return std::vector<const kg_sector*>(B.idx.size(), B.nb);
}

// Workspace (with `planes`) and `slots` rows of stored columns for block B.
static int block_prepare(kg_keldysh* X, KBlock& B, cudaStream_t st, int slots, bool planes) {
    const int na = (int)B.idx.size(), dn = (int)B.nb->d;
    if (!B.store || B.slots != slots) {
        cudaFree(B.store);
        B.store = nullptr;
        B.slots = 0;
        if (cudaMalloc(&B.store, sizeof(double2) * (size_t)slots * na * dn) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot hold %d rows of %d columns of dimension %d", slots, na, dn);
            return KG_ENOMEM;
        }
        B.slots = slots;
    }
    if (!B.ovbuf) KG_CUDA(cudaMalloc(&B.ovbuf, sizeof(double2) * (size_t)na * na));
    if (B.ready) return KG_OK;
    KG_TRY(krylov_alloc(B.K, block_cols(B), std::min(X->o.M, dn), X->fin->nsm, X->o.schedule, planes));
    // step (iii) propagates backward, e^{+iH tau}; a driven H takes two
    // exponentials of half the step each
    const double tau = -X->dt / X->n_sub * (X->drive ? 0.5 : 1.0);
    for (auto& D : B.K.hdesc) D.tau = tau;
    KG_TRY(krylov_upload(B.K, st));
    if (X->drive) {
        if (!B.dwork && cudaMalloc(&B.dwork, drive_bytes(X, B.nb)) != cudaSuccess) {
            cudaGetLastError();
            B.dwork = nullptr;
            set_error("cannot hold the driven diagonal of dimension %d", dn);
            return KG_ENOMEM;
        }
        KG_TRY(krylov_set_diag(B.K, B.dwork));
    }
    KG_TRY(B.R.init(B.K, X->o.reorth, st, X->o.use_graphs != 0));
    B.ready = true;
    return KG_OK;
}

// Phi(t_k) on the device (staged from host memory when it lives there).
static int phi_at(kg_keldysh* X, int k, cudaStream_t st, const double2** out) {
    const size_t d = (size_t)X->fin->d;
    if (X->phi) {
        *out = X->phi + (size_t)k * d;
        return KG_OK;
    }
    if (X->staged != k) {
        KG_CUDA(cudaMemcpyAsync(X->phi_stage, X->phi_host + (size_t)k * d, sizeof(double2) * d,
                                cudaMemcpyHostToDevice, st));
        X->staged = k;
    }
    *out = X->phi_stage;
    return KG_OK;
}

// Step (iii) for row k of block B: the columns c_a Phi(t_k) (or c^dag_a),
// propagated back by t_k, left in slot (k or 0) of the block's store.
static int block_row(kg_keldysh* X, KBlock& B, int k, cudaStream_t st) {
    const int na = (int)B.idx.size(), dn = (int)B.nb->d;
    const double2* phik = nullptr;
    KG_TRY(phi_at(X, k, st, &phik));
    KG_TRY(launch_reset_status(B.K, st));
    for (int a = 0; a < na; ++a)
        KG_TRY(launch_cop(X->fin, B.nb, X->orb[2 * B.idx[a]], B.spin, B.dagger, phik, B.K.vec(a, 0), st));
    if (X->drive) {
        for (int n = k * X->n_sub - 1; n >= 0; --n) KG_TRY(driven_step(X, B.nb, B.dwork, B.R, n, true, st));
    } else {
        for (int n = 0; n < k * X->n_sub; ++n) KG_TRY(B.R.run(st));
    }
    const int slot = B.slots > 1 ? k : 0;
    KG_CUDA(cudaMemcpy2DAsync(B.store + (size_t)slot * na * dn, (size_t)dn * sizeof(double2), B.K.vec(0, 0),
                              (size_t)(B.K.M + 1) * dn * sizeof(double2), (size_t)dn * sizeof(double2), na,
                              cudaMemcpyDeviceToDevice, st));
    return KG_OK;
}

static int block_status_of(Krylov& K, const char* what) {
    std::vector<ColScalars> h(K.B);
    KG_CUDA(cudaMemcpy(h.data(), K.cs, sizeof(ColScalars) * K.B, cudaMemcpyDeviceToHost));
    for (auto& c : h)
        if (c.status == KG_ENUMERIC) {
            set_error("non-finite value during %s", what);
            return KG_ENUMERIC;
        }
    return KG_OK;
}

static int block_status(KBlock& B) { return block_status_of(B.K, "step (iii)"); }

// Writes this block's part of G(t_k, t_l) for every stored k, l.
static void block_assemble(kg_keldysh* X, KBlock& B, const std::vector<std::complex<double>>& Gm, double* G) {
    const int na = (int)B.idx.size(), n = X->n_orb, nt = X->n_t, nv = nt * na;
    for (int k = 0; k < nt; ++k)
        for (int l = 0; l < nt; ++l)
            for (int a = 0; a < na; ++a)
                for (int ap = 0; ap < na; ++ap) {
                    std::complex<double> g;
                    if (!B.dagger)  // G^<_{a a'}(t_k,t_l) = i <Psi_a'(t_l) | Psi_a(t_k)>
                        g = std::complex<double>(0.0, 1.0) * Gm[(size_t)(l * na + ap) * nv + (k * na + a)];
                    else  // G^>_{a a'}(t_k,t_l) = -i <chi_a(t_k) | chi_a'(t_l)>
                        g = std::complex<double>(0.0, -1.0) * Gm[(size_t)(k * na + a) * nv + (l * na + ap)];
                    const size_t o = (((size_t)k * nt + l) * n + B.idx[a]) * n + B.idx[ap];
                    G[2 * o] = g.real();
                    G[2 * o + 1] = g.imag();
                }
}

static size_t device_budget(const kg_opts* o) {
    if (o->mem_budget_mb > 0) return (size_t)o->mem_budget_mb << 20;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
    const size_t reserve = std::max<size_t>(size_t(1) << 30, total_b / 32);
    return free_b > reserve ? free_b - reserve : 0;
}

// The staged API's plan (see the comment above KBlock); Phi's placement is
// decided before, together with its propagation's workspace.
static void plan_blocks(kg_keldysh* X) {
    const size_t d16 = (size_t)X->fin->d * sizeof(double2);
    const size_t phi_dev = X->phi ? (size_t)X->n_t * d16 : d16;
    size_t sum_store = 0, sum_kry = 0, max_kry = 0, max_kry_np = 0;
    for (auto& B : X->blocks) {
        const auto cols = block_cols(B);
        const int M = std::min(X->o.M, (int)B.nb->d);
        sum_store += (size_t)X->n_t * B.idx.size() * (size_t)B.nb->d * sizeof(double2);
        const size_t dw = drive_bytes(X, B.nb);
        sum_kry += krylov_bytes(cols, M, true) + dw;
        max_kry = std::max(max_kry, krylov_bytes(cols, M, true) + dw);
        max_kry_np = std::max(max_kry_np, krylov_bytes(cols, M, false) + dw);
    }
    const size_t B = X->budget;
    X->planes = true;
    X->keep_krylov = phi_dev + sum_store + sum_kry <= B;
    X->keep_stores = X->keep_krylov || phi_dev + sum_store + max_kry <= B;
    if (!X->keep_stores && phi_dev + sum_store + max_kry_np <= B) {
        X->keep_stores = true;
        X->planes = false;
    }
    if (!X->keep_stores) X->planes = phi_dev + max_kry <= B;
}

int keldysh_create(kg_sector* ini, kg_sector* fin, const int* orb, int n_orb, double dt, int n_t,
                   const kg_opts* o, kg_keldysh** out, const double* dparams) {
    *out = nullptr;
    if (ini->L != fin->L || ini->nu != fin->nu || ini->nd != fin->nd) {
        set_error("H_ini and H_fin must share (L, N_up, N_dn)");
        return KG_EINVAL;
    }
    KG_TRY(check_orbitals(fin, orb, n_orb));
    KG_TRY(check_opts(o));
    if (n_t < 1 || !(dt >= 0.0) || o->mem_budget_mb < 0) {
        set_error("bad time grid or memory budget");
        return KG_EINVAL;
    }
    KG_TRY(ensure_gs(ini, o));
    cudaStream_t st = pick_stream(fin, o);
    kg_keldysh* X = new kg_keldysh();
    X->ini = ini;
    X->fin = fin;
    X->orb.assign(orb, orb + 2 * n_orb);
    X->n_orb = n_orb;
    X->dt = dt;
    X->n_t = n_t;
    X->o = *o;
    X->n_sub = (o->dt_internal > 0.0) ? std::max(1, (int)std::lround(dt / o->dt_internal)) : 1;
    X->row_done.assign(n_t, 0);
    auto fail = [&](int r) {
        keldysh_free(X);
        return r;
    };
    if (dparams) {
        const int rc = drive_upload(X, dparams, (n_t - 1) * X->n_sub);
        if (rc != KG_OK) return fail(rc);
    }
    std::vector<int> idx[2];
    groups(orb, n_orb, idx);
    for (int spin = 0; spin < 2; ++spin) {
        if (idx[spin].empty()) continue;
        for (int dagger = 0; dagger < 2; ++dagger) {
            kg_sector* nb = nullptr;
            if (neighbour(fin, spin, dagger, &nb) != KG_OK) continue;  // that G part is zero
            KBlock B;
            B.spin = spin;
            B.dagger = dagger;
            B.idx = idx[spin];
            B.nb = nb;
            X->blocks.push_back(std::move(B));
        }
    }
    // Phi's placement: on the device when it fits beside one block's columns
    // and workspace (the one-shot path's peak), else in host memory
    const size_t d = (size_t)fin->d, d16 = d * sizeof(double2);
    X->budget = device_budget(o);
    size_t block_peak = 0;
    for (auto& B : X->blocks)
        block_peak = std::max(block_peak, (size_t)n_t * B.idx.size() * (size_t)B.nb->d * sizeof(double2) +
                                              krylov_bytes(block_cols(B), std::min(o->M, (int)B.nb->d), false) +
                                              drive_bytes(X, B.nb));
    const int Mf = std::min(o->M, (int)d);
    const size_t fin_dw = drive_bytes(X, fin);
    const bool fin_planes_dev = (size_t)n_t * d16 + krylov_bytes({fin}, Mf, true) + fin_dw <= X->budget;
    if ((size_t)n_t * d16 + block_peak <= X->budget &&
        (size_t)n_t * d16 + krylov_bytes({fin}, Mf, false) + fin_dw <= X->budget) {
        if (cudaMalloc(&X->phi, sizeof(double2) * n_t * d) != cudaSuccess) {
            cudaGetLastError();
            X->phi = nullptr;
        }
    }
    if (!X->phi) {
        if (cudaMalloc(&X->phi_stage, d16) != cudaSuccess) {
            set_error("cannot hold one Phi(t_k) of dimension %zu", d);
            return fail(KG_ENOMEM);
        }
        if (cudaHostAlloc(&X->phi_host, sizeof(double2) * n_t * d, cudaHostAllocDefault) == cudaSuccess) {
            X->phi_pinned = true;
        } else {
            cudaGetLastError();
            X->phi_host = static_cast<double2*>(std::malloc(sizeof(double2) * n_t * d));
            if (!X->phi_host) {
                set_error("cannot hold Phi(t_k) for %d times in device or host memory", n_t);
                return fail(KG_ENOMEM);
            }
        }
    }
    // step (ii): Phi(t_k) = e^{-iH t_k} |0>, stored on the grid
    auto put = [&](int k, const double2* src) -> int {
        const cudaError_t e =
            X->phi ? cudaMemcpyAsync(X->phi + k * d, src, d16, cudaMemcpyDeviceToDevice, st)
                   : cudaMemcpyAsync(X->phi_host + k * d, src, d16, cudaMemcpyDeviceToHost, st);
        return e == cudaSuccess ? KG_OK : cuda_fail(e, "Phi(t_k) store", __FILE__, __LINE__);
    };
    int rc = put(0, ini->gs);
    if (rc == KG_OK && n_t > 1) {
        Krylov K;
        StepRunner R;
        double* work = nullptr;
        rc = krylov_alloc(K, {fin}, Mf, fin->nsm, o->schedule, X->phi ? fin_planes_dev : true);
        if (rc == KG_OK) {
            K.hdesc[0].tau = dt / X->n_sub * (X->drive ? 0.5 : 1.0);
            rc = krylov_upload(K, st);
        }
        if (rc == KG_OK && X->drive) {
            if (cudaMalloc(&work, fin_dw) != cudaSuccess) {
                cudaGetLastError();
                work = nullptr;
                set_error("cannot hold the driven diagonal of dimension %zu", d);
                rc = KG_ENOMEM;
            }
            if (rc == KG_OK) rc = krylov_set_diag(K, work);
        }
        if (rc == KG_OK)
            rc = cudaMemcpyAsync(K.vec(0, 0), ini->gs, d16, cudaMemcpyDeviceToDevice, st) == cudaSuccess ? KG_OK
                                                                                                         : KG_ECUDA;
        if (rc == KG_OK) rc = R.init(K, o->reorth, st, o->use_graphs != 0);
        if (rc == KG_OK) rc = launch_reset_status(K, st);
        for (int k = 1; rc == KG_OK && k < n_t; ++k) {
            for (int n = 0; rc == KG_OK && n < X->n_sub; ++n)
                rc = X->drive ? driven_step(X, fin, work, R, (k - 1) * X->n_sub + n, false, st) : R.run(st);
            if (rc == KG_OK) rc = put(k, K.vec(0, 0));
        }
        if (rc == KG_OK) rc = cudaStreamSynchronize(st) == cudaSuccess ? KG_OK : KG_ECUDA;
        if (rc == KG_OK) rc = block_status_of(K, "step (ii)");
        R.release();
        krylov_free(K);
        cudaFree(work);
    } else if (rc == KG_OK) {
        rc = cudaStreamSynchronize(st) == cudaSuccess ? KG_OK : KG_ECUDA;
    }
    if (rc != KG_OK) return fail(rc);
    plan_blocks(X);
    *out = X;
    return KG_OK;
}

void keldysh_free(kg_keldysh* X) {
    if (!X) return;
    for (auto& B : X->blocks) block_release(B);
    cudaFree(X->drive);
    cudaFree(X->phi);
    cudaFree(X->phi_stage);
    if (X->phi_pinned)
        cudaFreeHost(X->phi_host);
    else
        std::free(X->phi_host);
    delete X;
}

int keldysh_row(kg_keldysh* X, int k, double* G_les_kk, double* G_gtr_kk) {
    if (k < 0 || k >= X->n_t) {
        set_error("row %d outside [0, %d)", k, X->n_t);
        return KG_EINVAL;
    }
    cudaStream_t st = pick_stream(X->fin, &X->o);
    const int n = X->n_orb;
    if (G_les_kk) std::memset(G_les_kk, 0, sizeof(double) * 2 * n * n);
    if (G_gtr_kk) std::memset(G_gtr_kk, 0, sizeof(double) * 2 * n * n);
    for (auto& B : X->blocks) {
        int rc = block_prepare(X, B, st, X->keep_stores ? X->n_t : 1, X->planes);
        if (rc == KG_OK) rc = block_row(X, B, k, st);
        const int na = (int)B.idx.size(), dn = (int)B.nb->d;
        const double2* xs = B.store + (B.slots > 1 ? (size_t)k * na * dn : 0);
        if (rc == KG_OK) rc = launch_inner_lib(xs, na, xs, na, dn, B.ovbuf, na, st);
        std::vector<double2> h((size_t)na * na);
        if (rc == KG_OK &&
            (cudaMemcpyAsync(h.data(), B.ovbuf, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st) !=
                 cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess))
            rc = cuda_fail(cudaGetLastError(), "row readback", __FILE__, __LINE__);
        if (rc == KG_OK) rc = block_status(B);
        if (!X->keep_krylov) block_release_krylov(B);
        if (!X->keep_stores) block_release(B);
        if (rc != KG_OK) return rc;
        double* G = B.dagger ? G_gtr_kk : G_les_kk;
        if (!G) continue;
        for (int bb = 0; bb < na; ++bb)
            for (int a = 0; a < na; ++a) {
                // h[bb][a] = <X_a | X_bb>
                const double2 v = h[(size_t)bb * na + a];
                const std::complex<double> ov(v.x, v.y);
                int r, c;
                std::complex<double> g;
                if (!B.dagger) {  // G^<_{bb a} = i <Psi_a | Psi_bb>
                    r = B.idx[bb];
                    c = B.idx[a];
                    g = std::complex<double>(0.0, 1.0) * ov;
                } else {  // G^>_{a bb} = -i <chi_a | chi_bb>
                    r = B.idx[a];
                    c = B.idx[bb];
                    g = std::complex<double>(0.0, -1.0) * ov;
                }
                G[2 * ((size_t)r * n + c)] = g.real();
                G[2 * ((size_t)r * n + c) + 1] = g.imag();
            }
    }
    X->row_done[k] = 1;
    return KG_OK;
}

int keldysh_gram(kg_keldysh* X, double* G_les, double* G_gtr) {
    if (!X->keep_stores) {
        set_error("the memory plan keeps no columns for step (iv) (they exceed the budget); "
                  "kg_green_keldysh computes the grid one block at a time");
        return KG_EINVAL;
    }
    for (int k = 0; k < X->n_t; ++k)
        if (!X->row_done[k]) {
            set_error("row %d of step (iii) not computed", k);
            return KG_EINVAL;
        }
    cudaStream_t st = pick_stream(X->fin, &X->o);
    const size_t tot = (size_t)X->n_t * X->n_t * X->n_orb * X->n_orb * 2;
    if (G_les) std::memset(G_les, 0, sizeof(double) * tot);
    if (G_gtr) std::memset(G_gtr, 0, sizeof(double) * tot);
    for (auto& B : X->blocks) {
        double* G = B.dagger ? G_gtr : G_les;
        if (!G) continue;
        const int na = (int)B.idx.size();
        std::vector<std::complex<double>> Gm;
        KG_TRY(gram(B.store, X->n_t * na, (int)B.nb->d, X->fin->nsm, Gm, st));
        block_assemble(X, B, Gm, G);
    }
    return KG_OK;
}

int keldysh_phi(kg_keldysh* X, int k, double* phi_host, const double* phi_in) {
    if (k < 0 || k >= X->n_t) {
        set_error("row %d outside [0, %d)", k, X->n_t);
        return KG_EINVAL;
    }
    const size_t d = (size_t)X->fin->d;
    if (!X->phi) {  // host placement
        if (phi_host) std::memcpy(phi_host, X->phi_host + k * d, sizeof(double2) * d);
        if (phi_in) {
            std::memcpy(X->phi_host + k * d, phi_in, sizeof(double2) * d);
            if (X->staged == k) X->staged = -1;
        }
        return KG_OK;
    }
    cudaStream_t st = pick_stream(X->fin, &X->o);
    if (phi_host) KG_CUDA(cudaMemcpyAsync(phi_host, X->phi + k * d, sizeof(double2) * d, cudaMemcpyDeviceToHost, st));
    if (phi_in) KG_CUDA(cudaMemcpyAsync(X->phi + k * d, phi_in, sizeof(double2) * d, cudaMemcpyHostToDevice, st));
    KG_CUDA(cudaStreamSynchronize(st));
    return KG_OK;
}

int keldysh_plan(const kg_keldysh* X, int* phi_on_host, int* stores_kept, int* planes, long long* budget) {
    if (phi_on_host) *phi_on_host = X->phi ? 0 : (X->phi_pinned ? 1 : 2);
    if (stores_kept) *stores_kept = X->keep_stores ? 1 : 0;
    if (planes) *planes = X->planes ? 1 : 0;
    if (budget) *budget = (long long)X->budget;
    return KG_OK;
}

// Whole Keldysh calculation, one (spin, kind) block at a time so that only
// one block's stored columns and workspace are resident.
int green_keldysh(kg_sector* ini, kg_sector* fin, const int* orb, int n_orb, double dt, int n_t,
                  const kg_opts* o, double* G_les, double* G_gtr, const double* dparams) {
    if (!G_les || !G_gtr) {
        set_error("NULL output");
        return KG_EINVAL;
    }
    kg_keldysh* X = nullptr;
    KG_TRY(keldysh_create(ini, fin, orb, n_orb, dt, n_t, o, &X, dparams));
    cudaStream_t st = pick_stream(fin, o);
    const size_t tot = (size_t)n_t * n_t * n_orb * n_orb * 2;
    std::memset(G_les, 0, sizeof(double) * tot);
    std::memset(G_gtr, 0, sizeof(double) * tot);
    const size_t phi_dev = X->phi ? (size_t)n_t * fin->d * sizeof(double2) : (size_t)fin->d * sizeof(double2);
    int rc = KG_OK;
    for (auto& B : X->blocks) {
        const size_t store = (size_t)n_t * B.idx.size() * (size_t)B.nb->d * sizeof(double2);
        const bool planes = phi_dev + store + krylov_bytes(block_cols(B), std::min(o->M, (int)B.nb->d), true) +
                                drive_bytes(X, B.nb) <=
                            X->budget;
        rc = block_prepare(X, B, st, n_t, planes);
        for (int k = 0; rc == KG_OK && k < n_t; ++k) rc = block_row(X, B, k, st);
        if (rc == KG_OK) rc = cudaStreamSynchronize(st) == cudaSuccess ? KG_OK : KG_ECUDA;
        if (rc == KG_OK) rc = block_status(B);
        // the workspace goes before the Gram, which needs its own scratch
        block_release_krylov(B);
        std::vector<std::complex<double>> Gm;
        if (rc == KG_OK) rc = gram(B.store, n_t * (int)B.idx.size(), (int)B.nb->d, fin->nsm, Gm, st);
        if (rc == KG_OK) block_assemble(X, B, Gm, B.dagger ? G_gtr : G_les);
        block_release(B);
        if (rc != KG_OK) break;
    }
    keldysh_free(X);
    return rc;
}

// Section 4, the remark after step (iv): the mixed components on the
// imaginary branch at zero temperature, with the initial state |0> of H_ini
// and K = H_ini - mu N there:
//   G^right_{aa'}(t_k, tau_j) = +i <xi_a'(tau_j) | Psi_a(t_k)>,
//   G^left_{aa'}(tau_j, t_k)  = -i <zeta_a(tau_j) | chi_a'(t_k)>,
// xi_a(tau) = e^{-(H_ini - E0 + mu) tau} c_a|0>, zeta_a(tau) =
// e^{-(H_ini - E0 - mu) tau} c^dag_a|0>, Psi and chi the step-(iii) columns
// of the quench.  Rectangular overlaps of the stored imaginary-time vectors
// (in the neighbour sectors of H_ini) with the stored Keldysh columns (the
// same sectors of H_fin: the same basis).
int green_mixed(kg_sector* ini, kg_sector* fin, const int* orb, int n_orb, double dt, int n_t, double mu, double dtau,
                int n_tau, const kg_opts* o, double* G_right, double* G_left) {
    if (!G_right || !G_left || n_tau < 0 || !(dtau > 0.0) || !std::isfinite(dtau) || !std::isfinite(mu)) {
        set_error("kg_green_mixed: need output buffers, n_tau >= 0, finite dtau > 0 and finite mu");
        return KG_EINVAL;
    }
    kg_keldysh* X = nullptr;
    KG_TRY(keldysh_create(ini, fin, orb, n_orb, dt, n_t, o, &X));
    auto done = [&](int rc) {
        keldysh_free(X);
        return rc;
    };
    if (!X->keep_stores) {
        set_error("kg_green_mixed needs every Keldysh column kept (they exceed the device-memory budget)");
        return done(KG_ENOMEM);
    }
    for (int k = 0; k < n_t; ++k) {
        const int rc = keldysh_row(X, k, nullptr, nullptr);
        if (rc != KG_OK) return done(rc);
    }
    cudaStream_t st = pick_stream(fin, o);
    const int nj = n_tau + 1, n = n_orb;
    std::memset(G_right, 0, sizeof(double) * 2 * (size_t)n_t * nj * n * n);
    std::memset(G_left, 0, sizeof(double) * 2 * (size_t)nj * n_t * n * n);
    for (auto& B : X->blocks) {
        const int na = (int)B.idx.size(), dn = (int)B.nb->d;
        double2 *tau_store = nullptr, *ov = nullptr;
        const int nx = nj * na, ny = n_t * na;
        if (cudaMalloc(&tau_store, sizeof(double2) * (size_t)nx * dn) != cudaSuccess ||
            cudaMalloc(&ov, sizeof(double2) * (size_t)nx * ny) != cudaSuccess) {
            cudaFree(tau_store);
            set_error("cannot hold the imaginary-time vectors of one block");
            return done(KG_ENOMEM);
        }
        int rc = imag_time_vectors(ini, orb, B.idx, B.spin, B.dagger, mu, dtau, n_tau, o, tau_store, st);
        // ov[y][x] = <tau vector x | Keldysh column y>, in chunks of kMaxOv tau vectors
        for (int x0 = 0; rc == KG_OK && x0 < nx; x0 += kMaxOv)
            rc = launch_inner_lib(tau_store + (size_t)x0 * dn, std::min(kMaxOv, nx - x0), B.store, ny, dn, ov + x0, nx,
                                  st);
        std::vector<double2> h((size_t)nx * ny);
        if (rc == KG_OK &&
            (cudaMemcpyAsync(h.data(), ov, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess))
            rc = cuda_fail(cudaGetLastError(), "mixed-component readback", __FILE__, __LINE__);
        cudaFree(tau_store);
        cudaFree(ov);
        if (rc != KG_OK) return done(rc);
        for (int k = 0; k < n_t; ++k)
            for (int j = 0; j < nj; ++j)
                for (int a = 0; a < na; ++a)
                    for (int ap = 0; ap < na; ++ap) {
                        if (!B.dagger) {  // G^right_{a a'}(t_k, tau_j) = i <xi_a'(tau_j) | Psi_a(t_k)>
                            const double2 v = h[(size_t)(k * na + a) * nx + (j * na + ap)];
                            const size_t off = (((size_t)k * nj + j) * n + B.idx[a]) * n + B.idx[ap];
                            G_right[2 * off] = -v.y;
                            G_right[2 * off + 1] = v.x;
                        } else {  // G^left_{a a'}(tau_j, t_k) = -i <zeta_a(tau_j) | chi_a'(t_k)>
                            const double2 v = h[(size_t)(k * na + ap) * nx + (j * na + a)];
                            const size_t off = (((size_t)j * n_t + k) * n + B.idx[a]) * n + B.idx[ap];
                            G_left[2 * off] = v.y;
                            G_left[2 * off + 1] = -v.x;
                        }
                    }
    }
    return done(KG_OK);
}


// ------------------------------------------- four-time correlation functions
// Section 6 (outlook): functions of four time arguments, as the
// nonequilibrium dual-fermion approach needs them, by the same Krylov steps.
//   G(t1, t2, t3, t4) = <0| A1(t1) A2(t2) A3(t3) A4(t4) |0>,  A(t) = e^{iHt} A e^{-iHt},
// H = H_fin, |0> the ground state of H_ini.  With Phi(t) = e^{-iHt}|0> this
// is <L(t1, t2) | R(t3, t4)> for the right vectors
//   R(t3, t4) = e^{iH t3} A3 e^{-iH(t3 - t4)} A4 Phi(t4)
// and the left vectors L(t1, t2) = e^{iH t2} A2^dag e^{-iH(t2 - t1)} A1^dag Phi(t1),
// both in the sector two operators away from H_fin's.  Each family is made
// by pair_vectors: one batch of n_t columns A Phi(t_b) swept forward and
// backward over the grid (every t_a - t_b), B applied at each grid point, and
// the results brought back by e^{iH t_a} in batches of equal t_a.
struct FourOp {
    int site, spin, dagger;
};

// n grid steps of the runner's sign on every column: n_sub Krylov steps each.
static int grid_steps(StepRunner& R, int n, int n_sub, cudaStream_t st) {
    for (int k = 0; k < n * n_sub; ++k) KG_TRY(R.run(st));
    return KG_OK;
}

// V[ta * n_t + tb] = e^{iH ta} B e^{-iH(ta - tb)} A Phi(tb) in sector s2.
static int pair_vectors(kg_sector* fin, kg_sector* s1, kg_sector* s2, FourOp A, FourOp B, const double2* phi, int n_t,
                        double dt, int n_sub, const kg_opts* o, double2* V, cudaStream_t st) {
    const size_t d0 = (size_t)fin->d, d1 = (size_t)s1->d, d2 = (size_t)s2->d;
    const double h = dt / n_sub;
    int rc = KG_OK;
    {
        // every t_a - t_b: the columns A Phi(t_b) forward, then again backward
        Krylov K;
        StepRunner R;
        rc = krylov_alloc(K, std::vector<const kg_sector*>(n_t, s1), std::min(o->M, (int)d1), fin->nsm, o->schedule);
        for (int sweep = 0; rc == KG_OK && sweep < 2; ++sweep) {
            const int sgn = sweep == 0 ? 1 : -1;
            for (auto& D : K.hdesc) D.tau = sgn * h;
            rc = krylov_upload(K, st);
            if (rc == KG_OK && sweep == 0) rc = R.init(K, o->reorth, st, o->use_graphs != 0);
            if (rc == KG_OK) rc = launch_reset_status(K, st);
            for (int tb = 0; rc == KG_OK && tb < n_t; ++tb)
                rc = launch_cop(fin, s1, A.site, A.spin, A.dagger, phi + tb * d0, K.vec(tb, 0), st);
            for (int m = sweep; rc == KG_OK && m < n_t; ++m) {
                if (m > 0) rc = grid_steps(R, 1, n_sub, st);
                for (int tb = 0; rc == KG_OK && tb < n_t; ++tb) {
                    const int ta = tb + sgn * m;
                    if (ta < 0 || ta >= n_t) continue;
                    rc = launch_cop(s1, s2, B.site, B.spin, B.dagger, K.vec(tb, 0), V + ((size_t)ta * n_t + tb) * d2,
                                    st);
                }
            }
            if (rc == KG_OK) rc = cudaStreamSynchronize(st) == cudaSuccess ? KG_OK : KG_ECUDA;
            if (rc == KG_OK) rc = block_status_of(K, "the four-time sweeps");
        }
        R.release();
        krylov_free(K);
    }
    if (rc != KG_OK || n_t < 2) return rc;
    // e^{iH t_a} on the n_t vectors of each t_a (t_a = 0 needs none)
    Krylov K;
    StepRunner R;
    rc = krylov_alloc(K, std::vector<const kg_sector*>(n_t, s2), std::min(o->M, (int)d2), fin->nsm, o->schedule);
    if (rc == KG_OK) {
        for (auto& D : K.hdesc) D.tau = -h;
        rc = krylov_upload(K, st);
    }
    if (rc == KG_OK) rc = R.init(K, o->reorth, st, o->use_graphs != 0);
    if (rc == KG_OK) rc = launch_reset_status(K, st);
    const size_t pitch = (size_t)(K.M + 1) * d2 * sizeof(double2);
    for (int ta = 1; rc == KG_OK && ta < n_t; ++ta) {
        double2* row = V + (size_t)ta * n_t * d2;
        if (cudaMemcpy2DAsync(K.vec(0, 0), pitch, row, d2 * sizeof(double2), d2 * sizeof(double2), n_t,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), "four-time columns in", __FILE__, __LINE__);
        if (rc == KG_OK) rc = grid_steps(R, ta, n_sub, st);
        if (rc == KG_OK && cudaMemcpy2DAsync(row, d2 * sizeof(double2), K.vec(0, 0), pitch, d2 * sizeof(double2), n_t,
                                             cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), "four-time columns out", __FILE__, __LINE__);
    }
    if (rc == KG_OK) rc = cudaStreamSynchronize(st) == cudaSuccess ? KG_OK : KG_ECUDA;
    if (rc == KG_OK) rc = block_status_of(K, "the four-time back-propagation");
    R.release();
    krylov_free(K);
    return rc;
}

// The sector after applying op to s, or null when it does not exist.
static int op_target(kg_sector* s, FourOp op, kg_sector** out) {
    *out = nullptr;
    const int nu = s->nu + (op.spin == 0 ? (op.dagger ? 1 : -1) : 0);
    const int nd = s->nd + (op.spin == 1 ? (op.dagger ? 1 : -1) : 0);
    if (nu < 0 || nd < 0 || nu > s->L || nd > s->L) return KG_OK;
    return neighbour(s, op.spin, op.dagger, out);
}

int green_four_time(kg_sector* ini, kg_sector* fin, const int* ops, double dt, int n_t, const kg_opts* o, double* G) {
    if (!ops || !G || n_t < 1 || !(dt >= 0.0) || !std::isfinite(dt)) {
        set_error("bad four-time arguments");
        return KG_EINVAL;
    }
    if (ini->L != fin->L || ini->nu != fin->nu || ini->nd != fin->nd) {
        set_error("H_ini and H_fin must share (L, N_up, N_dn)");
        return KG_EINVAL;
    }
    FourOp op[4];
    for (int i = 0; i < 4; ++i) {
        op[i] = FourOp{ops[3 * i], ops[3 * i + 1], ops[3 * i + 2]};
        if (op[i].site < 0 || op[i].site >= fin->L || (op[i].spin & ~1) || (op[i].dagger & ~1)) {
            set_error("operator %d: site in [0, L), spin and dagger 0 or 1", i);
            return KG_EINVAL;
        }
    }
    KG_TRY(check_opts(o));
    const size_t nv = (size_t)n_t * n_t;
    std::memset(G, 0, sizeof(double) * 2 * nv * nv);
    // sectors of the right (A4 then A3) and the left (A1^dag then A2^dag) vectors
    const FourOp l1op{op[0].site, op[0].spin, 1 - op[0].dagger}, l2op{op[1].site, op[1].spin, 1 - op[1].dagger};
    kg_sector *r1 = nullptr, *r2 = nullptr, *l1 = nullptr, *l2 = nullptr;
    KG_TRY(op_target(fin, op[3], &r1));
    if (r1) KG_TRY(op_target(r1, op[2], &r2));
    KG_TRY(op_target(fin, l1op, &l1));
    if (l1) KG_TRY(op_target(l1, l2op, &l2));
    if (!r2 || !l2 || r2->nu != l2->nu || r2->nd != l2->nd) return KG_OK;  // particle numbers not conserved
    KG_TRY(ensure_gs(ini, o));
    cudaStream_t st = pick_stream(fin, o);
    const int n_sub = (o->dt_internal > 0.0) ? std::max(1, (int)std::lround(dt / o->dt_internal)) : 1;
    const size_t d0 = (size_t)fin->d, d2 = (size_t)r2->d;
    double2 *phi = nullptr, *Rv = nullptr, *Lv = nullptr, *Gd = nullptr;
    auto done = [&](int r) {
        cudaFree(phi);
        cudaFree(Rv);
        cudaFree(Lv);
        cudaFree(Gd);
        return r;
    };
    if (cudaMalloc(&phi, sizeof(double2) * n_t * d0) != cudaSuccess ||
        cudaMalloc(&Rv, sizeof(double2) * nv * d2) != cudaSuccess ||
        cudaMalloc(&Lv, sizeof(double2) * nv * d2) != cudaSuccess ||
        cudaMalloc(&Gd, sizeof(double2) * nv * nv) != cudaSuccess) {
        cudaGetLastError();
        set_error("four-time vectors: 2 x %zu vectors of dimension %zu do not fit", nv, d2);
        return done(KG_ENOMEM);
    }
    // Phi(t_k) = e^{-iH t_k}|0>
    int rc = cudaMemcpyAsync(phi, ini->gs, sizeof(double2) * d0, cudaMemcpyDeviceToDevice, st) == cudaSuccess
                 ? KG_OK
                 : cuda_fail(cudaGetLastError(), "Phi(0)", __FILE__, __LINE__);
    if (rc == KG_OK && n_t > 1) {
        Krylov K;
        StepRunner R;
        rc = krylov_alloc(K, {fin}, std::min(o->M, (int)d0), fin->nsm, o->schedule);
        if (rc == KG_OK) {
            K.hdesc[0].tau = dt / n_sub;
            rc = krylov_upload(K, st);
        }
        if (rc == KG_OK && cudaMemcpyAsync(K.vec(0, 0), ini->gs, sizeof(double2) * d0, cudaMemcpyDeviceToDevice, st) !=
                               cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), "Phi start", __FILE__, __LINE__);
        if (rc == KG_OK) rc = R.init(K, o->reorth, st, o->use_graphs != 0);
        if (rc == KG_OK) rc = launch_reset_status(K, st);
        for (int k = 1; rc == KG_OK && k < n_t; ++k) {
            rc = grid_steps(R, 1, n_sub, st);
            if (rc == KG_OK && cudaMemcpyAsync(phi + k * d0, K.vec(0, 0), sizeof(double2) * d0,
                                               cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                rc = cuda_fail(cudaGetLastError(), "Phi(t_k)", __FILE__, __LINE__);
        }
        if (rc == KG_OK) rc = cudaStreamSynchronize(st) == cudaSuccess ? KG_OK : KG_ECUDA;
        if (rc == KG_OK) rc = block_status_of(K, "step (ii)");
        R.release();
        krylov_free(K);
    }
    if (rc == KG_OK) rc = pair_vectors(fin, r1, r2, op[3], op[2], phi, n_t, dt, n_sub, o, Rv, st);
    if (rc == KG_OK) rc = pair_vectors(fin, l1, l2, l1op, l2op, phi, n_t, dt, n_sub, o, Lv, st);
    // Gd[q * nv + p] = <L_p | R_q>, p = t2 n_t + t1, q = t3 n_t + t4
    for (size_t p0 = 0; rc == KG_OK && p0 < nv; p0 += kMaxOv) {
        const int np = (int)std::min<size_t>(kMaxOv, nv - p0);
        rc = launch_inner_lib(Lv + p0 * d2, np, Rv, (int)nv, (int)d2, Gd + p0, (int)nv, st);
    }
    std::vector<double2> h(nv * nv);
    if (rc == KG_OK && (cudaMemcpyAsync(h.data(), Gd, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
        rc = cuda_fail(cudaGetLastError(), "four-time readback", __FILE__, __LINE__);
    if (rc != KG_OK) return done(rc);
    for (int k1 = 0; k1 < n_t; ++k1)
        for (int k2 = 0; k2 < n_t; ++k2)
            for (int k3 = 0; k3 < n_t; ++k3)
                for (int k4 = 0; k4 < n_t; ++k4) {
                    const double2 v = h[((size_t)k3 * n_t + k4) * nv + ((size_t)k2 * n_t + k1)];
                    const size_t off = (((size_t)k1 * n_t + k2) * n_t + k3) * n_t + k4;
                    G[2 * off] = v.x;
                    G[2 * off + 1] = v.y;
                }
    return done(KG_OK);
}

}  // namespace kg

extern "C" int kg_green_matsubara_steps(kg_sector* s, const int* orb, int n_orb, double mu, double dtau,
                                        int n_steps, const kg_opts* o, double* G_plus, double* G_minus) {
    if (!s) {
        kg::set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    if (!o) {
        kg_opts_default(&tmp);
        o = &tmp;
    }
    return kg::green_matsubara_steps(s, orb, n_orb, mu, dtau, n_steps, o, G_plus, G_minus);
}

extern "C" int kg_green_equilibrium_fine(kg_sector* s, const int* orb, int n_orb, double dt, int n_steps, int fine,
                                         const kg_opts* o, double* G_gtr, double* G_les) {
    kg_opts tmp;
    if (!o) {
        kg_opts_default(&tmp);
        o = &tmp;
    }
    if (!s || fine < 1 || fine > 32) {
        kg::set_error("kg_green_equilibrium_fine: need a sector and 1 <= fine <= 32");
        return KG_EINVAL;
    }
    return kg::green_eq_batch(&s, 1, orb, n_orb, dt, n_steps, o, G_gtr, G_les, nullptr, false, fine);
}

extern "C" int kg_green_mixed(kg_sector* H_ini, kg_sector* H_fin, const int* orb, int n_orb, double dt, int n_t,
                              double mu, double dtau, int n_tau, const kg_opts* o, double* G_right, double* G_left) {
    if (!H_ini || !H_fin) {
        kg::set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    if (!o) {
        kg_opts_default(&tmp);
        o = &tmp;
    }
    return kg::green_mixed(H_ini, H_fin, orb, n_orb, dt, n_t, mu, dtau, n_tau, o, G_right, G_left);
}

extern "C" int kg_green_restarted(kg_sector* s, const int* orb, int n_orb, int n, int f, int q, double dt,
                                  const kg_opts* o, double* G_gtr, double* G_les) {
    if (!s) {
        kg::set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    if (!o) {
        kg_opts_default(&tmp);
        o = &tmp;
    }
    return kg::green_restarted(s, orb, n_orb, n, f, q, dt, o, G_gtr, G_les);
}
