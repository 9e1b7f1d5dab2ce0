// kg_adjoint.cu -- the adjoint (vector-Jacobian product) of the
// equilibrium Green's function with respect to the Hamiltonian parameters
// eps_{i sigma}, U_i and h_ij.  The paper has no gradients; this follows the
// structure of its propagation (Section 3, Eqs. (psit), (psigreen),
// (newstate), (udelta)):
//
//   G_{ab}(t_k) = p_k <chi_a | psi_b(t_k)>,  psi_b(t_k) = U^k chi_b,
//   U = exp(-i H tau), tau = +dt (particle, chi = c^dag|0>) or -dt (hole,
//   chi = c|0>), p_k = -i e^{i E0 t_k} or +i e^{-i E0 t_k}.
//
// For a loss L with cotangents Gbar = dL/dRe G + i dL/dIm G:
//   * adjoint states lambda_n = s_n, lambda_{k-1} = U^dag lambda_k + s_{k-1},
//     s_k = sum_a Gbar_{ab,k} conj(p_k) chi_a, propagated backward with the
//     same Krylov steps;
//   * each step contributes Re <lambda_k| dU |psi_{k-1}> with the Frechet
//     derivative dU = -i tau int_0^1 e^{-iH tau (1-x)} dH e^{-iH tau x} dx,
//     evaluated by Gauss-Legendre nodes x_q; the node vectors
//     e^{-iH tau x_q} psi_{k-1} and e^{+iH tau (1-x_q)} lambda_k come from the
//     Krylov spaces of that step (the paper's evaluation of Eq. (udelta) at
//     intermediate times), so they cost no extra H*psi;
//   * one fused kernel accumulates Re(c_q <w_q| dH/dtheta |u_q>) for every
//     parameter theta at once (occupations, double occupations, hops);
//   * the ground state enters through E0 (Hellmann-Feynman, <0|dH|0>) and
//     through |0> (a projected linear solve (H - E0) x = P z by conjugate
//     gradients, then -Re <x| dH |0>).
// Forward states are kept at checkpoints every `checkpoint` steps and
// recomputed segment by segment during the backward sweep.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "kg_internal.h"

namespace kg {

constexpr int kMaxNodes = 16;
constexpr int kMaxPairs = 128;

// ------------------------------------------------------- node vectors
// out[outoff[b] + t*d_b + i] = sum_k cq[b][t][k] V_k[i] for every column b
// of K (columns may differ in dimension d_b).
__global__ void __launch_bounds__(kThreads) k_lincomb(const ColDesc* desc, const ColScalars* cs, int Mcap,
                                                      const double2* cq, int ntau, double2* out,
                                                      const size_t* outoff) {
    __shared__ double2 c[kMaxNodes + 1][kMaxM];
    const int b = blockIdx.y;
    const ColDesc D = desc[b];
    const int m = cs[b].m_eff;
    for (int t = 0; t < ntau; ++t)
        for (int k = threadIdx.x; k < m; k += blockDim.x) c[t][k] = cq[((size_t)b * ntau + t) * Mcap + k];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D.d; i += gridDim.x * blockDim.x) {
        double2 acc[kMaxNodes + 1];
        for (int t = 0; t < ntau; ++t) acc[t] = make_double2(0.0, 0.0);
        for (int k = 0; k < m; ++k) {
            const double2 v = D.V[(size_t)k * D.d + i];
            for (int t = 0; t < ntau; ++t) {
                acc[t].x = fma(c[t][k].x, v.x, fma(-c[t][k].y, v.y, acc[t].x));
                acc[t].y = fma(c[t][k].x, v.y, fma(c[t][k].y, v.x, acc[t].y));
            }
        }
        for (int t = 0; t < ntau; ++t) out[outoff[b] + (size_t)t * D.d + i] = acc[t];
    }
}

// ---------------------------------------------------- parameter gradient
// For the pairs (u_q, w_q), q < nq, with complex weights c_q, accumulate
//   g[sigma*L + i]      += Re sum_q c_q <w_q| n_{i sigma} |u_q>
//   g[2L + i]           += Re sum_q c_q <w_q| n_{i up} n_{i dn} |u_q>
//   g[3L + 2p (+1)]     += Re (Im) sum_q c_q <w_q| sum_sigma c^dag_a c_b |u_q>
// for every ordered hop pair p = (a, b) of the sector's hop tables.
struct NodeWeights {
    double2 c[kMaxNodes];
};

__global__ void __launch_bounds__(kThreads) k_param_grad(SecView S, const double2* __restrict__ U,
                                                         const double2* __restrict__ Wv, NodeWeights wts, int nq,
                                                         const short* __restrict__ pairmap, int nparam,
                                                         double* partial) {
    __shared__ short pm[kMaxL * kMaxL];
    __shared__ double sm[(kThreads / 32) * (3 * kMaxL + 2 * kMaxPairs)];
    for (int k = threadIdx.x; k < S.L * S.L; k += blockDim.x) pm[k] = pairmap[k];
    __syncthreads();
    const int L = S.L;
    double acc[3 * kMaxL + 2 * kMaxPairs];
    for (int p = 0; p < nparam; ++p) acc[p] = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.d; s += gridDim.x * blockDim.x) {
        int i_dn, i_up;
        split_index(S, s, i_dn, i_up);
        double2 a[kMaxNodes];  // c_q conj(w_q[s])
        double P = 0.0;
        for (int q = 0; q < nq; ++q) {
            const double2 w = Wv[(size_t)q * S.d + s], u = U[(size_t)q * S.d + s];
            const double2 c = wts.c[q];
            a[q] = make_double2(c.x * w.x + c.y * w.y, c.y * w.x - c.x * w.y);
            P += a[q].x * u.x - a[q].y * u.y;
        }
        const uint32_t bu = S.up_bits[i_up], bd = S.dn_bits[i_dn];
        for (uint32_t m = bu; m; m &= m - 1u) acc[__ffs(m) - 1] += P;
        for (uint32_t m = bd; m; m &= m - 1u) acc[L + __ffs(m) - 1] += P;
        for (uint32_t m = bu & bd; m; m &= m - 1u) acc[2 * L + __ffs(m) - 1] += P;
        for (int pass = 0; pass < 2; ++pass) {
            const int e0 = pass == 0 ? S.up_off[i_up] : S.dn_off[i_dn];
            const int e1 = pass == 0 ? S.up_off[i_up + 1] : S.dn_off[i_dn + 1];
            for (int e = e0; e < e1; ++e) {
                const uint2 en = pass == 0 ? S.up_ent[e] : S.dn_ent[e];
                const size_t src = pass == 0 ? (size_t)i_dn * S.Du + en.x : (size_t)en.x * S.Du + i_up;
                double zr = 0.0, zi = 0.0;
                for (int q = 0; q < nq; ++q) {
                    const double2 u = U[(size_t)q * S.d + src];
                    zr += a[q].x * u.x - a[q].y * u.y;
                    zi += a[q].x * u.y + a[q].y * u.x;
                }
                if (en.y >> 31) {
                    zr = -zr;
                    zi = -zi;
                }
                const int p = pm[en.y & 1023u];
                acc[3 * L + 2 * p] += zr;
                acc[3 * L + 2 * p + 1] += zi;
            }
        }
    }
    // block reduction in a fixed order: warp sums, then warps in order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p = 0; p < nparam; ++p) {
        const double v = warp_sum(acc[p]);
        if (lane == 0) sm[warp * nparam + p] = v;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < nparam; p += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += sm[w * nparam + p];
        partial[(size_t)blockIdx.x * nparam + p] = t;
    }
}

__global__ void k_param_reduce(const double* partial, int nblk, int nparam, double* g) {
    for (int p = threadIdx.x; p < nparam; p += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < nblk; ++b) t += partial[(size_t)b * nparam + p];
        g[p] += t;
    }
}

// ----------------------------------------------------------- utilities
// y[b] += sum_a coef[b][a] x[a] for columns b < ny (complex, length d).
struct Coefs {
    double2 c[kMaxOv * kMaxOv];
};

__global__ void k_combo(const double2* __restrict__ X, int nx, double2* __restrict__ Y, int ny, int d, Coefs cf) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x)
        for (int b = 0; b < ny; ++b) {
            double2 y = Y[(size_t)b * d + i];
            for (int a = 0; a < nx; ++a) {
                const double2 c = cf.c[b * nx + a], x = X[(size_t)a * d + i];
                y.x = fma(c.x, x.x, fma(-c.y, x.y, y.x));
                y.y = fma(c.x, x.y, fma(c.y, x.x, y.y));
            }
            Y[(size_t)b * d + i] = y;
        }
}

// y = a x + b y (complex a, b)
__global__ void k_axpby(double2 a, const double2* __restrict__ x, double2 b, double2* __restrict__ y, int d) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        const double2 u = x[i], v = y[i];
        y[i] = make_double2(a.x * u.x - a.y * u.y + b.x * v.x - b.y * v.y, a.x * u.y + a.y * u.x + b.x * v.y + b.y * v.x);
    }
}

static int grid_for(int d) { return std::max(1, std::min((d + kThreads - 1) / kThreads, 148 * 8)); }

static int axpby(std::complex<double> a, const double2* x, std::complex<double> b, double2* y, int d, cudaStream_t st) {
    k_axpby<<<grid_for(d), kThreads, 0, st>>>(make_double2(a.real(), a.imag()), x, make_double2(b.real(), b.imag()), y, d);
    KG_LAUNCHED();
    return KG_OK;
}

// <x|y> (host result), through the overlap kernel
static int dotc(const double2* x, const double2* y, int d, double2* dscratch, std::complex<double>* out,
                cudaStream_t st) {
    KG_TRY(launch_inner_lib(x, 1, y, 1, d, dscratch, 1, st));
    double2 h;
    KG_CUDA(cudaMemcpyAsync(&h, dscratch, sizeof(double2), cudaMemcpyDeviceToHost, st));
    KG_CUDA(cudaStreamSynchronize(st));
    *out = std::complex<double>(h.x, h.y);
    return KG_OK;
}

// Gauss-Legendre nodes and weights on [0, 1] (Newton on the Legendre
// recurrence).
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        const double pi = 3.14159265358979323846;
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/((1-z^2) p'^2) on [-1,1], halved
    }
}

// Solves (H - E0) x = P z with P = 1 - |0><0| by conjugate gradients on the
// positive semi-definite projected operator; x stays orthogonal to |0>.
static int cg_projected(kg_sector* s, const double2* gs, double E0, const double2* z, double2* x, double tol,
                        int maxit, cudaStream_t st) {
    const int d = (int)s->d;
    double2 *r = nullptr, *p = nullptr, *Ap = nullptr, *sc = nullptr;
    KG_CUDA(cudaMalloc(&r, sizeof(double2) * d));
    KG_CUDA(cudaMalloc(&p, sizeof(double2) * d));
    KG_CUDA(cudaMalloc(&Ap, sizeof(double2) * d));
    KG_CUDA(cudaMalloc(&sc, sizeof(double2)));
    auto fin = [&](int rc) {
        cudaFree(r);
        cudaFree(p);
        cudaFree(Ap);
        cudaFree(sc);
        return rc;
    };
    auto project = [&](double2* v) -> int {
        std::complex<double> c;
        KG_TRY(dotc(gs, v, d, sc, &c, st));
        return axpby(-c, gs, 1.0, v, d, st);
    };
    if (cudaMemcpyAsync(r, z, sizeof(double2) * d, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(x, 0, sizeof(double2) * d, st) != cudaSuccess)
        return fin(KG_ECUDA);
    int rc = project(r);
    std::complex<double> rr;
    if (rc == KG_OK) rc = dotc(r, r, d, sc, &rr, st);
    const double rz = std::sqrt(std::max(0.0, rr.real()));
    if (rc != KG_OK || rz == 0.0) return fin(rc);
    if (cudaMemcpyAsync(p, r, sizeof(double2) * d, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return fin(KG_ECUDA);
    for (int it = 0; rc == KG_OK && it < maxit; ++it) {
        if ((rc = launch_hpsi(s, p, Ap, st)) != KG_OK) break;
        if ((rc = axpby(-E0, p, 1.0, Ap, d, st)) != KG_OK) break;
        if ((rc = project(Ap)) != KG_OK) break;
        std::complex<double> pAp;
        if ((rc = dotc(p, Ap, d, sc, &pAp, st)) != KG_OK) break;
        if (!(pAp.real() > 0.0)) break;
        const double alpha = rr.real() / pAp.real();
        if ((rc = axpby(alpha, p, 1.0, x, d, st)) != KG_OK) break;
        if ((rc = axpby(-alpha, Ap, 1.0, r, d, st)) != KG_OK) break;
        std::complex<double> rn;
        if ((rc = dotc(r, r, d, sc, &rn, st)) != KG_OK) break;
        if (std::sqrt(std::max(0.0, rn.real())) <= tol * rz) break;
        if ((rc = axpby(1.0, r, rn.real() / rr.real(), p, d, st)) != KG_OK) break;
        rr = rn;
    }
    if (rc == KG_OK) rc = project(x);
    return fin(rc);
}

// ----------------------------------------------------------- the driver
struct ParamMap {
    int L = 0, npairs = 0, nparam = 0;
    std::vector<short> map;  // a*L + b -> pair index
    std::vector<int2> pairs;
};

static ParamMap param_map(const kg_sector* s) {
    ParamMap P;
    P.L = s->L;
    P.map.assign(kMaxL * kMaxL, 0);
    for (int a = 0; a < s->L; ++a)
        for (int b = 0; b < s->L; ++b)
            if (a != b && (s->h_re[a * s->L + b] != 0.0 || s->h_im[a * s->L + b] != 0.0)) {
                P.map[a * s->L + b] = (short)P.pairs.size();
                P.pairs.push_back(make_int2(a, b));
            }
    P.npairs = (int)P.pairs.size();
    P.nparam = 3 * s->L + 2 * P.npairs;
    return P;
}

static int grad_pass(const kg_sector* sec, const double2* U, const double2* Wv, const std::vector<std::complex<double>>& c,
                     const short* dmap, const ParamMap& P, double* partial, int nblk, double* g, cudaStream_t st) {
    NodeWeights wts;
    const int nq = (int)c.size();
    for (int q = 0; q < nq; ++q) wts.c[q] = make_double2(c[q].real(), c[q].imag());
    ProfScope ps("param_grad", st);
    k_param_grad<<<nblk, kThreads, 0, st>>>(sec->view(), U, Wv, wts, nq, dmap, P.nparam, partial);
    KG_LAUNCHED();
    k_param_reduce<<<1, 256, 0, st>>>(partial, nblk, P.nparam, g);
    KG_LAUNCHED();
    return KG_OK;
}

// Lanczos space of every column's V_0 without the final combination (the
// caller forms the vectors it needs at the times it needs).
int build_space(Krylov& K, int reorth, cudaStream_t st) {
    KG_TRY(launch_colnorm(K, st));
    const bool ain = alpha_in_dots(K, reorth);
    for (int j = 0; j < K.M; ++j) {
        KG_TRY(launch_lanczos_hpsi(K, j, st, !ain));
        if (reorth >= 1)
            for (int k0 = 0; k0 <= j; k0 += kChunk)
                KG_TRY(launch_reorth_dots(K, j, k0, std::min(kChunk, j + 1 - k0), false, st));
        KG_TRY(launch_update(K, j, reorth, false, st));
        if (reorth >= 2) {
            for (int k0 = 0; k0 <= j; k0 += kChunk)
                KG_TRY(launch_reorth_dots(K, j, k0, std::min(kChunk, j + 1 - k0), true, st));
            KG_TRY(launch_update(K, j, reorth, true, st));
        }
    }
    return KG_OK;
}

int green_equilibrium_vjp(kg_sector* s, const int* orb, int n_orb, double dt, int n_steps, const kg_opts* o,
                          int checkpoint, const double* dGgtr, const double* dGles, double* g_eps, double* g_hre,
                          double* g_him, double* g_U) {
    if (!orb || n_orb < 1 || n_orb > kMaxOv || n_steps < 0 || !g_eps || !g_hre || !g_him || !g_U ||
        o->M < 1 || o->M > kMaxM) {
        set_error("bad arguments to the Green's-function adjoint");
        return KG_EINVAL;
    }
    for (int a = 0; a < n_orb; ++a)
        if (orb[2 * a] < 0 || orb[2 * a] >= s->L || (orb[2 * a + 1] != 0 && orb[2 * a + 1] != 1)) {
            set_error("orbital %d out of range", a);
            return KG_EINVAL;
        }
    if (!s->has_gs) KG_TRY(ground_state(s, o));
    const int Kc = std::max(1, checkpoint > 0 ? checkpoint : 20);
    cudaStream_t st = pick_stream(s, o);
    const int L = s->L, d0 = (int)s->d, rows = n_steps + 1, nq = 10;
    const ParamMap P = param_map(s);
    if (P.npairs > kMaxPairs) {
        set_error("too many hopping pairs for the adjoint (%d > %d)", P.npairs, kMaxPairs);
        return KG_EINVAL;
    }
    std::vector<double> xq, wq;
    gauss_legendre(nq, xq, wq);
    const double E0 = s->E0;
    const int nblk = 152 * 2;
    double *g = nullptr, *partial = nullptr;
    short* dmap = nullptr;
    double2* z = nullptr;
    KG_CUDA(cudaMalloc(&g, sizeof(double) * P.nparam));
    KG_CUDA(cudaMalloc(&partial, sizeof(double) * P.nparam * nblk));
    KG_CUDA(cudaMalloc(&dmap, sizeof(short) * kMaxL * kMaxL));
    KG_CUDA(cudaMalloc(&z, sizeof(double2) * d0));
    KG_CUDA(cudaMemsetAsync(g, 0, sizeof(double) * P.nparam, st));
    KG_CUDA(cudaMemsetAsync(z, 0, sizeof(double2) * d0, st));
    KG_CUDA(cudaMemcpyAsync(dmap, P.map.data(), sizeof(short) * kMaxL * kMaxL, cudaMemcpyHostToDevice, st));
    double Ebar = 0.0;
    std::vector<int> idx[2];
    for (int a = 0; a < n_orb; ++a) idx[orb[2 * a + 1]].push_back(a);
    std::vector<void*> frees;
    auto cleanup = [&](int rc) {
        for (void* p : frees) cudaFree(p);
        cudaFree(g);
        cudaFree(partial);
        cudaFree(dmap);
        cudaFree(z);
        return rc;
    };
    auto dalloc = [&](void** p, size_t bytes) -> int {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            set_error("adjoint workspace allocation failed");
            return KG_ENOMEM;
        }
        frees.push_back(*p);
        return KG_OK;
    };
    int rc = KG_OK;
    // ---- the (spin, kind) groups of columns, all propagated in the same
    // launches (like the forward): column b is orbital a of group g, a
    // vector of that group's neighbour sector
    struct Group {
        int spin, dagger, na, dn, col0;
        kg_sector* nb;
        double tau;
        std::vector<int> idx;
        std::vector<std::complex<double>> Gb, pk;  // cotangent Gbar_{ab,k}, phase p_k
    };
    std::vector<Group> grp;
    for (int spin = 0; spin < 2; ++spin) {
        if (idx[spin].empty()) continue;
        for (int dagger = 1; dagger >= 0; --dagger) {
            kg_sector* nb = nullptr;
            const double* dG = dagger ? dGgtr : dGles;
            if (!dG || neighbour(s, spin, dagger, &nb) != KG_OK) continue;
            Group G;
            G.spin = spin;
            G.dagger = dagger;
            G.na = (int)idx[spin].size();
            G.dn = (int)nb->d;
            G.nb = nb;
            G.tau = dagger ? dt : -dt;
            G.idx = idx[spin];
            const int na = G.na;
            G.Gb.resize((size_t)rows * na * na);
            G.pk.resize(rows);
            for (int k = 0; k < rows; ++k) {
                const double t = dt * k;
                G.pk[k] = dagger ? std::complex<double>(0, -1) * std::exp(std::complex<double>(0, E0 * t))
                                 : std::complex<double>(0, 1) * std::exp(std::complex<double>(0, -E0 * t));
                for (int a = 0; a < na; ++a)
                    for (int b = 0; b < na; ++b) {
                        // particle: G^>_{ab}; hole: G^<_{ba} = p <phi_a | psi_b>
                        const int r = dagger ? G.idx[a] : G.idx[b];
                        const int c = dagger ? G.idx[b] : G.idx[a];
                        const size_t e = ((size_t)k * n_orb + r) * n_orb + c;
                        G.Gb[((size_t)k * na + a) * na + b] = std::complex<double>(dG[2 * e], dG[2 * e + 1]);
                    }
            }
            grp.push_back(std::move(G));
        }
    }
    // columns: per-column sector, dimension and offsets into the concatenated buffers
    std::vector<const kg_sector*> cols;
    std::vector<int> colg;
    std::vector<size_t> off;  // element offset of column b in a [tot] buffer
    size_t tot = 0;
    for (int g = 0; g < (int)grp.size(); ++g) {
        grp[g].col0 = (int)cols.size();
        for (int a = 0; a < grp[g].na; ++a) {
            cols.push_back(grp[g].nb);
            colg.push_back(g);
            off.push_back(tot);
            tot += (size_t)grp[g].dn;
        }
    }
    const int NC = (int)cols.size();
    auto gcol = [&](int g) { return off[grp[g].col0]; };  // first element of group g
    Krylov KF, KB;
    double2 *chi = nullptr, *ckpt = nullptr, *seg = nullptr, *lam = nullptr, *y = nullptr, *Uq = nullptr,
            *Wq = nullptr, *ov = nullptr, *tmp = nullptr, *cqF = nullptr, *cqB = nullptr;
    double *tauF = nullptr, *tauB = nullptr;
    size_t *offU = nullptr, *offW = nullptr;
    const int nck = n_steps / Kc + 1;
    size_t nov = 0;
    for (auto& G : grp) nov += (size_t)G.na * rows * G.na;
    if (NC > 0) {
        rc = dalloc((void**)&chi, sizeof(double2) * tot);
        if (rc == KG_OK) rc = dalloc((void**)&ckpt, sizeof(double2) * (size_t)nck * tot);
        if (rc == KG_OK) rc = dalloc((void**)&seg, sizeof(double2) * (size_t)(Kc + 1) * tot);
        if (rc == KG_OK) rc = dalloc((void**)&lam, sizeof(double2) * tot);
        if (rc == KG_OK) rc = dalloc((void**)&y, sizeof(double2) * tot);
        if (rc == KG_OK) rc = dalloc((void**)&Uq, sizeof(double2) * (size_t)nq * tot);
        if (rc == KG_OK) rc = dalloc((void**)&Wq, sizeof(double2) * (size_t)(nq + 1) * tot);
        if (rc == KG_OK) rc = dalloc((void**)&ov, sizeof(double2) * nov);
        if (rc == KG_OK) rc = dalloc((void**)&tmp, sizeof(double2) * d0);
        if (rc == KG_OK) rc = dalloc((void**)&cqF, sizeof(double2) * (size_t)NC * nq * o->M);
        if (rc == KG_OK) rc = dalloc((void**)&cqB, sizeof(double2) * (size_t)NC * (nq + 1) * o->M);
        if (rc == KG_OK) rc = dalloc((void**)&tauF, sizeof(double) * NC * nq);
        if (rc == KG_OK) rc = dalloc((void**)&tauB, sizeof(double) * NC * (nq + 1));
        if (rc == KG_OK) rc = dalloc((void**)&offU, sizeof(size_t) * NC);
        if (rc == KG_OK) rc = dalloc((void**)&offW, sizeof(size_t) * NC);
    }
    std::vector<size_t> hOffU(NC), hOffW(NC), ovoff(grp.size());
    {
        size_t o2 = 0;
        for (int g = 0; g < (int)grp.size(); ++g) {
            ovoff[g] = o2;
            o2 += (size_t)grp[g].na * rows * grp[g].na;
        }
    }
    std::vector<double> hF((size_t)NC * nq), hB((size_t)NC * (nq + 1));
    for (int b = 0; b < NC; ++b) {
        hOffU[b] = off[b] * nq;
        hOffW[b] = off[b] * (nq + 1);
        const double tau = grp[colg[b]].tau;
        // node times: forward e^{-iH tau x_q}, backward e^{+iH tau (1-x_q)} and the full step
        for (int q = 0; q < nq; ++q) {
            hF[(size_t)b * nq + q] = tau * xq[q];
            hB[(size_t)b * (nq + 1) + q] = -tau * (1.0 - xq[q]);
        }
        hB[(size_t)b * (nq + 1) + nq] = -tau;
    }
    if (rc == KG_OK && NC > 0 &&
        (cudaMemcpyAsync(tauF, hF.data(), sizeof(double) * hF.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync(tauB, hB.data(), sizeof(double) * hB.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync(offU, hOffU.data(), sizeof(size_t) * NC, cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync(offW, hOffW.data(), sizeof(size_t) * NC, cudaMemcpyHostToDevice, st) != cudaSuccess))
        rc = KG_ECUDA;
    for (int b = 0; rc == KG_OK && b < NC; ++b) {
        const Group& G = grp[colg[b]];
        rc = launch_cop(s, G.nb, orb[2 * G.idx[b - G.col0]], G.spin, G.dagger, s->gs, chi + off[b], st);
    }
    // ---- forward pass: checkpoints and the overlaps (for dL/dE0)
    if (rc == KG_OK && NC > 0) rc = krylov_alloc(KF, cols, o->M, s->nsm, o->schedule);
    if (rc == KG_OK && NC > 0) rc = krylov_alloc(KB, cols, o->M, s->nsm, o->schedule);
    auto load = [&](Krylov& K, const double2* src) -> int {
        for (int b = 0; b < NC; ++b)
            KG_CUDA(cudaMemcpyAsync(K.vec(b, 0), src + off[b], sizeof(double2) * K.dim(b), cudaMemcpyDeviceToDevice,
                                    st));
        return KG_OK;
    };
    auto save = [&](Krylov& K, double2* dst) -> int {
        for (int b = 0; b < NC; ++b)
            KG_CUDA(cudaMemcpyAsync(dst + off[b], K.vec(b, 0), sizeof(double2) * K.dim(b), cudaMemcpyDeviceToDevice,
                                    st));
        return KG_OK;
    };
    if (rc == KG_OK && NC > 0) {
        for (int b = 0; b < NC; ++b) {
            const int g = colg[b], a = b - grp[g].col0;
            ColDesc& D = KF.hdesc[b];
            D.tau = grp[g].tau;
            D.ov = chi + gcol(g);
            D.n_ov = grp[g].na;
            D.ov_stride = grp[g].dn;
            D.ov_out = ov + ovoff[g] + (size_t)a * rows * grp[g].na;
            D.ov_rows = rows;
            KB.hdesc[b].tau = -grp[g].tau;
        }
        rc = krylov_upload(KF, st);
        if (rc == KG_OK) rc = krylov_upload(KB, st);
        for (int g = 0; rc == KG_OK && g < (int)grp.size(); ++g)
            rc = launch_inner_lib(chi + gcol(g), grp[g].na, chi + gcol(g), grp[g].na, grp[g].dn, ov + ovoff[g],
                                  rows * grp[g].na, st);
        if (rc == KG_OK) rc = launch_set_slots(KF, 1, st);
        if (rc == KG_OK) rc = load(KF, chi);
    }
    if (rc == KG_OK && NC > 0) {
        StepRunner RF;
        rc = RF.init(KF, o->reorth, st, o->use_graphs != 0);
        for (int k = 0; rc == KG_OK && k <= n_steps; ++k) {
            if (k % Kc == 0) rc = save(KF, ckpt + (size_t)(k / Kc) * tot);
            if (rc == KG_OK && k < n_steps) rc = RF.run(st);
        }
        RF.release();
    }
    std::vector<double2> hov(nov);
    if (rc == KG_OK && NC > 0)
        rc = cudaMemcpyAsync(hov.data(), ov, sizeof(double2) * nov, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                     cudaStreamSynchronize(st) == cudaSuccess
                 ? KG_OK
                 : KG_ECUDA;
    // dL/dE0: dp_k/dE0 = (+i t_k) p_k (particle) or (-i t_k) p_k (hole)
    for (int g = 0; rc == KG_OK && g < (int)grp.size(); ++g) {
        const Group& G = grp[g];
        const int na = G.na;
        for (int k = 0; k < rows; ++k) {
            const std::complex<double> dp = std::complex<double>(0.0, G.dagger ? dt * k : -dt * k) * G.pk[k];
            for (int b = 0; b < na; ++b)
                for (int a = 0; a < na; ++a) {
                    const double2 v = hov[ovoff[g] + ((size_t)b * rows + k) * na + a];
                    Ebar += (std::conj(G.Gb[((size_t)k * na + a) * na + b]) * dp * std::complex<double>(v.x, v.y)).real();
                }
        }
    }
    // ---- backward sweep, segment by segment
    auto sources = [&](int k, double2* dst) -> int {  // dst[b] += sum_a Gbar_{ab,k} conj(p_k) chi_a
        for (int g = 0; g < (int)grp.size(); ++g) {
            const Group& G = grp[g];
            const int na = G.na;
            Coefs cf;
            for (int b = 0; b < na; ++b)
                for (int a = 0; a < na; ++a) {
                    const std::complex<double> c = G.Gb[((size_t)k * na + a) * na + b] * std::conj(G.pk[k]);
                    cf.c[b * na + a] = make_double2(c.real(), c.imag());
                }
            k_combo<<<grid_for(G.dn), kThreads, 0, st>>>(chi + gcol(g), na, dst + gcol(g), na, G.dn, cf);
            KG_LAUNCHED();
        }
        return KG_OK;
    };
    auto bra_part = [&](int k, const double2* psi) -> int {  // y[a] += sum_b conj(Gbar_{ab,k}) p_k psi_b
        for (int g = 0; g < (int)grp.size(); ++g) {
            const Group& G = grp[g];
            const int na = G.na;
            Coefs cf;
            for (int a = 0; a < na; ++a)
                for (int b = 0; b < na; ++b) {
                    const std::complex<double> c = std::conj(G.Gb[((size_t)k * na + a) * na + b]) * G.pk[k];
                    cf.c[a * na + b] = make_double2(c.real(), c.imag());
                }
            k_combo<<<grid_for(G.dn), kThreads, 0, st>>>(psi + gcol(g), na, y + gcol(g), na, G.dn, cf);
            KG_LAUNCHED();
        }
        return KG_OK;
    };
    if (rc == KG_OK && NC > 0) rc = cudaMemsetAsync(lam, 0, sizeof(double2) * tot, st) == cudaSuccess ? KG_OK : KG_ECUDA;
    if (rc == KG_OK && NC > 0) rc = cudaMemsetAsync(y, 0, sizeof(double2) * tot, st) == cudaSuccess ? KG_OK : KG_ECUDA;
    if (rc == KG_OK && NC > 0) rc = sources(n_steps, lam);  // lambda_n = s_n
    std::vector<std::vector<std::complex<double>>> cw(grp.size(), std::vector<std::complex<double>>(nq));
    for (int g = 0; g < (int)grp.size(); ++g)
        for (int q = 0; q < nq; ++q) cw[g][q] = std::complex<double>(0.0, -grp[g].tau) * wq[q];
    if (rc == KG_OK && NC > 0) {
        StepRunner RS;
        // forward recompute inside a segment: plain steps without overlaps
        for (auto& D : KF.hdesc) {
            D.n_ov = 0;
            D.ov = nullptr;
        }
        rc = krylov_upload(KF, st);
        if (rc == KG_OK) rc = RS.init(KF, o->reorth, st, o->use_graphs != 0);
        // The Krylov spaces that the segment's forward steps build are kept
        // (basis and scalars per step) when the memory is there, so that the
        // backward sweep reads them instead of rebuilding them.
        const int MK = KF.M + 1;
        double2* segV = nullptr;
        ColScalars* segC = nullptr;
        if (rc == KG_OK && (cudaMalloc(&segV, sizeof(double2) * (size_t)Kc * MK * tot) != cudaSuccess ||
                            cudaMalloc(&segC, sizeof(ColScalars) * (size_t)Kc * NC) != cudaSuccess)) {
            cudaGetLastError();
            cudaFree(segV);
            cudaFree(segC);
            segV = nullptr;
            segC = nullptr;
        }
        if (segV) frees.push_back(segV);
        if (segC) frees.push_back(segC);
        std::vector<double2*> baseV(NC);
        for (int b = 0; b < NC; ++b) baseV[b] = KF.hdesc[b].V;
        auto segbase = [&](int step, int b) { return segV + (size_t)step * MK * tot + (size_t)MK * off[b]; };
        auto point_kf = [&](int step) -> int {  // step < 0: KF's own basis
            for (int b = 0; b < NC; ++b) KF.hdesc[b].V = step < 0 ? baseV[b] : segbase(step, b);
            KG_TRY(krylov_upload(KF, st));
            if (step >= 0)
                KG_CUDA(cudaMemcpyAsync(KF.cs, segC + (size_t)step * NC, sizeof(ColScalars) * NC,
                                        cudaMemcpyDeviceToDevice, st));
            return KG_OK;
        };
        for (int c = (n_steps - 1) / Kc; rc == KG_OK && c >= 0 && n_steps > 0; --c) {
            const int k0 = c * Kc, k1 = std::min(n_steps, k0 + Kc);
            rc = load(KF, ckpt + (size_t)c * tot);
            if (rc == KG_OK) rc = save(KF, seg);
            for (int k = k0 + 1; rc == KG_OK && k <= k1; ++k) {
                rc = RS.run(st);
                if (rc == KG_OK) rc = save(KF, seg + (size_t)(k - k0) * tot);
                if (rc == KG_OK && segV) {
                    // basis of the step k-1 -> k: v_0 = psi_{k-1}, then V_1..V_M as built
                    const int sidx = k - 1 - k0;
                    for (int b = 0; rc == KG_OK && b < NC; ++b) {
                        const int db = KF.dim(b);
                        double2* dst = segbase(sidx, b);
                        if (cudaMemcpyAsync(dst, seg + (size_t)sidx * tot + off[b], sizeof(double2) * db,
                                            cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                            cudaMemcpyAsync(dst + db, KF.vec(b, 1), sizeof(double2) * (size_t)(MK - 1) * db,
                                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                            rc = KG_ECUDA;
                    }
                    if (rc == KG_OK && cudaMemcpyAsync(segC + (size_t)sidx * NC, KF.cs, sizeof(ColScalars) * NC,
                                                       cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                        rc = KG_ECUDA;
                }
            }
            for (int k = k1; rc == KG_OK && k > k0; --k) {
                rc = bra_part(k, seg + (size_t)(k - k0) * tot);
                // forward space of psi_{k-1}: node vectors u_q
                if (segV) {
                    if (rc == KG_OK) rc = point_kf(k - 1 - k0);
                } else {
                    if (rc == KG_OK) rc = load(KF, seg + (size_t)(k - 1 - k0) * tot);
                    if (rc == KG_OK) rc = build_space(KF, o->reorth, st);
                }
                if (rc == KG_OK) rc = launch_tridiag_multi(KF, tauF, nq, cqF, st);
                if (rc == KG_OK) {
                    k_lincomb<<<dim3(grid_for((int)(tot / NC) + 1), NC), kThreads, 0, st>>>(KF.desc, KF.cs, KF.M, cqF,
                                                                                         nq, Uq, offU);
                    KG_LAUNCHED();
                }
                // backward space of lambda_k: node vectors w_q and U^dag lambda_k
                if (rc == KG_OK) rc = load(KB, lam);
                if (rc == KG_OK) rc = build_space(KB, o->reorth, st);
                if (rc == KG_OK) rc = launch_tridiag_multi(KB, tauB, nq + 1, cqB, st);
                if (rc == KG_OK) {
                    k_lincomb<<<dim3(grid_for((int)(tot / NC) + 1), NC), kThreads, 0, st>>>(KB.desc, KB.cs, KB.M, cqB,
                                                                                         nq + 1, Wq, offW);
                    KG_LAUNCHED();
                }
                for (int b = 0; rc == KG_OK && b < NC; ++b)
                    rc = grad_pass(grp[colg[b]].nb, Uq + hOffU[b], Wq + hOffW[b], cw[colg[b]], dmap, P, partial, nblk,
                                   g, st);
                // lambda_{k-1} = U^dag lambda_k + s_{k-1}
                for (int b = 0; rc == KG_OK && b < NC; ++b)
                    rc = cudaMemcpyAsync(lam + off[b], Wq + hOffW[b] + (size_t)nq * KB.dim(b),
                                         sizeof(double2) * KB.dim(b), cudaMemcpyDeviceToDevice, st) == cudaSuccess
                             ? KG_OK
                             : KG_ECUDA;
                if (rc == KG_OK) rc = sources(k - 1, lam);
            }
            if (rc == KG_OK && segV) rc = point_kf(-1);  // the step graph reads KF's own basis
        }
        RS.release();
    }
    if (rc == KG_OK && NC > 0) rc = bra_part(0, chi);
    // z += c_op^dag applied to lambda_0 and to y (back to the N sector)
    for (int b = 0; rc == KG_OK && b < NC; ++b) {
        const Group& G = grp[colg[b]];
        const int site = orb[2 * G.idx[b - G.col0]];
        for (int which = 0; rc == KG_OK && which < 2; ++which) {
            const double2* v = (which == 0 ? lam : y) + off[b];
            rc = launch_cop(G.nb, s, site, G.spin, G.dagger ? 0 : 1, v, tmp, st);
            if (rc == KG_OK) rc = axpby(1.0, tmp, 1.0, z, d0, st);
        }
    }
    // propagation states are checked for NaN/Inf by the Lanczos kernels
    if (rc == KG_OK && NC > 0) {
        std::vector<ColScalars> h(NC);
        if (cudaMemcpy(h.data(), KB.cs, sizeof(ColScalars) * NC, cudaMemcpyDeviceToHost) != cudaSuccess) rc = KG_ECUDA;
        for (auto& c : h)
            if (rc == KG_OK && c.status == KG_ENUMERIC) {
                set_error("non-finite value in the adjoint sweep");
                rc = KG_ENUMERIC;
            }
    }
    if (NC > 0) {
        krylov_free(KF);
        krylov_free(KB);
    }
    // ---- ground-state terms in the N sector
    double2* x = nullptr;
    if (rc == KG_OK && cudaMalloc(&x, sizeof(double2) * d0) != cudaSuccess) rc = KG_ENOMEM;
    if (x) frees.push_back(x);
    if (rc == KG_OK) rc = grad_pass(s, s->gs, s->gs, {std::complex<double>(Ebar, 0.0)}, dmap, P, partial, nblk, g, st);
    if (rc == KG_OK) rc = cg_projected(s, s->gs, s->E0, z, x, 1e-13, 20000, st);
    if (rc == KG_OK) rc = grad_pass(s, s->gs, x, {std::complex<double>(-1.0, 0.0)}, dmap, P, partial, nblk, g, st);
    std::vector<double> hg(P.nparam);
    if (rc == KG_OK)
        rc = cudaMemcpyAsync(hg.data(), g, sizeof(double) * P.nparam, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                     cudaStreamSynchronize(st) == cudaSuccess
                 ? KG_OK
                 : cuda_fail(cudaGetLastError(), "adjoint readback", __FILE__, __LINE__);
    if (rc != KG_OK) return cleanup(rc);
    // ---- map onto the parameters of the ABI
    for (int k = 0; k < 2 * L; ++k) g_eps[k] = hg[k];
    for (int i = 0; i < L; ++i) g_U[i] = hg[2 * L + i];
    std::memset(g_hre, 0, sizeof(double) * L * L);
    std::memset(g_him, 0, sizeof(double) * L * L);
    std::vector<double> R(P.npairs), I(P.npairs);
    for (int p = 0; p < P.npairs; ++p) {
        R[p] = hg[3 * L + 2 * p];
        I[p] = hg[3 * L + 2 * p + 1];
    }
    for (int p = 0; p < P.npairs; ++p) {
        const int a = P.pairs[p].x, b = P.pairs[p].y;
        if (a > b) continue;
        const int q = P.map[b * L + a];  // the reverse pair (Hermitian h has both)
        const double dre = R[p] + R[q];  // d/dRe h_ab with h_ba = conj(h_ab)
        const double dim = -I[p] + I[q];  // d/dIm h_ab
        g_hre[a * L + b] = g_hre[b * L + a] = dre;
        g_him[a * L + b] = dim;
        g_him[b * L + a] = -dim;
    }
    for (int i = 0; i < L; ++i) g_hre[i * L + i] = g_eps[i] + g_eps[L + i];
    return cleanup(KG_OK);
}

}  // namespace kg

extern "C" int kg_green_equilibrium_vjp(kg_sector* s, const int* orb, int n_orb, double dt, int n_steps,
                                        const kg_opts* o, int checkpoint, const double* dG_gtr, const double* dG_les,
                                        double* g_eps, double* g_hre, double* g_him, double* g_U) {
    if (!s) {
        kg::set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    if (!o) {
        kg_opts_default(&tmp);
        o = &tmp;
    }
    return kg::green_equilibrium_vjp(s, orb, n_orb, dt, n_steps, o, checkpoint, dG_gtr, dG_les, g_eps, g_hre, g_him,
                                     g_U);
}
