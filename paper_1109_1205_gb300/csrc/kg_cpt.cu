// kg_cpt.cu -- nonequilibrium cluster-perturbation theory (Section 5,
// Eq. (cpteq); the bath Green's function of Eqs. (gb1), (gb2)).
//
// The model of the paper's application: a cluster of L sites (H_ini, H_fin:
// the impurity model of Section 4) whose last site couples by the hopping V to
// the first site of a non-interacting chain of L_b sites with hopping -T_b
// (on-site energy and chemical potential 0).  Eq. (cpteq), G = (G'^{-1} -
// V)^{-1} on the Keldysh-Matsubara contour, with the bath integrated out, is
// the Dyson equation G = G' + G' * Delta * G of the cluster block, Delta =
// V^2 g_00 acting on the coupled site, * the contour integral.  The contour
// 0 -> t_max -> 0 -> -i beta is discretised by the trapezoidal rule (forward
// points t_j with weight dt, backward points with -dt, imaginary points
// -i tau_k with -i dtau, half weights at the ends of each branch), so
//   G_{Li} = (1 - G'_{LL} M)^{-1} G'_{Li},   G_{ii} = G'_{ii} + G'_{iL} M G_{Li},
// M = W Delta W.  The occupations n_i(t) = -i G^<_ii(t, t) come from the
// forward point t against the backward point t.
//
// The cluster's functions at inverse temperature beta are assembled from the
// zero-temperature components of the four-step method (G^>, G^<, G^right,
// G^left, G^M; the library's GPU routines) plus the antiperiodic tails that
// the trace adds near the end of the imaginary branch (terms of relative size
// e^{-beta gap} are dropped):
//   G(t, -i tau)  = G^right(t, tau) + conj(G^left_{ji}(beta - tau, t)),
//   G(-i tau, t)  = G^left(tau, t) + conj(G^right_{ji}(t, beta - tau)),
//   G(-i tau, -i tau') = i G^M_beta(tau - tau'),
//   G^M_beta(tau) = G^M(tau) - G^M(tau - beta), G^M_beta(-tau) = G^M(-tau) - G^M(beta - tau).
// On the diagonal z = z' every function takes the mean of its two orderings.
//
// The dense linear algebra of the contour (the matrix product, the LU
// factorisation with partial pivoting and the solves, complex FP64 on
// matrices of 2 n_t + n_tau + 1 contour points) runs in the kernels below;
// the assembly of the contour matrices from the components is host work.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "kg_internal.h"

namespace kg {

using cplx = std::complex<double>;

__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double s = 1.0 / fma(b.x, b.x, b.y * b.y);
    return make_double2(fma(a.x, b.x, a.y * b.y) * s, fma(a.y, b.x, -a.x * b.y) * s);
}

// C (m x n) = scale A (m x kd) B (kd x n) (+ C when accumulating), column-major,
// 16 x 16 tiles staged in shared memory.
constexpr int kZT = 16;
constexpr size_t kCptMaxColumn = 3072u * sizeof(double2);  // one right-hand side in shared memory
__global__ void __launch_bounds__(kZT* kZT) k_zgemm(const double2* __restrict__ A, int lda,
                                                    const double2* __restrict__ B, int ldb, double2* __restrict__ C,
                                                    int ldc, int m, int n, int kd, double scale, int accumulate) {
    __shared__ double2 As[kZT][kZT + 1];
    __shared__ double2 Bs[kZT][kZT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.x * kZT + tx, col = blockIdx.y * kZT + ty;
    double2 acc = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < kd; k0 += kZT) {
        // As[r][c] = A(row0 + r, k0 + c); Bs[r][c] = B(k0 + r, col0 + c)
        const int ar = blockIdx.x * kZT + tx, ac = k0 + ty;
        As[tx][ty] = (ar < m && ac < kd) ? A[(size_t)ac * lda + ar] : make_double2(0.0, 0.0);
        const int br = k0 + tx, bc = blockIdx.y * kZT + ty;
        Bs[tx][ty] = (br < kd && bc < n) ? B[(size_t)bc * ldb + br] : make_double2(0.0, 0.0);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kZT; ++q) {
            const double2 a = As[tx][q], b = Bs[q][ty];
            acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
            acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
        }
        __syncthreads();
    }
    if (row < m && col < n) {
        double2* c = C + (size_t)col * ldc + row;
        double2 r = make_double2(scale * acc.x, scale * acc.y);
        if (accumulate) {
            r.x += c->x;
            r.y += c->y;
        }
        *c = r;
    }
}

static int zgemm(const double2* A, int lda, const double2* B, int ldb, double2* C, int ldc, int m, int n, int kd,
                 double scale, bool accumulate, cudaStream_t st) {
    const dim3 blk(kZT, kZT), grd((m + kZT - 1) / kZT, (n + kZT - 1) / kZT);
    k_zgemm<<<grd, blk, 0, st>>>(A, lda, B, ldb, C, ldc, m, n, kd, scale, accumulate ? 1 : 0);
    KG_LAUNCHED();
    return KG_OK;
}

// LU step k (column-major n x n): the pivot of column k (largest |K_ik|^2,
// i >= k, the first such row on ties), rows k and p swapped over all columns,
// the column below the pivot divided by it.  A zero pivot sets *info.
constexpr int kLuThreads = 1024;
__global__ void __launch_bounds__(kLuThreads) k_lu_pivot(double2* K, int n, int k, int* perm, int* info) {
    __shared__ double sv[kLuThreads / 32];
    __shared__ int si[kLuThreads / 32];
    __shared__ int piv;
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
        const double2 v = K[(size_t)k * n + i];
        const double a = fma(v.x, v.x, v.y * v.y);
        if (a > best) {
            best = a;
            bi = i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    if ((threadIdx.x & 31) == 0) {
        sv[threadIdx.x >> 5] = best;
        si[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = sv[0];
        int p = si[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sv[w] > b || (sv[w] == b && si[w] < p)) {
                b = sv[w];
                p = si[w];
            }
        piv = p;
        perm[k] = p;
        if (!(b > 0.0)) *info = 1;
    }
    __syncthreads();
    const int p = piv;
    if (p != k)
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double2 t = K[(size_t)j * n + k];
            K[(size_t)j * n + k] = K[(size_t)j * n + p];
            K[(size_t)j * n + p] = t;
        }
    __syncthreads();
    const double2 d = K[(size_t)k * n + k];
    if (d.x == 0.0 && d.y == 0.0) return;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) K[(size_t)k * n + i] = zdiv(K[(size_t)k * n + i], d);
}

// Trailing update of step k: K_ij -= K_ik K_kj for i, j > k.
__global__ void __launch_bounds__(kThreads) k_lu_update(double2* K, int n, int k) {
    const int r = n - k - 1;
    const long long total = (long long)r * r;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = k + 1 + (int)(e % r), j = k + 1 + (int)(e / r);
        const double2 a = K[(size_t)k * n + i], b = K[(size_t)j * n + k];
        double2& c = K[(size_t)j * n + i];
        c.x -= fma(a.x, b.x, -a.y * b.y);
        c.y -= fma(a.x, b.y, a.y * b.x);
    }
}

// One right-hand side per block: X = K^{-1} X from the factorisation (row
// swaps, unit lower then upper triangle), the column held in shared memory.
__global__ void __launch_bounds__(kThreads) k_lu_solve(const double2* __restrict__ K, int n, const int* perm,
                                                       double2* X, int ldx) {
    extern __shared__ double2 s[];
    double2* x = X + (size_t)blockIdx.x * ldx;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = x[i];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < n; ++k) {
            const int p = perm[k];
            if (p != k) {
                const double2 t = s[k];
                s[k] = s[p];
                s[p] = t;
            }
        }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const double2 v = s[k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const double2 l = K[(size_t)k * n + i];
            s[i].x -= fma(l.x, v.x, -l.y * v.y);
            s[i].y -= fma(l.x, v.y, l.y * v.x);
        }
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        if (threadIdx.x == 0) s[k] = zdiv(s[k], K[(size_t)k * n + k]);
        __syncthreads();
        const double2 v = s[k];
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            const double2 u = K[(size_t)k * n + i];
            s[i].x -= fma(u.x, v.x, -u.y * v.y);
            s[i].y -= fma(u.x, v.y, u.y * v.x);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = s[i];
}

// ------------------------------------------------------------- contour
// Positions p = 0..n_t-1 forward (t_p), n_t..2n_t-1 backward (t_{2n_t-1-p}),
// 2n_t..2n_t+n_tau imaginary (tau_{p-2n_t}); a later point has a larger p.
struct Contour {
    int n_t, n_tau, n;
    double dt, dtau;
    int kind(int p) const { return p < n_t ? 0 : (p < 2 * n_t ? 1 : 2); }
    int index(int p) const { return p < n_t ? p : (p < 2 * n_t ? 2 * n_t - 1 - p : p - 2 * n_t); }
    cplx weight(int p) const {
        const int k = kind(p), j = index(p);
        if (k < 2) {
            if (n_t < 2) return 0.0;
            const double w = dt * ((j == 0 || j == n_t - 1) ? 0.5 : 1.0);
            return k == 0 ? w : -w;
        }
        return cplx(0.0, -dtau * ((j == 0 || j == n_tau) ? 0.5 : 1.0));
    }
};

// The cluster's zero-temperature components of one spin, host complex arrays.
struct Components {
    int L = 0, n_t = 0, n_tau = 0;
    std::vector<cplx> les, gtr;    // [n_t][n_t][L][L]
    std::vector<cplx> right, left;  // [n_t][n_tau+1][L][L], [n_tau+1][n_t][L][L]
    std::vector<cplx> mp, mm;       // G^M(+tau_k), G^M(-tau_k): [n_tau+1][L][L]
    cplx kel(const std::vector<cplx>& g, int k, int l, int a, int b) const {
        return g[(((size_t)k * n_t + l) * L + a) * L + b];
    }
    cplx rgt(int k, int j, int a, int b) const { return right[(((size_t)k * (n_tau + 1) + j) * L + a) * L + b]; }
    cplx lft(int j, int k, int a, int b) const { return left[(((size_t)j * n_t + k) * L + a) * L + b]; }
    cplx mat(const std::vector<cplx>& g, int k, int a, int b) const { return g[((size_t)k * L + a) * L + b]; }
    // G^M_beta(+tau_k), G^M_beta(-tau_k) with the antiperiodic tails
    cplx gm_pos(int k, int a, int b) const { return mat(mp, k, a, b) - mat(mm, n_tau - k, a, b); }
    cplx gm_neg(int k, int a, int b) const { return mat(mm, k, a, b) - mat(mp, n_tau - k, a, b); }
    // G'_{ab}(z_p, z_q) on the contour
    cplx value(const Contour& C, int a, int b, int p, int q) const {
        const int kp = C.kind(p), kq = C.kind(q), ip = C.index(p), iq = C.index(q);
        if (kp < 2 && kq < 2) {
            const cplx later = kel(gtr, ip, iq, a, b), earlier = kel(les, ip, iq, a, b);
            return p > q ? later : (p < q ? earlier : 0.5 * (later + earlier));
        }
        if (kp < 2) return rgt(ip, iq, a, b) + std::conj(lft(n_tau - iq, ip, b, a));
        if (kq < 2) return lft(ip, iq, a, b) + std::conj(rgt(iq, n_tau - ip, b, a));
        const cplx I(0.0, 1.0);
        if (ip > iq) return I * gm_pos(ip - iq, a, b);
        if (ip < iq) return I * gm_neg(iq - ip, a, b);
        return I * 0.5 * (gm_pos(0, a, b) + gm_neg(0, a, b));
    }
};

static int cluster_components(kg_sector* ini, kg_sector* fin, int spin, const Contour& C, double beta,
                              const kg_opts* o, Components& X) {
    const int L = fin->L;
    X.L = L;
    X.n_t = C.n_t;
    X.n_tau = C.n_tau;
    std::vector<int> orb(2 * L);
    for (int i = 0; i < L; ++i) {
        orb[2 * i] = i;
        orb[2 * i + 1] = spin;
    }
    const size_t kk = (size_t)C.n_t * C.n_t * L * L, mx = (size_t)C.n_t * (C.n_tau + 1) * L * L,
                 mm = (size_t)(C.n_tau + 1) * L * L;
    X.les.assign(kk, 0.0);
    X.gtr.assign(kk, 0.0);
    X.right.assign(mx, 0.0);
    X.left.assign(mx, 0.0);
    X.mp.assign(mm, 0.0);
    X.mm.assign(mm, 0.0);
    auto d = [](std::vector<cplx>& v) { return reinterpret_cast<double*>(v.data()); };
    KG_TRY(green_keldysh(ini, fin, orb.data(), L, C.dt, C.n_t, o, d(X.les), d(X.gtr)));
    KG_TRY(green_mixed(ini, fin, orb.data(), L, C.dt, C.n_t, 0.0, beta / C.n_tau, C.n_tau, o, d(X.right), d(X.left)));
    KG_TRY(green_matsubara_steps(ini, orb.data(), L, 0.0, beta / C.n_tau, C.n_tau, o, d(X.mp), d(X.mm)));
    return KG_OK;
}

// Delta(z_p, z_q) = V^2 g_00(z_p, z_q): the first site of the chain of L_b
// sites, modes e_n = -2 T_b cos(n pi / (L_b + 1)), first components
// w_n = 2 / (L_b + 1) sin^2(n pi / (L_b + 1)); Eqs. (gb1), (gb2) with
// f(e) = 1 / (e^{beta e} + 1).  Each ordering depends on the complex time
// difference only, so the sums over the modes are tabulated per difference.
static void bath_delta(const Contour& C, int L_b, double T_b, double V, double beta, std::vector<cplx>& D) {
    const int n = C.n, nt = C.n_t, ntau = C.n_tau;
    const double kPi = 3.14159265358979323846;
    std::vector<double> e(L_b), w(L_b), f(L_b);
    for (int m = 0; m < L_b; ++m) {
        const double th = kPi * (m + 1) / (L_b + 1);
        e[m] = -2.0 * T_b * std::cos(th);
        w[m] = 2.0 / (L_b + 1) * std::sin(th) * std::sin(th);
        f[m] = 1.0 / (std::exp(beta * e[m]) + 1.0);
    }
    const cplx I(0.0, 1.0);
    // per-mode factors: phases e^{-i e t_j}, imaginary-time weights
    // w f e^{e tau_l} (real earlier) and w (1 - f) e^{-e tau_l} (imaginary later)
    std::vector<cplx> ph((size_t)nt * L_b);
    std::vector<double> ep((size_t)(ntau + 1) * L_b), em((size_t)(ntau + 1) * L_b);
    for (int j = 0; j < nt; ++j)
        for (int m = 0; m < L_b; ++m) ph[(size_t)j * L_b + m] = std::exp(-I * (e[m] * j * C.dt));
    for (int l = 0; l <= ntau; ++l)
        for (int m = 0; m < L_b; ++m) {
            ep[(size_t)l * L_b + m] = w[m] * f[m] * std::exp(e[m] * l * C.dtau);
            em[(size_t)l * L_b + m] = w[m] * (1.0 - f[m]) * std::exp(-e[m] * l * C.dtau);
        }
    // real-real: difference k = j_p - j_q in [-(nt-1), nt-1]
    std::vector<cplx> rr_later(2 * nt - 1), rr_earlier(2 * nt - 1);
    for (int k = -(nt - 1); k <= nt - 1; ++k) {
        cplx a = 0.0, b = 0.0;
        for (int m = 0; m < L_b; ++m) {
            const cplx z = k >= 0 ? ph[(size_t)k * L_b + m] : std::conj(ph[(size_t)(-k) * L_b + m]);
            a += w[m] * (1.0 - f[m]) * z;
            b += w[m] * f[m] * z;
        }
        rr_later[k + nt - 1] = -I * a;
        rr_earlier[k + nt - 1] = I * b;
    }
    // real (earlier) - imaginary: e^{-i e (t_j + i tau_l)}; imaginary (later)
    // - real: e^{-i e (-i tau_l - t_j)}
    std::vector<cplx> ri((size_t)nt * (ntau + 1)), ir((size_t)nt * (ntau + 1));
    for (int j = 0; j < nt; ++j)
        for (int l = 0; l <= ntau; ++l) {
            cplx a = 0.0, b = 0.0;
            const cplx* z = &ph[(size_t)j * L_b];
            const double* pp = &ep[(size_t)l * L_b];
            const double* pm = &em[(size_t)l * L_b];
            for (int m = 0; m < L_b; ++m) {
                a += pp[m] * z[m];
                b += pm[m] * std::conj(z[m]);
            }
            ri[(size_t)j * (ntau + 1) + l] = I * a;
            ir[(size_t)j * (ntau + 1) + l] = -I * b;
        }
    // imaginary-imaginary: l_p - l_q = dl (later) or -dl (earlier)
    std::vector<cplx> ii_later(ntau + 1), ii_earlier(ntau + 1);
    for (int dl = 0; dl <= ntau; ++dl) {
        double a = 0.0, b = 0.0;
        for (int m = 0; m < L_b; ++m) {
            a += w[m] * (1.0 - f[m]) * std::exp(-e[m] * dl * C.dtau);
            b += w[m] * f[m] * std::exp(e[m] * dl * C.dtau);
        }
        ii_later[dl] = -I * a;
        ii_earlier[dl] = I * b;
    }
    D.assign((size_t)n * n, 0.0);
    const double v2 = V * V;
    for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
            const int kp = C.kind(p), kq = C.kind(q), ip = C.index(p), iq = C.index(q);
            cplx g;
            if (kp < 2 && kq < 2) {
                const int k = ip - iq + nt - 1;
                g = p > q ? rr_later[k] : (p < q ? rr_earlier[k] : 0.5 * (rr_later[k] + rr_earlier[k]));
            } else if (kp < 2) {
                g = ri[(size_t)ip * (ntau + 1) + iq];
            } else if (kq < 2) {
                g = ir[(size_t)iq * (ntau + 1) + ip];
            } else if (ip > iq) {
                g = ii_later[ip - iq];
            } else if (ip < iq) {
                g = ii_earlier[iq - ip];
            } else {
                g = 0.5 * (ii_later[0] + ii_earlier[0]);
            }
            D[(size_t)q * n + p] = v2 * g;
        }
}

__global__ void k_set_identity(double2* K, int n) {
    const size_t nn = (size_t)n * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x)
        K[e] = make_double2((e % n) == (e / n) ? 1.0 : 0.0, 0.0);
}

// One spin: the cluster components, the contour matrices, K = 1 - A M on the
// device, its LU factorisation, Y = K^{-1} Y, MY = M Y, then the occupations.
struct CptWork {
    double2 *M = nullptr, *A = nullptr, *K = nullptr, *Y = nullptr, *MY = nullptr;
    int *perm = nullptr, *info = nullptr;
};

static int necpt_spin(kg_sector* ini, kg_sector* fin, int spin, const Contour& C, double beta, const kg_opts* o,
                      CptWork& Wk, cudaStream_t st, double* n_out) {
    const int n = C.n, L = fin->L, n_t = C.n_t, nrhs = L * n_t, Ls = L - 1;
    const size_t nn = (size_t)n * n, ny = (size_t)n * nrhs;
    Components X;
    KG_TRY(cluster_components(ini, fin, spin, C, beta, o, X));
    // A = G'_{LL}; right-hand sides Y[:, (i, t)] = G'_{Li}(., b_t); rows
    // Brow[(i, t), :] = G'_{iL}(f_t, .); diag0 = G'_{ii}(f_t, b_t)
    std::vector<cplx> A(nn), Y(ny), Brow(ny), MY(ny), diag0((size_t)nrhs);
    for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) A[(size_t)q * n + p] = X.value(C, Ls, Ls, p, q);
    for (int i = 0; i < L; ++i)
        for (int t = 0; t < n_t; ++t) {
            const int col = i * n_t + t, f = t, b = 2 * n_t - 1 - t;
            for (int p = 0; p < n; ++p) {
                Y[(size_t)col * n + p] = X.value(C, Ls, i, p, b);
                Brow[(size_t)col * n + p] = X.value(C, i, Ls, f, p);
            }
            diag0[col] = X.value(C, i, i, f, b);
        }
    KG_CUDA(cudaMemcpyAsync(Wk.A, A.data(), sizeof(double2) * nn, cudaMemcpyHostToDevice, st));
    KG_CUDA(cudaMemcpyAsync(Wk.Y, Y.data(), sizeof(double2) * ny, cudaMemcpyHostToDevice, st));
    const int nbe = (int)std::min<size_t>((nn + kThreads - 1) / kThreads, (size_t)fin->nsm * 8);
    k_set_identity<<<nbe, kThreads, 0, st>>>(Wk.K, n);
    KG_LAUNCHED();
    KG_TRY(zgemm(Wk.A, n, Wk.M, n, Wk.K, n, n, n, n, -1.0, true, st));
    KG_CUDA(cudaMemsetAsync(Wk.info, 0, sizeof(int), st));
    for (int k = 0; k < n; ++k) {
        k_lu_pivot<<<1, kLuThreads, 0, st>>>(Wk.K, n, k, Wk.perm, Wk.info);
        KG_LAUNCHED();
        const long long r = (long long)(n - k - 1) * (n - k - 1);
        if (r > 0) {
            const int nb = (int)std::min<long long>((r + kThreads - 1) / kThreads, (long long)fin->nsm * 8);
            k_lu_update<<<nb, kThreads, 0, st>>>(Wk.K, n, k);
            KG_LAUNCHED();
        }
    }
    k_lu_solve<<<nrhs, kThreads, sizeof(double2) * n, st>>>(Wk.K, n, Wk.perm, Wk.Y, n);
    KG_LAUNCHED();
    KG_TRY(zgemm(Wk.M, n, Wk.Y, n, Wk.MY, n, n, nrhs, n, 1.0, false, st));
    int info = 0;
    KG_CUDA(cudaMemcpyAsync(&info, Wk.info, sizeof(int), cudaMemcpyDeviceToHost, st));
    KG_CUDA(cudaMemcpyAsync(MY.data(), Wk.MY, sizeof(double2) * ny, cudaMemcpyDeviceToHost, st));
    KG_CUDA(cudaStreamSynchronize(st));
    if (info) {
        set_error("NE-CPT: the contour matrix 1 - G' W Delta W is singular");
        return KG_ENUMERIC;
    }
    // G_ii(f_t, b_t) = G'_ii + Brow . (M Y); n = Re(-i G^<)
    for (int i = 0; i < L; ++i)
        for (int t = 0; t < n_t; ++t) {
            const int col = i * n_t + t;
            cplx g = diag0[col];
            for (int p = 0; p < n; ++p) g += Brow[(size_t)col * n + p] * MY[(size_t)col * n + p];
            const double occ = (cplx(0.0, -1.0) * g).real();
            if (!std::isfinite(occ)) {
                set_error("NE-CPT: non-finite occupation");
                return KG_ENUMERIC;
            }
            n_out[((size_t)spin * n_t + t) * L + i] = occ;
        }
    return KG_OK;
}

int necpt_occupations(kg_sector* ini, kg_sector* fin, int L_b, double T_b, double V, double dt, int n_t, double beta,
                      int n_tau, const kg_opts* o, double* n_out) {
    if (!n_out || L_b < 1 || n_t < 1 || n_tau < 2 || !(dt >= 0.0) || !std::isfinite(dt) || !(beta > 0.0) ||
        !std::isfinite(beta) || !std::isfinite(V) || !std::isfinite(T_b)) {
        set_error("NE-CPT: need L_b >= 1, n_t >= 1, n_tau >= 2, finite dt >= 0, beta > 0, V and T_b");
        return KG_EINVAL;
    }
    if (ini->L != fin->L || ini->nu != fin->nu || ini->nd != fin->nd) {
        set_error("H_ini and H_fin must share (L, N_up, N_dn)");
        return KG_EINVAL;
    }
    const Contour C{n_t, n_tau, 2 * n_t + n_tau + 1, dt, beta / n_tau};
    const int n = C.n, nrhs = fin->L * n_t;
    if ((size_t)n * sizeof(double2) > kCptMaxColumn) {
        set_error("NE-CPT: %d contour points exceed the solver's column of %zu bytes", n, kCptMaxColumn);
        return KG_EINVAL;
    }
    if (o->M < 1 || o->M > kMaxM) {
        set_error("NE-CPT: Krylov dimension M must be in [1, %d]", kMaxM);
        return KG_EINVAL;
    }
    cudaStream_t st = pick_stream(fin, o);
    // M = W Delta W (host), shared by both spins
    std::vector<cplx> D;
    bath_delta(C, L_b, T_b, V, beta, D);
    std::vector<cplx> w(n);
    for (int p = 0; p < n; ++p) w[p] = C.weight(p);
    for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) D[(size_t)q * n + p] *= w[p] * w[q];
    CptWork Wk;
    auto done = [&](int r) {
        cudaFree(Wk.M);
        cudaFree(Wk.A);
        cudaFree(Wk.K);
        cudaFree(Wk.Y);
        cudaFree(Wk.MY);
        cudaFree(Wk.perm);
        cudaFree(Wk.info);
        return r;
    };
    const size_t nn = (size_t)n * n, ny = (size_t)n * nrhs;
    if (cudaMalloc(&Wk.M, sizeof(double2) * nn) != cudaSuccess || cudaMalloc(&Wk.A, sizeof(double2) * nn) != cudaSuccess ||
        cudaMalloc(&Wk.K, sizeof(double2) * nn) != cudaSuccess || cudaMalloc(&Wk.Y, sizeof(double2) * ny) != cudaSuccess ||
        cudaMalloc(&Wk.MY, sizeof(double2) * ny) != cudaSuccess ||
        cudaMalloc(&Wk.perm, sizeof(int) * n) != cudaSuccess || cudaMalloc(&Wk.info, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error("NE-CPT: contour matrices of %d points do not fit", n);
        return done(KG_ENOMEM);
    }
    if (cudaMemcpy(Wk.M, D.data(), sizeof(double2) * nn, cudaMemcpyHostToDevice) != cudaSuccess)
        return done(cuda_fail(cudaGetLastError(), "NE-CPT bath upload", __FILE__, __LINE__));
    for (int spin = 0; spin < 2; ++spin) {
        const int rc = necpt_spin(ini, fin, spin, C, beta, o, Wk, st, n_out);
        if (rc != KG_OK) return done(rc);
    }
    return done(KG_OK);
}

}  // namespace kg

extern "C" int kg_necpt_occupations(kg_sector* H_ini, kg_sector* H_fin, int L_b, double T_b, double V, double dt,
                                    int n_t, double beta, int n_tau, const kg_opts* o, double* n_out) {
    if (!H_ini || !H_fin) {
        kg::set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    if (!o) {
        kg_opts_default(&tmp);
        o = &tmp;
    }
    return kg::necpt_occupations(H_ini, H_fin, L_b, T_b, V, dt, n_t, beta, n_tau, o, n_out);
}
