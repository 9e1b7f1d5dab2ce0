// kg_krylov.cu -- a3-a5: the Lanczos recursion with full
// reorthogonalisation, the small tridiagonal eigenproblem and exponential,
// and the basis combination (Section 2, Eqs. (recursion), (tmatrix),
// (tdiag), (eigen); Section 3, Eqs. (newstate) and (udelta)).
//
// Every kernel works on B independent columns (blockIdx.y = column) of one
// sector.  Lanczos vectors are stored unnormalised, V_k, with v_k = s_k V_k
// and s_k = 1/||V_k|| kept on the device, so normalisation never costs a
// separate pass.  Scalars (a_k, b_k, Gram-Schmidt coefficients, combination
// coefficients) never leave the device: a whole propagation step is a fixed
// launch sequence that a CUDA graph can replay.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "kg_internal.h"

namespace kg {

int krylov_alloc(Krylov& K, int B, int M, int d, int nsm) {
    K = Krylov();
    K.B = B;
    K.M = M;
    K.d = d;
    K.nsm = nsm;
    // partial-sum rows: enough for a one-wave launch of any kernel (<= 8
    // resident 256-thread blocks per SM) spread over the B columns
    K.nblk = std::max(1, std::min((d + kThreads - 1) / kThreads, (nsm * 8 + B - 1) / B));
    const size_t nv = (size_t)B * (M + 1) * (size_t)d;
    KG_CUDA(cudaMalloc(&K.V, sizeof(double2) * nv));
    KG_CUDA(cudaMalloc(&K.W, sizeof(double2) * (size_t)B * d));
    KG_CUDA(cudaMalloc(&K.cs, sizeof(ColScalars) * B));
    KG_CUDA(cudaMalloc(&K.part, sizeof(double) * (size_t)B * K.nblk * kPart));
    KG_CUDA(cudaMalloc(&K.cnt, sizeof(unsigned) * B));
    KG_CUDA(cudaMalloc(&K.Q, sizeof(double) * (size_t)B * M * M));
    KG_CUDA(cudaMemset(K.cs, 0, sizeof(ColScalars) * B));
    KG_CUDA(cudaMemset(K.cnt, 0, sizeof(unsigned) * B));
    return KG_OK;
}

int wave_blocks(const Krylov& K, const void* kern, size_t smem) {
    static std::mutex mu;
    static std::map<const void*, int> occ;
    int bps = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = occ.find(kern);
        if (it == occ.end()) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kThreads, smem) != cudaSuccess || bps < 1)
                bps = 1;
            occ[kern] = bps;
        } else {
            bps = it->second;
        }
    }
    const int per = std::max(1, (K.nsm * bps) / K.B);
    return std::max(1, std::min(per, K.nblk));
}

void krylov_free(Krylov& K) {
    cudaFree(K.V);
    cudaFree(K.W);
    cudaFree(K.cs);
    cudaFree(K.part);
    cudaFree(K.cnt);
    cudaFree(K.Q);
    K = Krylov();
}

// ------------------------------------------------- start-of-step norm
// beta0 = ||V_0||, s_0, the largest exponent of V_0, m_eff = M.
__global__ void __launch_bounds__(kThreads) k_colnorm(double2* V, size_t colV, int d, ColScalars* cs, int M,
                                                      double* part, unsigned* cnt, int pstride) {
    __shared__ double sm[(kThreads / 32) * 2];
    __shared__ int smi[kThreads / 32];
    __shared__ double bs[2], red[2];
    const int b = blockIdx.y;
    const double2* x = V + (size_t)b * colV;
    double acc[1] = {0.0};
    int em = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        const double2 v = x[i];
        acc[0] = fma(v.x, v.x, fma(v.y, v.y, acc[0]));
        em = max(em, max(exp_field(v.x), exp_field(v.y)));
    }
    em = block_max_int(em, smi);
    block_sum<1>(acc, 1, sm, bs);
    if (threadIdx.x == 0) bs[1] = (double)em;
    __syncthreads();
    if (grid_finish(bs, 1, part + (size_t)b * pstride, cnt + b, 0, red, 1) && threadIdx.x == 0) {
        ColScalars* C = cs + b;
        const double n = sqrt(red[0]);
        C->beta0 = n;
        C->beta[0] = 0.0;
        C->scale[0] = n > 0.0 ? 1.0 / n : 0.0;
        C->emax[0] = (int)red[1];
        C->m_eff = n > 0.0 ? M : 0;
        C->status = isfinite(n) ? KG_OK : KG_ENUMERIC;
        if (!isfinite(n)) C->m_eff = 0;
    }
}

int launch_colnorm(Krylov& K, cudaStream_t st) {
    ProfScope ps("colnorm", st);
    k_colnorm<<<dim3(wave_blocks(K, (const void*)k_colnorm), K.B), kThreads, 0, st>>>(
        K.V, K.colV(), K.d, K.cs, K.M, K.part, K.cnt, K.nblk * kPart);
    KG_LAUNCHED();
    return KG_OK;
}

// ---------------------------------------- a3: Gram-Schmidt coefficients
// First pass:  u = W - a_j v_j,  h_k = <v_k, u>   for k in [k0, k0+nk)
// Second pass: u = V_{j+1},      h_k = <v_k, u>
// NK (compile time) bounds nk so that the accumulators stay in registers
// without holding 64 of them when only a few vectors are needed.
template <int NK>
__global__ void __launch_bounds__(kThreads) k_reorth_dots(double2* V, size_t colV, const double2* W, int d,
                                                          ColScalars* cs, int j, int k0, int nk, int second,
                                                          double* part, unsigned* cnt, int pstride) {
    __shared__ double sm[(kThreads / 32) * 2 * NK];
    __shared__ double bs[2 * NK], red[2 * NK];
    const int b = blockIdx.y;
    ColScalars* C = cs + b;
    if (j >= C->m_eff) return;
    const double2* Vb = V + (size_t)b * colV;
    const double2* w = second ? Vb + (size_t)(j + 1) * d : W + (size_t)b * d;
    const double2* vj = Vb + (size_t)j * d;
    const double aj = second ? 0.0 : C->alpha[j] * C->scale[j];
    double acc[2 * NK];
#pragma unroll
    for (int k = 0; k < 2 * NK; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        double2 u = w[i];
        if (!second) {
            const double2 p = vj[i];
            u.x = fma(-aj, p.x, u.x);
            u.y = fma(-aj, p.y, u.y);
        }
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            if (k < nk) {
                const double2 v = Vb[(size_t)(k0 + k) * d + i];
                acc[2 * k] = fma(v.x, u.x, fma(v.y, u.y, acc[2 * k]));
                acc[2 * k + 1] = fma(v.x, u.y, fma(-v.y, u.x, acc[2 * k + 1]));
            }
        }
    }
    block_sum<2 * NK>(acc, 2 * nk, sm, bs);
    if (grid_finish(bs, 2 * nk, part + (size_t)b * pstride, cnt + b, 0, red)) {
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            const double s = C->scale[k0 + k];
            C->h[k0 + k] = make_double2(s * red[2 * k], s * red[2 * k + 1]);
        }
    }
}

int launch_reorth_dots(Krylov& K, int j, int k0, int nk, bool second, cudaStream_t st) {
    ProfScope ps("reorth_dots", st);
    const int sec = second ? 1 : 0;
    const int pst = K.nblk * kPart;
#define KG_DOTS(NK) k_reorth_dots<NK><<<dim3(wave_blocks(K, (const void*)k_reorth_dots<NK>), K.B), kThreads, 0, st>>>( \
        K.V, K.colV(), K.W, K.d, K.cs, j, k0, nk, sec, K.part, K.cnt, pst)
    if (nk <= 4) KG_DOTS(4);
    else if (nk <= 8) KG_DOTS(8);
    else if (nk <= 16) KG_DOTS(16);
    else if (nk <= 24) KG_DOTS(24);
    else KG_DOTS(32);
#undef KG_DOTS
    KG_LAUNCHED();
    return KG_OK;
}

// ------------------------------------------------------ a3: the update
// First pass:  V_{j+1} = W - a_j v_j - [reorth] sum_{k<=j} h_k v_k
// Second pass: V_{j+1} -= sum_{k<=j} h_k v_k
// then b_{j+1} = ||V_{j+1}||, s_{j+1} = 1/b_{j+1}, a_j += Re h_j, and the
// breakdown test (the Krylov space is invariant when b_{j+1} is at rounding
// level relative to |a_j| + b_j).
//
// After the three-term subtraction the Gram-Schmidt coefficients are at
// rounding level (|h_k| ~ 1e-14 for unit vectors).  A term whose coefficient
// is below kSmallCoef is accumulated in FP32 (FP32 FMA on the truncated
// vector): its error, < 2^-23 |h_k| |v_k[i]| < 1.2e-17 |v_k[i]|, is far
// below the FP64 rounding of the result, and the FP32 pipe is 64 times wider
// than the FP64 pipe on this GPU.  Larger coefficients use FP64.
constexpr double kSmallCoef = 1e-10;

__global__ void __launch_bounds__(kThreads) k_update(double2* V, size_t colV, const double2* W, int d,
                                                     ColScalars* cs, int j, int reorth, int second,
                                                     double* part, unsigned* cnt, int pstride) {
    __shared__ double2 coef[kMaxMgs + 1];
    __shared__ float2 coef32[kMaxMgs + 1];
    __shared__ int small[kMaxMgs + 1];
    __shared__ double sm[(kThreads / 32) * 2];
    __shared__ int smi[kThreads / 32];
    __shared__ double bs[2], red[2];
    const int b = blockIdx.y;
    ColScalars* C = cs + b;
    if (j >= C->m_eff) return;
    double2* Vb = V + (size_t)b * colV;
    const int nk = reorth ? j + 1 : 0;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        const double s = C->scale[k];
        const double2 h = C->h[k];
        const double2 c = make_double2(s * h.x, s * h.y);
        coef[k] = c;
        coef32[k] = make_float2((float)c.x, (float)c.y);
        // |c| relative to the unit vector v_k = s_k V_k
        small[k] = (fabs(h.x) + fabs(h.y)) < kSmallCoef;
    }
    __syncthreads();
    const double aj = C->alpha[j] * C->scale[j];
    const double2* w = second ? Vb + (size_t)(j + 1) * d : W + (size_t)b * d;
    const double2* vj = Vb + (size_t)j * d;
    double2* out = Vb + (size_t)(j + 1) * d;
    double acc[1] = {0.0};
    int em = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        double2 u = w[i];
        if (!second) {
            const double2 p = vj[i];
            u.x = fma(-aj, p.x, u.x);
            u.y = fma(-aj, p.y, u.y);
        }
        float cx = 0.f, cy = 0.f;
        for (int k = 0; k < nk; ++k) {
            const double2 v = Vb[(size_t)k * d + i];
            if (small[k]) {
                const float2 c = coef32[k];
                const float vx = f64_to_f32_trunc(v.x), vy = f64_to_f32_trunc(v.y);
                cx = fmaf(c.x, vx, fmaf(-c.y, vy, cx));
                cy = fmaf(c.x, vy, fmaf(c.y, vx, cy));
            } else {
                const double2 c = coef[k];
                u.x -= fma(c.x, v.x, -c.y * v.y);
                u.y -= fma(c.x, v.y, c.y * v.x);
            }
        }
        u.x -= (double)cx;
        u.y -= (double)cy;
        out[i] = u;
        acc[0] = fma(u.x, u.x, fma(u.y, u.y, acc[0]));
        em = max(em, max(exp_field(u.x), exp_field(u.y)));
    }
    em = block_max_int(em, smi);
    block_sum<1>(acc, 1, sm, bs);
    if (threadIdx.x == 0) bs[1] = (double)em;
    __syncthreads();
    if (grid_finish(bs, 1, part + (size_t)b * pstride, cnt + b, 0, red, 1) && threadIdx.x == 0) {
        C->emax[j + 1] = (int)red[1];
        const double n = sqrt(red[0]);
        double a = C->alpha[j];
        if (reorth) a += C->h[j].x;
        C->alpha[j] = a;
        C->beta[j + 1] = n;
        C->scale[j + 1] = n > 0.0 ? 1.0 / n : 0.0;
        const double ref = fabs(a) + C->beta[j];
        if (!isfinite(n) || !isfinite(a)) {
            C->status = KG_ENUMERIC;
            C->m_eff = j + 1;
        } else if (n <= 1e-12 * fmax(ref, 1e-300)) {
            C->m_eff = j + 1;  // happy breakdown: K_{j+1} is invariant
        }
    }
}

int launch_update(Krylov& K, int j, int reorth, bool second, cudaStream_t st) {
    ProfScope ps("update", st);
    k_update<<<dim3(wave_blocks(K, (const void*)k_update), K.B), kThreads, 0, st>>>(
        K.V, K.colV(), K.W, K.d, K.cs, j, reorth ? 1 : 0, second ? 1 : 0, K.part, K.cnt, K.nblk * kPart);
    KG_LAUNCHED();
    return KG_OK;
}

// ------------------------------------------- a4: tridiagonal eigenproblem
// One warp per column.  Implicit symmetric QR with Wilkinson shifts on the
// unreduced blocks of T (Golub and Van Loan, Section 8.3): lane 0 chases the
// bulge and records the Givens rotations of one sweep in shared memory, then
// all lanes apply them to their rows of Q (Q <- Q R_k).  On exit T = Q D Q^T.
//   mode 0 (propagation, Eq. (udelta)):
//       c_k = beta0 * sum_m Q[k][m] e^{-i lambda_m tau} Q[0][m]
//   mode 1 (ground state, Eq. (eigen)): c_k = Q[k][m0] for the lowest m0,
//       lam0, lam1 = two lowest Ritz values, resest = |b_m Q[m-1][m0]|.
// The stored combination coefficient is c_k * s_k (Lanczos vectors are
// unnormalised).
constexpr int kTriWarps = 4;

__global__ void __launch_bounds__(32 * kTriWarps) k_tridiag(ColScalars* cs, int B, int Mcap, double* Qall, int mode,
                                                           double tau) {
    __shared__ double sd[kTriWarps][kMaxMgs], se[kTriWarps][kMaxMgs];
    __shared__ double rc[kTriWarps][kMaxMgs], rs[kTriWarps][kMaxMgs];
    __shared__ int ctl[kTriWarps][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * kTriWarps + warp;
    if (b >= B) return;
    ColScalars* C = cs + b;
    const int m = C->m_eff;
    double* Q = Qall + (size_t)b * Mcap * Mcap;
    double* d = sd[warp];
    double* e = se[warp];
    if (m == 0) {
        for (int k = lane; k < Mcap; k += 32) C->c[k] = make_double2(0.0, 0.0);
        if (lane == 0) {
            C->lam0 = C->lam1 = 0.0;
            C->resest = 0.0;
        }
        return;
    }
    for (int k = lane; k < m; k += 32) {
        d[k] = C->alpha[k];
        e[k] = (k + 1 < m) ? C->beta[k + 1] : 0.0;
    }
    for (int r = lane; r < m; r += 32)
        for (int c = 0; c < m; ++c) Q[r * m + c] = (r == c) ? 1.0 : 0.0;
    __syncwarp();
    const double eps = 2.220446049250313e-16;
    int iter = 0;
    const int max_iter = 60 * m + 60;
    while (true) {
        if (lane == 0) {
            // deflate negligible off-diagonals, then locate the last unreduced block
            for (int i = 0; i + 1 < m; ++i)
                if (fabs(e[i]) <= eps * (fabs(d[i]) + fabs(d[i + 1]))) e[i] = 0.0;
            int hi = m - 1;
            while (hi > 0 && e[hi - 1] == 0.0) --hi;
            int lo = hi;
            while (lo > 0 && e[lo - 1] != 0.0) --lo;
            ctl[warp][0] = lo;
            ctl[warp][1] = hi;
            if (hi > 0 && iter < max_iter) {
                // Wilkinson shift from the trailing 2x2 of the block
                const double dd = 0.5 * (d[hi - 1] - d[hi]);
                const double bb = e[hi - 1];
                const double den = dd + copysign(hypot(dd, bb), dd == 0.0 ? 1.0 : dd);
                const double mu = d[hi] - bb * bb / den;
                double x = d[lo] - mu, z = e[lo];
                for (int k = lo; k < hi; ++k) {
                    const double r = hypot(x, z);
                    double c = 1.0, s = 0.0;
                    if (r > 0.0) {
                        c = x / r;
                        s = z / r;
                    }
                    if (k > lo) e[k - 1] = r;
                    const double ak = d[k], ak1 = d[k + 1], bk = e[k];
                    const double cc = c * c, ss = s * s, cs2 = 2.0 * c * s * bk;
                    d[k] = cc * ak + cs2 + ss * ak1;
                    d[k + 1] = ss * ak - cs2 + cc * ak1;
                    e[k] = c * s * (ak1 - ak) + (cc - ss) * bk;
                    if (k + 1 < hi) {
                        const double bulge = s * e[k + 1];
                        e[k + 1] *= c;
                        x = e[k];
                        z = bulge;
                    }
                    rc[warp][k] = c;
                    rs[warp][k] = s;
                }
            }
        }
        __syncwarp();
        const int lo = ctl[warp][0], hi = ctl[warp][1];
        if (hi == 0 || iter >= max_iter) break;
        for (int r = lane; r < m; r += 32) {
            double* row = Q + (size_t)r * m;
            double q0 = row[lo];
            for (int k = lo; k < hi; ++k) {
                const double c = rc[warp][k], s = rs[warp][k];
                const double q1 = row[k + 1];
                row[k] = c * q0 + s * q1;
                q0 = -s * q0 + c * q1;
            }
            row[hi] = q0;
        }
        __syncwarp();
        ++iter;
    }
    if (lane == 0 && iter >= max_iter) C->status = KG_ENOCONV;
    __syncwarp();
    if (mode == 0) {
        const double beta0 = C->beta0;
        double* pc = rc[warp];  // rotation buffers are free now: phases of e^{-i lambda tau}
        double* ps = rs[warp];
        for (int mm = lane; mm < m; mm += 32) {
            double sn, cn;
            sincos(d[mm] * tau, &sn, &cn);
            pc[mm] = cn * Q[mm];  // Q[0][mm] is Q[mm]
            ps[mm] = sn * Q[mm];
        }
        __syncwarp();
        for (int k = lane; k < m; k += 32) {
            double re = 0.0, im = 0.0;
            for (int mm = 0; mm < m; ++mm) {
                const double q = Q[(size_t)k * m + mm];
                re = fma(q, pc[mm], re);
                im = fma(-q, ps[mm], im);
            }
            const double s = beta0 * C->scale[k];
            C->c[k] = make_double2(s * re, s * im);
        }
    } else {
        int m0 = 0, m1 = -1;
        for (int i = 1; i < m; ++i)
            if (d[i] < d[m0]) m0 = i;
        for (int i = 0; i < m; ++i)
            if (i != m0 && (m1 < 0 || d[i] < d[m1])) m1 = i;
        for (int k = lane; k < m; k += 32) C->c[k] = make_double2(Q[(size_t)k * m + m0] * C->scale[k], 0.0);
        if (lane == 0) {
            C->lam0 = d[m0];
            C->lam1 = m1 >= 0 ? d[m1] : INFINITY;
            C->resest = fabs(C->beta[m] * Q[(size_t)(m - 1) * m + m0]);
        }
    }
}

int launch_tridiag(Krylov& K, int mode, double tau, cudaStream_t st) {
    const int nb = (K.B + kTriWarps - 1) / kTriWarps;
    ProfScope ps("tridiag", st);
    k_tridiag<<<nb, 32 * kTriWarps, 0, st>>>(K.cs, K.B, K.M, K.Q, mode, tau);
    KG_LAUNCHED();
    return KG_OK;
}

// ----------------------------------- a5 + a7: combination and overlaps
// out_b = sum_{k<m} c_k V_k  (Eq. (udelta) in the form V x small vector),
// then ||out_b|| and <ov_a, out_b> for the n_ov overlap vectors, written to
// row cs[b].ov_slot of ov_out (the slot advances by one).  NOV bounds n_ov at
// compile time so that the accumulators stay in registers.
template <int NOV>
__global__ void __launch_bounds__(kThreads) k_combine(const double2* V, size_t colV, int d, ColScalars* cs,
                                                      double2* out, size_t out_stride, const double2* ov,
                                                      int n_ov, size_t ov_stride, double2* ov_out, int ov_rows,
                                                      double* part, unsigned* cnt, int pstride) {
    __shared__ double2 coef[kMaxMgs];
    __shared__ double sm[(kThreads / 32) * (2 * NOV + 2)];
    __shared__ double bs[2 * NOV + 2], red[2 * NOV + 2];
    const int b = blockIdx.y;
    ColScalars* C = cs + b;
    const int m = C->m_eff;
    for (int k = threadIdx.x; k < m; k += blockDim.x) coef[k] = C->c[k];
    __syncthreads();
    const double2* Vb = V + (size_t)b * colV;
    double2* o = out + (size_t)b * out_stride;
    double acc[2 * NOV + 2];
#pragma unroll
    for (int k = 0; k < 2 * NOV + 2; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        double2 u = make_double2(0.0, 0.0);
        for (int k = 0; k < m; ++k) {
            const double2 v = Vb[(size_t)k * d + i];
            const double2 c = coef[k];
            u.x = fma(c.x, v.x, fma(-c.y, v.y, u.x));
            u.y = fma(c.x, v.y, fma(c.y, v.x, u.y));
        }
        o[i] = u;
        acc[0] = fma(u.x, u.x, fma(u.y, u.y, acc[0]));
#pragma unroll
        for (int a = 0; a < NOV; ++a) {
            if (a < n_ov) {
                const double2 v = ov[(size_t)a * ov_stride + i];
                acc[2 + 2 * a] = fma(v.x, u.x, fma(v.y, u.y, acc[2 + 2 * a]));
                acc[3 + 2 * a] = fma(v.x, u.y, fma(-v.y, u.x, acc[3 + 2 * a]));
            }
        }
    }
    const int nv = 2 + 2 * n_ov;
    block_sum<2 * NOV + 2>(acc, nv, sm, bs);
    if (grid_finish(bs, nv, part + (size_t)b * pstride, cnt + b, 0, red)) {
        const int slot = C->ov_slot;
        for (int a = threadIdx.x; a < n_ov; a += blockDim.x)
            if (slot < ov_rows) ov_out[((size_t)b * ov_rows + slot) * n_ov + a] = make_double2(red[2 + 2 * a], red[3 + 2 * a]);
        __syncthreads();
        if (threadIdx.x == 0) {
            C->ovnorm = sqrt(red[0]);
            if (n_ov > 0) C->ov_slot = slot + 1;
        }
    }
}

int launch_combine(Krylov& K, double2* out, size_t out_stride, const double2* ov, int n_ov, size_t ov_stride,
                   double2* ov_out, int ov_rows, bool, cudaStream_t st) {
    if (n_ov > kMaxOv) {
        set_error("at most %d overlap vectors per combination pass", kMaxOv);
        return KG_EINVAL;
    }
    ProfScope ps("combine", st);
    const int pst = K.nblk * kPart;
#define KG_COMB(NOV) k_combine<NOV><<<dim3(wave_blocks(K, (const void*)k_combine<NOV>), K.B), kThreads, 0, st>>>( \
        K.V, K.colV(), K.d, K.cs, out, out_stride, ov, n_ov, ov_stride, ov_out, ov_rows, K.part, K.cnt, pst)
    if (n_ov == 0) KG_COMB(0);
    else if (n_ov <= 4) KG_COMB(4);
    else if (n_ov <= 12) KG_COMB(12);
    else KG_COMB(32);
#undef KG_COMB
    KG_LAUNCHED();
    return KG_OK;
}

// Overlaps <ov_a, x_b> of arbitrary vectors into row cs[b].ov_slot (a7).
__global__ void __launch_bounds__(kThreads) k_overlaps(const double2* x, size_t x_stride, int d, ColScalars* cs,
                                                       const double2* ov, int n_ov, size_t ov_stride,
                                                       double2* ov_out, int ov_rows, double* part, unsigned* cnt,
                                                       int pstride) {
    __shared__ double sm[(kThreads / 32) * 2 * kMaxOv];
    __shared__ double bs[2 * kMaxOv], red[2 * kMaxOv];
    const int b = blockIdx.y;
    const double2* xb = x + (size_t)b * x_stride;
    double acc[2 * kMaxOv];
#pragma unroll
    for (int k = 0; k < 2 * kMaxOv; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        const double2 u = xb[i];
#pragma unroll
        for (int a = 0; a < kMaxOv; ++a) {
            if (a < n_ov) {
                const double2 v = ov[(size_t)a * ov_stride + i];
                acc[2 * a] = fma(v.x, u.x, fma(v.y, u.y, acc[2 * a]));
                acc[2 * a + 1] = fma(v.x, u.y, fma(-v.y, u.x, acc[2 * a + 1]));
            }
        }
    }
    block_sum<2 * kMaxOv>(acc, 2 * n_ov, sm, bs);
    if (grid_finish(bs, 2 * n_ov, part + (size_t)b * pstride, cnt + b, 0, red)) {
        ColScalars* C = cs + b;
        const int slot = C->ov_slot;
        for (int a = threadIdx.x; a < n_ov; a += blockDim.x)
            if (slot < ov_rows) ov_out[((size_t)b * ov_rows + slot) * n_ov + a] = make_double2(red[2 * a], red[2 * a + 1]);
        __syncthreads();
        if (threadIdx.x == 0) C->ov_slot = slot + 1;
    }
}

int launch_overlaps_cs(Krylov& K, const double2* x, size_t x_stride, const double2* ov, int n_ov, size_t ov_stride,
                       double2* ov_out, int ov_rows, cudaStream_t st) {
    if (n_ov > kMaxOv || n_ov < 1) {
        set_error("1..%d overlap vectors per pass", kMaxOv);
        return KG_EINVAL;
    }
    ProfScope ps("overlaps", st);
    k_overlaps<<<dim3(wave_blocks(K, (const void*)k_overlaps), K.B), kThreads, 0, st>>>(
        x, x_stride, K.d, K.cs, ov, n_ov, ov_stride, ov_out, ov_rows, K.part, K.cnt, K.nblk * kPart);
    KG_LAUNCHED();
    return KG_OK;
}

// -------------------------------------------- ground-state residual
// rq = <x, y> (x normalised), then rnorm = ||y - rq x||.
__global__ void __launch_bounds__(kThreads) k_rq(const double2* x, const double2* y, int d, ColScalars* cs,
                                                 int phase, double* part, unsigned* cnt, int nblk) {
    __shared__ double sm[(kThreads / 32) * 2];
    __shared__ double bs[2], red[2];
    const double rq = phase ? cs->rq : 0.0;
    double acc[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        const double2 a = x[i], b = y[i];
        if (phase == 0) {
            acc[0] = fma(a.x, b.x, fma(a.y, b.y, acc[0]));
        } else {
            const double rx = fma(-rq, a.x, b.x), ry = fma(-rq, a.y, b.y);
            acc[0] = fma(rx, rx, fma(ry, ry, acc[0]));
        }
    }
    block_sum<1>(acc, 1, sm, bs);
    if (grid_finish(bs, 1, part, cnt, 0, red) && threadIdx.x == 0) {
        if (phase == 0)
            cs->rq = red[0];
        else
            cs->rnorm = sqrt(red[0]);
    }
}

// -------------------------------------------------- step sequencing
int enqueue_step(const StepPlan& P, cudaStream_t st) {
    Krylov& K = *P.K;
    const SecView S = P.sec->view();
    KG_TRY(launch_colnorm(K, st));
    for (int j = 0; j < K.M; ++j) {
        KG_TRY(launch_lanczos_hpsi(S, K, j, P.int_hops != 0, st));
        if (P.reorth >= 1)
            for (int k0 = 0; k0 <= j; k0 += kChunk)
                KG_TRY(launch_reorth_dots(K, j, k0, std::min(kChunk, j + 1 - k0), false, st));
        KG_TRY(launch_update(K, j, P.reorth >= 1, false, st));
        if (P.reorth >= 2) {
            for (int k0 = 0; k0 <= j; k0 += kChunk)
                KG_TRY(launch_reorth_dots(K, j, k0, std::min(kChunk, j + 1 - k0), true, st));
            KG_TRY(launch_update(K, j, 1, true, st));
        }
    }
    KG_TRY(launch_tridiag(K, 0, P.tau, st));
    KG_TRY(launch_combine(K, K.V, K.colV(), P.ov, P.n_ov, P.ov_stride, P.ov_out, P.ov_rows, true, st));
    return KG_OK;
}

// ------------------------------------------------------ ground state
int ground_state(kg_sector* s, const kg_opts* o) {
    cudaStream_t st = pick_stream(s, o);
    const int d = (int)s->d;
    const int M = std::max(1, std::min(o->M_gs, d));
    if (o->M_gs < 2 || o->M_gs > kMaxMgs) {
        set_error("M_gs must be in [2, %d]", kMaxMgs);
        return KG_EINVAL;
    }
    if (!s->gs) KG_CUDA(cudaMalloc(&s->gs, sizeof(double2) * d));
    Krylov K;
    int rc = krylov_alloc(K, 1, M, d, s->nsm);
    if (rc != KG_OK) {
        krylov_free(K);
        return rc;
    }
    auto done = [&](int r) {
        krylov_free(K);
        return r;
    };
    const SecView S = s->view();
    rc = launch_random_start(K.V, d, o->seed, st);
    ColScalars h;
    bool converged = false;
    for (int r = 0; rc == KG_OK && r < o->max_restarts; ++r) {
        if ((rc = launch_colnorm(K, st)) != KG_OK) break;
        for (int j = 0; j < M && rc == KG_OK; ++j) {
            rc = launch_lanczos_hpsi(S, K, j, o->schedule != 1, st);
            for (int k0 = 0; rc == KG_OK && k0 <= j; k0 += kChunk)
                rc = launch_reorth_dots(K, j, k0, std::min(kChunk, j + 1 - k0), false, st);
            if (rc == KG_OK) rc = launch_update(K, j, 1, false, st);
            if (rc == KG_OK && o->reorth >= 2) {
                for (int k0 = 0; rc == KG_OK && k0 <= j; k0 += kChunk)
                    rc = launch_reorth_dots(K, j, k0, std::min(kChunk, j + 1 - k0), true, st);
                if (rc == KG_OK) rc = launch_update(K, j, 1, true, st);
            }
        }
        if (rc == KG_OK) rc = launch_tridiag(K, 1, 0.0, st);
        if (rc == KG_OK) rc = launch_combine(K, s->gs, 0, nullptr, 0, 0, nullptr, 0, false, st);
        if (rc != KG_OK) break;
        if (cudaMemcpyAsync(&h, K.cs, sizeof(ColScalars), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "ground-state readback", __FILE__, __LINE__);
            break;
        }
        if (h.status == KG_ENUMERIC || !(h.ovnorm > 0.0) || !std::isfinite(h.ovnorm)) {
            set_error("non-finite value in the ground-state Lanczos recursion");
            rc = KG_ENUMERIC;
            break;
        }
        if ((rc = launch_scale_copy(s->gs, s->gs, d, 1.0 / h.ovnorm, st)) != KG_OK) break;
        if ((rc = launch_hpsi(S, s->gs, K.W, st)) != KG_OK) break;
        k_rq<<<K.nblk, kThreads, 0, st>>>(s->gs, K.W, d, K.cs, 0, K.part, K.cnt, K.nblk);
        count_launch();
        k_rq<<<K.nblk, kThreads, 0, st>>>(s->gs, K.W, d, K.cs, 1, K.part, K.cnt, K.nblk);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) {
            rc = KG_ECUDA;
            break;
        }
        if (cudaMemcpyAsync(&h, K.cs, sizeof(ColScalars), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "ground-state readback", __FILE__, __LINE__);
            break;
        }
        s->E0 = h.rq;
        s->resid = h.rnorm;
        s->gap = h.lam1 - h.lam0;
        if (!std::isfinite(h.rq) || !std::isfinite(h.rnorm)) {
            set_error("non-finite Rayleigh quotient");
            rc = KG_ENUMERIC;
            break;
        }
        if (h.rnorm <= o->tol_resid * std::max(1.0, std::fabs(h.rq)) || M >= d) {
            converged = true;
            break;
        }
        // restart from the Ritz vector
        if (cudaMemcpyAsync(K.V, s->gs, sizeof(double2) * d, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            rc = KG_ECUDA;
            break;
        }
    }
    if (rc != KG_OK) return done(rc);
    s->has_gs = converged;
    if (!converged) {
        set_error("ground state not converged: residual %.3e after %d restarts", s->resid, o->max_restarts);
        return done(KG_ENOCONV);
    }
    if (s->gap < 1e-8 * std::max(1.0, std::fabs(s->E0))) {
        set_error("ground state looks degenerate: Ritz gap %.3e", s->gap);
        return done(KG_EDEGEN);
    }
    return done(KG_OK);
}

}  // namespace kg
