// kg_krylov.cu -- the Lanczos recursion with full
// reorthogonalisation, the small tridiagonal eigenproblem and exponential,
// and the basis combination (Section 2, Eqs. (recursion), (tmatrix),
// (tdiag), (eigen); Section 3, Eqs. (newstate) and (udelta)).
//
// Every kernel works on a batch of B independent columns, possibly of
// different sectors and dimensions (many instances, or many columns of one
// Green's-function calculation).  A launch walks a work list of (column,
// block, blocks-of-that-column) items, so one launch per phase serves the
// whole batch.  Lanczos vectors are stored unnormalised, V_k, with v_k = s_k
// V_k and s_k = 1/||V_k|| kept on the device, so normalisation never costs a
// separate pass.  Scalars (a_k, b_k, Gram-Schmidt and combination
// coefficients) never leave the device: a whole propagation step is a fixed
// launch sequence that a CUDA graph can replay.
#include <algorithm>
#include <array>
#include <utility>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "kg_internal.h"

namespace kg {

// ------------------------------------------------------------ workspace
size_t krylov_bytes(const std::vector<const kg_sector*>& cols, int M, bool planes, int schedule) {
    size_t nv = 0, nw = 0;
    for (auto* s : cols) {
        nv += (size_t)(M + 1) * (size_t)s->d;
        nw += (size_t)s->d;
    }
    // basis, W and U, fixed-point image; partial sums (at most 16 blocks per
    // SM of 72 doubles per column), work lists and descriptors
    size_t b = nv * sizeof(double2) + 3 * nw * sizeof(double2) + (cols.size() + 2) * (size_t(2) << 20);
    if (planes) b += nv * (sizeof(double) + sizeof(float2) + ((schedule & 4) ? 0 : sizeof(int4)));
    return b;
}

int krylov_alloc(Krylov& K, const std::vector<const kg_sector*>& cols, int M, int nsm, int schedule, bool planes) {
    K = Krylov();
    K.schedule = schedule;
    const bool int_hops = !(schedule & 1);
    K.B = (int)cols.size();
    K.M = M;
    K.nsm = nsm;
    if (K.B < 1) {
        set_error("empty Krylov batch");
        return KG_EINVAL;
    }
    size_t nv = 0, nw = 0, np = 0, nx = 0;
    for (auto* s : cols) K.total_d += s->d;
    K.hdesc.resize(K.B);
    K.hsec.resize(K.B);
    for (int b = 0; b < K.B; ++b) {
        const kg_sector* s = cols[b];
        ColDesc& D = K.hdesc[b];
        std::memset(&D, 0, sizeof D);
        D.d = (int)s->d;
        K.hsec[b] = s->view();
        const SecView& S = K.hsec[b];
        D.mode = S.hopmode == 0 ? ((int_hops && S.fix_pre >= 0) ? 3 : 0) : S.hopmode;
        D.Du = S.Du;
        D.Dd = S.Dd;
        D.fix_pre = S.fix_pre;
        if (D.mode == 3) nx += (size_t)D.d;
        nv += (size_t)(M + 1) * D.d;
        nw += (size_t)D.d;
    }
    // H*psi groups: consecutive columns of one mode while their inputs fit
    // kHpsiGroupBytes; then partial-sum rows for a one-wave list (<= 8 blocks
    // per SM) of any kernel at up to twice the wave, shared in proportion to
    // d over the batch or over the column's group, whichever is larger
    K.group.assign(K.B, 0);
    std::vector<long long> gbytes, gd;
    {
        // balanced: as few groups as the budget allows, filled to the mean
        long long mbytes[4] = {0, 0, 0, 0};
        for (auto& D : K.hdesc) mbytes[D.mode] += 16LL * D.d;
        long long target[4];
        for (int m = 0; m < 4; ++m) {
            const long long ng = std::max(1LL, (mbytes[m] + kHpsiGroupBytes - 1) / kHpsiGroupBytes);
            target[m] = (mbytes[m] + ng - 1) / ng;
        }
        int cur[4] = {-1, -1, -1, -1};
        for (int b = 0; b < K.B; ++b) {
            ColDesc& D = K.hdesc[b];
            const long long bytes = 16LL * D.d;
            if (cur[D.mode] < 0 || gbytes[cur[D.mode]] + bytes > target[D.mode]) {
                cur[D.mode] = (int)gbytes.size();
                gbytes.push_back(0);
                gd.push_back(0);
                K.group[b] = K.ngroups[D.mode]++;
            } else {
                K.group[b] = K.ngroups[D.mode] - 1;
            }
            gbytes[cur[D.mode]] += bytes;
            gd[cur[D.mode]] += D.d;
            D.pad = cur[D.mode];  // global group slot, used below only
        }
    }
    np = 0;
    for (int b = 0; b < K.B; ++b) {
        ColDesc& D = K.hdesc[b];
        const double share = std::max((double)D.d / (double)K.total_d, (double)D.d / (double)gd[D.pad]);
        const long long want = (long long)std::ceil(16.0 * nsm * share) + 2;
        D.nblk_max = (int)std::max(1LL, std::min(want, (long long)(D.d + kThreads - 1) / kThreads));
        D.pad = 0;
        np += (size_t)D.nblk_max * kPart;
    }
    // on any failure the workspace is released whole (krylov_free skips null)
    auto need = [&](cudaError_t e, const char* what) -> int {
        if (e == cudaSuccess) return KG_OK;
        cudaGetLastError();
        krylov_free(K);
        set_error("Krylov workspace: %s failed (%s)", what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? KG_ENOMEM : KG_ECUDA;
    };
    KG_TRY(need(cudaMalloc(&K.Vbuf, sizeof(double2) * nv), "basis allocation"));
    // Planes read by the Gram-Schmidt kernels (Re+Im for the three-multiply
    // dot products, a truncated FP32 copy for the small correction terms).
    // They are optional: without the memory the kernels use V alone.
    if (!planes || cudaMalloc(&K.Sbuf, sizeof(double) * nv) != cudaSuccess ||
        cudaMalloc(&K.V32buf, sizeof(float2) * nv) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(K.Sbuf);
        cudaFree(K.V32buf);
        K.Sbuf = nullptr;
        K.V32buf = nullptr;
    }
    // fixed-point images for the exact integer Gram-Schmidt dots (schedule
    // bit 2 clear), optional like the planes
    if (K.Sbuf && !(schedule & 4) && cudaMalloc(&K.Ibuf, sizeof(int4) * nv) != cudaSuccess) {
        cudaGetLastError();
        K.Ibuf = nullptr;
    }
    KG_TRY(need(cudaMalloc(&K.Wbuf, sizeof(double2) * 2 * nw), "work vector allocation"));
    if (nx) KG_TRY(need(cudaMalloc(&K.Xfbuf, sizeof(longlong2) * nx), "fixed-point image allocation"));
    KG_TRY(need(cudaMalloc(&K.partbuf, sizeof(double) * np), "partial-sum allocation"));
    KG_TRY(need(cudaMalloc(&K.desc, sizeof(ColDesc) * K.B), "descriptor allocation"));
    KG_TRY(need(cudaMalloc(&K.secs, sizeof(SecView) * K.B), "sector view allocation"));
    KG_TRY(need(cudaMalloc(&K.cs, sizeof(ColScalars) * K.B), "scalar allocation"));
    KG_TRY(need(cudaMalloc(&K.cnt, sizeof(unsigned) * K.B), "ticket allocation"));
    KG_TRY(need(cudaMalloc(&K.Q, sizeof(double) * (size_t)K.B * M * M), "eigenvector allocation"));
    KG_TRY(need(cudaMemset(K.cs, 0, sizeof(ColScalars) * K.B), "scalar reset"));
    KG_TRY(need(cudaMemset(K.cnt, 0, sizeof(unsigned) * K.B), "ticket reset"));
    size_t ov = 0, ow = 0, op = 0, ox = 0;
    for (int b = 0; b < K.B; ++b) {
        ColDesc& D = K.hdesc[b];
        D.sec = K.secs + b;
        D.V = K.Vbuf + ov;
        D.S = K.Sbuf ? K.Sbuf + ov : nullptr;
        D.V32 = K.V32buf ? K.V32buf + ov : nullptr;
        D.I = K.Ibuf ? K.Ibuf + ov : nullptr;
        if (D.mode == 3) {
            D.Xf = K.Xfbuf + ox;
            ox += (size_t)D.d;
        }
        D.W = K.Wbuf + ow;
        D.U = K.Wbuf + nw + ow;
        D.part = K.partbuf + op;
        D.out = D.V;
        ov += (size_t)(M + 1) * D.d;
        ow += (size_t)D.d;
        op += (size_t)D.nblk_max * kPart;
    }
    KG_TRY(need(cudaMemcpy(K.secs, K.hsec.data(), sizeof(SecView) * K.B, cudaMemcpyHostToDevice), "upload"));
    KG_TRY(need(cudaMemcpy(K.desc, K.hdesc.data(), sizeof(ColDesc) * K.B, cudaMemcpyHostToDevice), "upload"));
    return KG_OK;
}

int krylov_upload(Krylov& K, cudaStream_t st) {
    KG_CUDA(cudaMemcpyAsync(K.desc, K.hdesc.data(), sizeof(ColDesc) * K.B, cudaMemcpyHostToDevice, st));
    return KG_OK;
}

int krylov_set_diag(Krylov& K, const double* diag) {
    for (auto& S : K.hsec) S.diag = diag;
    KG_CUDA(cudaMemcpy(K.secs, K.hsec.data(), sizeof(SecView) * K.B, cudaMemcpyHostToDevice));
    return KG_OK;
}

void krylov_free(Krylov& K) {
    for (auto& kv : K.lists) cudaFree(kv.second.first);
    cudaFree(K.Vbuf);
    cudaFree(K.Sbuf);
    cudaFree(K.V32buf);
    cudaFree(K.Ibuf);
    cudaFree(K.Xfbuf);
    cudaFree(K.Wbuf);
    cudaFree(K.partbuf);
    cudaFree(K.desc);
    cudaFree(K.secs);
    cudaFree(K.cs);
    cudaFree(K.cnt);
    cudaFree(K.Q);
    K = Krylov();
}

static int occupancy(const void* kern) {
    static std::mutex mu;
    static std::map<const void*, int> occ;
    std::lock_guard<std::mutex> lk(mu);
    auto it = occ.find(kern);
    if (it != occ.end()) return it->second;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kThreads, 0) != cudaSuccess || bps < 1) bps = 1;
    occ[kern] = bps;
    return bps;
}

// Work list of a kernel over the columns whose mode is `mode` (-1: all) and,
// with group >= 0, whose H*psi group is `group`: column b gets blocks in
// proportion to its dimension, one wave in total.
int work_list(Krylov& K, const void* kern, int mode, const int4** items, int* n, int group) {
    const int bps = occupancy(kern);
    const long long key = ((long long)bps << 8) + (mode + 1) + ((long long)std::lround(K.wave_scale * 64.0) << 20) +
                          ((long long)(group + 1) << 32);
    auto it = K.lists.find(key);
    if (it == K.lists.end()) {
        auto take = [&](const ColDesc& D, int b) {
            return (mode < 0 || D.mode == mode) && (group < 0 || K.group[b] == group);
        };
        long long dsel = 0;
        for (int b = 0; b < K.B; ++b)
            if (take(K.hdesc[b], b)) dsel += K.hdesc[b].d;
        const double total = std::max(1.0, K.wave_scale * K.nsm * bps);
        std::vector<int4> v;
        for (int b = 0; b < K.B; ++b) {
            const ColDesc& D = K.hdesc[b];
            if (!take(D, b)) continue;
            int nb = (int)std::lround(total * (double)D.d / (double)std::max(1LL, dsel));
            nb = std::max(1, std::min(nb, std::min(D.nblk_max, (D.d + kThreads - 1) / kThreads)));
            for (int k = 0; k < nb; ++k) v.push_back(make_int4(b, k, nb, 0));
        }
        int4* d = nullptr;
        if (!v.empty()) {
            KG_CUDA(cudaMalloc(&d, sizeof(int4) * v.size()));
            KG_CUDA(cudaMemcpy(d, v.data(), sizeof(int4) * v.size(), cudaMemcpyHostToDevice));
        }
        it = K.lists.emplace(key, std::make_pair(d, (int)v.size())).first;
    }
    *items = it->second.first;
    *n = it->second.second;
    return KG_OK;
}

// ------------------------------------------------- start-of-step norm
// beta0 = ||V_0||, s_0, the largest exponent of V_0, m_eff = M.
__global__ void __launch_bounds__(kThreads) k_colnorm(const ColDesc* desc, const int4* items, ColScalars* cs, int M,
                                                      unsigned* cnt) {
    __shared__ double sm[(kThreads / 32) * 2];
    __shared__ int smi[kThreads / 32];
    __shared__ double bs[2], red[2];
    KG_ITEM();
    const double2* x = D.V;
    double acc[1] = {0.0};
    int em = 0;
    KG_FOR(i) {
        const double2 v = x[i];
        acc[0] = fma(v.x, v.x, fma(v.y, v.y, acc[0]));
        em = max(em, max(exp_field(v.x), exp_field(v.y)));
        if (D.S) {
            D.S[i] = v.x + v.y;
            D.V32[i] = make_float2(f64_to_f32_trunc(v.x), f64_to_f32_trunc(v.y));
        }
    }
    em = block_max_int(em, smi);
    block_sum<1>(acc, 1, sm, bs);
    if (threadIdx.x == 0) bs[1] = (double)em;
    __syncthreads();
    if (grid_finish(bs, 1, D.part, cnt + b, blk, nblk, red, 1) && threadIdx.x == 0) {
        const double n = sqrt(red[0]);
        C->beta0 = n;
        C->beta[0] = 0.0;
        C->scale[0] = n > 0.0 ? 1.0 / n : 0.0;
        C->emax[0] = (int)red[1];
        C->eimg[0] = (int)red[1];  // I_0 is written by the first H*psi on this exponent
        C->m_eff = n > 0.0 ? M : 0;
        // the status is sticky over the steps of one call (reset by
        // launch_reset_status), so a non-finite column stays reported
        if (!isfinite(n)) {
            C->status = KG_ENUMERIC;
            C->m_eff = 0;
        }
    }
}

int launch_colnorm(Krylov& K, cudaStream_t st) {
    ProfScope ps("colnorm", st);
    const int4* items;
    int n;
    KG_TRY(work_list(K, (const void*)k_colnorm, -1, &items, &n));
    k_colnorm<<<n, kThreads, 0, st>>>(K.desc, items, K.cs, K.M, K.cnt);
    KG_LAUNCHED();
    return KG_OK;
}

// ---------------------------------------- Gram-Schmidt coefficients
// First pass:  u = W - a_j v_j,  h_k = <v_k, u>   for k in [k0, k0+NK)
// Second pass: u = V_{j+1},      h_k = <v_k, u>
//
// With the plane S_k = Re V_k + Im V_k present, each complex product takes
// three FP64 multiply-adds instead of four (v = a + ib, u = c + id):
//   T1 = sum a c,  T2 = sum b d,  T3 = sum (a + b)(d - c),
//   Re <v,u> = T1 + T2,  Im <v,u> = T3 + T1 - T2,
// with d - c formed once per element and shared by all k.  The FP64 pipe
// bounds this kernel, so the extra 8 bytes per element of S cost less than
// the multiply-add they save.
//
// The accumulators live in registers.  For more than 12 vectors the two
// halves of the block take the two halves of the k range over the same
// elements (u is read twice, the second time from cache), which keeps the
// kernel at two blocks per SM without spilling.
template <int NK>
__global__ void __launch_bounds__(kThreads, 2) k_reorth_dots(const ColDesc* desc, const int4* items, ColScalars* cs,
                                                             int j, int k0, int nk, int second, unsigned* cnt) {
    constexpr int G = NK > 12 ? 2 : 1;         // thread groups splitting the k range
    constexpr int KH = (NK + G - 1) / G;       // vectors per group
    constexpr int TG = kThreads / G;           // threads per group
    __shared__ double sm[(kThreads / 32) * 3 * KH];
    __shared__ double bs[3 * NK], red[3 * NK];
    KG_ITEM();
    if (j >= C->m_eff) return;
    const int d = D.d;
    const int grp = threadIdx.x / TG, t = threadIdx.x % TG;
    const int kb = grp * KH, kn = min(KH, NK - kb);
    const double2* Vb = D.V + (size_t)(k0 + kb) * d;
    const double2* w = second ? D.V + (size_t)(j + 1) * d : D.W;
    const double2* vj = D.V + (size_t)j * d;
    const double aj = second ? 0.0 : C->alpha[j] * C->scale[j];
    double acc[3 * KH];
#pragma unroll
    for (int k = 0; k < 3 * KH; ++k) acc[k] = 0.0;
    const bool three = D.S != nullptr;
    // the last chunk of a first pass leaves u = W - a_j v_j in U for the update
    const bool keep = !second && k0 + NK == j + 1 && grp == 0;
    double2* wu = D.U;
    if (three) {
        const double* Sb = D.S + (size_t)(k0 + kb) * d;
        for (int i = blk * TG + t; i < d; i += nblk * TG) {
            double2 u = w[i];
            if (!second) {
                const double2 p = vj[i];
                u.x = fma(-aj, p.x, u.x);
                u.y = fma(-aj, p.y, u.y);
                if (keep) wu[i] = u;
            }
            const double dmc = u.y - u.x;
#pragma unroll
            for (int k = 0; k < KH; ++k) {
                if (k < kn) {
                    const size_t o = (size_t)k * d + i;
                    const double2 v = Vb[o];
                    const double sv = Sb[o];
                    acc[3 * k] = fma(v.x, u.x, acc[3 * k]);
                    acc[3 * k + 1] = fma(v.y, u.y, acc[3 * k + 1]);
                    acc[3 * k + 2] = fma(sv, dmc, acc[3 * k + 2]);
                }
            }
        }
    } else {
        for (int i = blk * TG + t; i < d; i += nblk * TG) {
            double2 u = w[i];
            if (!second) {
                const double2 p = vj[i];
                u.x = fma(-aj, p.x, u.x);
                u.y = fma(-aj, p.y, u.y);
            }
            if (keep) wu[i] = u;
#pragma unroll
            for (int k = 0; k < KH; ++k) {
                if (k < kn) {
                    const double2 v = Vb[(size_t)k * d + i];
                    acc[3 * k] = fma(v.x, u.x, fma(v.y, u.y, acc[3 * k]));
                    acc[3 * k + 1] = fma(v.x, u.y, fma(-v.y, u.x, acc[3 * k + 1]));
                }
            }
        }
    }
    // block sums: warps reduce their accumulators, then each group's warps
    // are added in warp order (fixed order, so results are reproducible)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3 * KH; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sm[warp * 3 * KH + k] = v;
    }
    __syncthreads();
    constexpr int WG = TG / 32;  // warps per group
    for (int q = threadIdx.x; q < 3 * NK; q += blockDim.x) {
        const int g = q / (3 * KH), l = q - g * 3 * KH;
        double s = 0.0;
        for (int w2 = 0; w2 < WG; ++w2) s += sm[(g * WG + w2) * 3 * KH + l];
        bs[q] = s;
    }
    __syncthreads();
    if (grid_finish(bs, 3 * NK, D.part, cnt + b, blk, nblk, red)) {
        for (int k = threadIdx.x; k < NK; k += blockDim.x) {
            const double s = C->scale[k0 + k];
            const double t1 = red[3 * k], t2 = red[3 * k + 1], t3 = red[3 * k + 2];
            C->h[k0 + k] = three ? make_double2(s * (t1 + t2), s * (t3 + t1 - t2)) : make_double2(s * t1, s * t2);
        }
    }
}

// Exact-product Gram-Schmidt coefficients (first pass): h_k = s_k <V_k, u>
// with u = W - a_j v_j, from 52-bit fixed-point images.  Each V_k comes as
// its image I_k (written by the kernel that produced V_k, on the exponent
// bound eimg[k]); u is formed in FP64 here and converted on a bound E_u of
// its largest exponent.  With both numbers split into 26-bit halves, every
// partial product (hi*hi, hi*lo, lo*hi, lo*lo) is an exact 64-bit integer
// (one wide integer multiply-add).  The hi*hi and cross products are summed
// exactly in two 64-bit accumulators (units 2^52 and 2^26 of the full
// product); only lo*lo is rounded to the nearest 2^26, an error of 2^-79 of
// the product of the two vectors' largest components per element.  A
// thread's sums are converted to FP64 once per tile and reduced in a fixed
// order.  The FP64 pipe of this GPU issues
// about 2 multiply-adds per clock per SM, the integer pipe far more, so these
// dots are bounded by the 16 bytes of I_k per element and vector instead of
// the 3 FP64 multiply-adds per complex product of the Re+Im form.
//
// Each block takes its elements in tiles of kIntTile: first every thread
// forms kIntTile / kThreads elements of u and their images (shared memory),
// then the G thread groups take the tile's elements for their KH vectors
// each, the loads of an element's KH vectors issued first.
//
// The update writes I_{j+1} on an exponent bounded before V_{j+1} exists.
// Near a breakdown (||V_{j+1}|| far below ||W||) that bound is loose and the
// image keeps too few of V_{j+1}'s own bits; a vector whose bound exceeds
// its true largest exponent by more than kFixSlack bits is therefore
// converted here from V_k on its exact exponent, the fresh image is stored
// back (each block its own elements) and its exponent updated at the end.
constexpr int kIntTile = 1024;

template <int NK>
struct IntDots {
    static constexpr int G = NK <= 3 ? 1 : (NK <= 6 ? 2 : (NK <= 12 ? 4 : 8));  // groups splitting k
    static constexpr int KH = (NK + G - 1) / G;                                  // vectors per group
    static constexpr int TG = kThreads / G;                                      // threads per group
};

// Re and Im of conj(v) u for v and u given as split 52-bit images (v:
// {x_hi, x_lo, y_hi, y_lo}; u: Re hi/lo, Im hi/lo and -Re hi/lo): the
// hi*hi part in units of 2^52 (re2, im2) and the rest in units of 2^26
// (re1, im1) of the full product.
__device__ __forceinline__ void cdot_fix(const int4 v, const int* uw, long long& re2, long long& re1,
                                         long long& im2, long long& im1) {
    const int p1 = uw[0], p0 = uw[1], q1 = uw[2], q0 = uw[3], n1 = uw[4], n0 = uw[5];
    // Re = vx ux + vy uy
    re2 += (long long)v.x * p1 + (long long)v.z * q1;
    re1 += (long long)v.x * p0 + (long long)v.y * p1 + (long long)v.z * q0 + (long long)v.w * q1 +
           (((long long)v.y * p0 + (long long)v.w * q0 + (1ll << 25)) >> 26);
    // Im = vx uy - vy ux
    im2 += (long long)v.x * q1 + (long long)v.z * n1;
    im1 += (long long)v.x * q0 + (long long)v.y * q1 + (long long)v.z * n0 + (long long)v.w * n1 +
           (((long long)v.y * q0 + (long long)v.w * n0 + (1ll << 25)) >> 26);
}

template <int NK>
__global__ void __launch_bounds__(kThreads, 3) k_reorth_dots_int(const ColDesc* desc, const int4* items,
                                                                 ColScalars* cs, int j, int k0, int nk,
                                                                 unsigned* cnt) {
    constexpr int G = IntDots<NK>::G, KH = IntDots<NK>::KH, TG = IntDots<NK>::TG;
    constexpr int R = kIntTile / kThreads;         // elements of u per thread and tile
    __shared__ int up[kIntTile][6];                // image of u: Re hi/lo, Im hi/lo, -Re hi/lo
    __shared__ double sm[(kThreads / 32) * 2 * KH];
    __shared__ double bs[2 * NK], red[2 * NK];
    __shared__ int eu_s;
    __shared__ int fresh_s[NK], ek_s[NK];
    KG_ITEM();
    if (j >= C->m_eff) return;
    const int d = D.d;
    const int grp = threadIdx.x / TG, t = threadIdx.x % TG;
    const int kb = grp * KH, kn = min(KH, NK - kb);
    int4* Ib = D.I + (size_t)(k0 + kb) * d;
    const double2* Vk = D.V + (size_t)(k0 + kb) * d;
    const double2* w = D.W;
    const double2* vj = D.V + (size_t)j * d;
    const double aj = C->alpha[j] * C->scale[j];
    // a_j = 0 here means a_j comes from these dots (u = W, which the update
    // reads itself); otherwise the last chunk leaves u = W - a_j v_j in U
    const bool sub = aj != 0.0;
    const bool keep = sub && k0 + NK == j + 1;
    if (threadIdx.x < NK) {
        ek_s[threadIdx.x] = C->emax[k0 + threadIdx.x];
        fresh_s[threadIdx.x] = C->eimg[k0 + threadIdx.x] - C->emax[k0 + threadIdx.x] > kFixSlack;
    }
    if (threadIdx.x == 0) {
        // |u_i| <= |W_i| + |a_j| |V_j[i]| < (1 + |a_j| 2^(E_j - E_w)) 2^(E_w - 1022), with a margin
        const int Ew = C->ew;
        const double r = (1.0 + fabs(aj) * ldexp(1.0, C->emax[j] - Ew)) * (1.0 + 1.0 / 1024.0);
        int ex;
        const double fr = frexp(r, &ex);
        eu_s = Ew + (fr == 0.5 ? ex - 1 : ex);
    }
    __syncthreads();
    const int Eu = eu_s;
    double acc[2 * KH];
#pragma unroll
    for (int q = 0; q < 2 * KH; ++q) acc[q] = 0.0;
    auto load = [&](int k, int i) -> int4 {
        if (fresh_s[kb + k]) {
            const int4 v = fix_image(Vk[(size_t)k * d + i], ek_s[kb + k]);
            Ib[(size_t)k * d + i] = v;
            return v;
        }
        return Ib[(size_t)k * d + i];
    };
    for (int base = blk * kIntTile; base < d; base += nblk * kIntTile) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = threadIdx.x + r * kThreads, i = base + e;
            if (i < d) {
                double2 u = w[i];
                if (sub) {
                    const double2 p = vj[i];
                    u.x = fma(-aj, p.x, u.x);
                    u.y = fma(-aj, p.y, u.y);
                }
                if (keep) D.U[i] = u;
                const long long px = fix52(u.x, Eu), py = fix52(u.y, Eu);
                up[e][0] = fix_hi(px);
                up[e][1] = fix_lo(px);
                up[e][2] = fix_hi(py);
                up[e][3] = fix_lo(py);
                up[e][4] = fix_hi(-px);
                up[e][5] = fix_lo(-px);
            }
        }
        __syncthreads();
        const int end = min(kIntTile, d - base);
        long long re2[KH], re1[KH], im2[KH], im1[KH];
#pragma unroll
        for (int k = 0; k < KH; ++k) re2[k] = re1[k] = im2[k] = im1[k] = 0;
        // a thread takes kIntTile / TG <= 32 elements of the tile, each adding
        // at most 2^54.1 to an accumulator: the sums stay below 2^60
        for (int e = t; e < end; e += TG) {
            int4 va[KH];
#pragma unroll
            for (int k = 0; k < KH; ++k)
                if (k < kn) va[k] = load(k, base + e);
#pragma unroll
            for (int k = 0; k < KH; ++k)
                if (k < kn) cdot_fix(va[k], up[e], re2[k], re1[k], im2[k], im1[k]);
        }
#pragma unroll
        for (int k = 0; k < KH; ++k) {
            acc[2 * k] += fma((double)re1[k], 0x1p-26, (double)re2[k]);
            acc[2 * k + 1] += fma((double)im1[k], 0x1p-26, (double)im2[k]);
        }
        __syncthreads();
    }
    // block sums: warps reduce, then each group's warps in warp order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 2 * KH; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) sm[warp * 2 * KH + q] = v;
    }
    __syncthreads();
    constexpr int WG = TG / 32;  // warps per group
    for (int q = threadIdx.x; q < 2 * NK; q += blockDim.x) {
        const int g = q / (2 * KH), l = q - g * 2 * KH;
        double sum = 0.0;
        for (int w2 = 0; w2 < WG; ++w2) sum += sm[(g * WG + w2) * 2 * KH + l];
        bs[q] = sum;
    }
    __syncthreads();
    if (grid_finish(bs, 2 * NK, D.part, cnt + b, blk, nblk, red)) {
        for (int k = threadIdx.x; k < NK; k += blockDim.x) {
            // units: 2^52 of 2^(E_k - 1074) 2^(E_u - 1074), E_k the exponent of V_k's image
            const int Ei = fresh_s[k] ? C->emax[k0 + k] : C->eimg[k0 + k];
            const double f = C->scale[k0 + k] * ldexp(1.0, Ei + Eu - 2096);
            C->h[k0 + k] = make_double2(f * red[2 * k], f * red[2 * k + 1]);
            C->eimg[k0 + k] = Ei;
        }
    }
}

// The accumulators of k_reorth_dots are compile-time sized and a kernel
// built for more vectors than a launch needs would still issue the FP64
// multiply-adds of the unused slots, so every count up to kChunk has its own
// instantiation (nk == NK in every launch).
using DotsKernel = void (*)(const ColDesc*, const int4*, ColScalars*, int, int, int, int, unsigned*);

template <int... N>
static constexpr std::array<DotsKernel, sizeof...(N)> dots_table(std::integer_sequence<int, N...>) {
    return {{&k_reorth_dots<N + 1>...}};
}

static DotsKernel dots_kernel(int nk) {
    static const std::array<DotsKernel, kChunk> exact = dots_table(std::make_integer_sequence<int, kChunk>{});
    return exact[nk - 1];
}

using IntDotsKernel = void (*)(const ColDesc*, const int4*, ColScalars*, int, int, int, unsigned*);

template <int... N>
static constexpr std::array<IntDotsKernel, sizeof...(N)> int_dots_table(std::integer_sequence<int, N...>) {
    return {{&k_reorth_dots_int<N + 1>...}};
}

static IntDotsKernel int_dots_kernel(int nk) {
    static const std::array<IntDotsKernel, kChunk> exact =
        int_dots_table(std::make_integer_sequence<int, kChunk>{});
    return exact[nk - 1];
}

// The exact integer dots serve first passes when every column has its images.
static bool use_int_dots(const Krylov& K, bool second) {
    if (second || (K.schedule & 4) || !K.Ibuf) return false;
    for (auto& D : K.hdesc)
        if (!D.I) return false;
    return true;
}

// a_j from the exact dots in the same pass as the Gram-Schmidt corrections
// (classical Gram-Schmidt of w against v_0..v_j at once) loses
// orthogonality over long Lanczos runs (a 120-step run past its exhausted
// 100-state sector diverged); a_j is therefore always H*psi's FP64 dot, and
// the exact dots correct it (u = w - a_j v_j first), as in the FP64 form.
bool alpha_in_dots(const Krylov&, int) { return false; }

int launch_reorth_dots(Krylov& K, int j, int k0, int nk, bool second, cudaStream_t st) {
    ProfScope ps("reorth_dots", st);
    if (use_int_dots(K, second)) {
        const IntDotsKernel ik = int_dots_kernel(nk);
        const int4* items;
        int n;
        KG_TRY(work_list(K, (const void*)ik, -1, &items, &n));
        ik<<<n, kThreads, 0, st>>>(K.desc, items, K.cs, j, k0, nk, K.cnt);
        KG_LAUNCHED();
        return KG_OK;
    }
    const DotsKernel kern = dots_kernel(nk);
    const int4* items;
    int n;
    KG_TRY(work_list(K, (const void*)kern, -1, &items, &n));
    kern<<<n, kThreads, 0, st>>>(K.desc, items, K.cs, j, k0, nk, second ? 1 : 0, K.cnt);
    KG_LAUNCHED();
    return KG_OK;
}

// ------------------------------------------------------ the update
// First pass:  V_{j+1} = W - a_j v_j - [reorth] sum_{k<=j} h_k v_k
// Second pass: V_{j+1} -= sum_{k<=j} h_k v_k
// then b_{j+1} = ||V_{j+1}||, s_{j+1} = 1/b_{j+1}, a_j += Re h_j, the
// largest exponent of V_{j+1}, and the breakdown test (the Krylov space is
// invariant when b_{j+1} is at rounding level relative to |a_j| + b_j).
//
// After the three-term subtraction the Gram-Schmidt coefficients are at
// rounding level (|h_k| ~ 1e-14 for unit vectors).  A term whose coefficient
// is below kSmallCoef is accumulated in FP32 (FP32 FMA on the truncated
// vector): its error, < 2^-23 |h_k| |v_k[i]| < 1.2e-17 |v_k[i]|, is far
// below the FP64 rounding of the result, and the FP32 pipe is 64 times wider
// than the FP64 pipe on this GPU.  Larger coefficients use FP64.
constexpr double kSmallCoef = 1e-10;

__global__ void __launch_bounds__(kThreads) k_update(const ColDesc* desc, const int4* items, ColScalars* cs, int j,
                                                     int level, int second, unsigned* cnt) {
    // block-uniform term lists: FP32 terms (small coefficients), FP64 terms
    __shared__ double2 coef64[kMaxMgs + 1];
    __shared__ float2 coef32[kMaxMgs + 1];
    __shared__ int idx32[kMaxMgs + 1], idx64[kMaxMgs + 1];
    __shared__ int n32, n64, efix_s;
    __shared__ double coefA;
    __shared__ double sm[(kThreads / 32) * 2];
    __shared__ int smi[kThreads / 32];
    __shared__ double bs[2], red[2];
    KG_ITEM();
    if (j >= C->m_eff) return;
    const int d = D.d;
    double2* Vb = D.V;
    const int nk = (level >= 1 || second) ? j + 1 : 0;
    // a first pass whose a_j came from the exact dots (alpha[j] still 0):
    // Re h_j is a_j, subtracted here in FP64 (its tiny imaginary part joins
    // the other Gram-Schmidt terms), from w itself
    const bool ain = !second && level >= 1 && C->alpha[j] == 0.0;
    if (threadIdx.x == 0) {
        int a32 = 0, a64 = 0;
        coefA = 0.0;
        for (int k = 0; k < nk; ++k) {
            const double s = C->scale[k];
            double2 h = C->h[k];
            if (ain && k == j) {
                coefA = s * h.x;
                h.x = 0.0;
            }
            const double2 c = make_double2(s * h.x, s * h.y);
            if ((fabs(h.x) + fabs(h.y)) < kSmallCoef) {  // |h_k| for the unit vector v_k
                coef32[a32] = make_float2((float)c.x, (float)c.y);
                idx32[a32++] = k;
            } else {
                coef64[a64] = c;
                idx64[a64++] = k;
            }
        }
        n32 = a32;
        n64 = a64;
    }
    __syncthreads();
    const int m32 = n32, m64 = n64;
    const double aj = C->alpha[j] * C->scale[j], cA = coefA;
    const double2* w = second ? Vb + (size_t)(j + 1) * d : D.W;
    const double2* vj = Vb + (size_t)j * d;
    double2* out = Vb + (size_t)(j + 1) * d;
    const float2* V32 = D.V32;
    double* S1 = D.S ? D.S + (size_t)(j + 1) * d : nullptr;
    float2* V32_1 = D.V32 ? D.V32 + (size_t)(j + 1) * d : nullptr;
    double acc[1] = {0.0};
    int em = 0;
    // after a first-pass Gram-Schmidt (level >= 1) U holds W - a_j v_j
    const bool sub = !second && level < 1;
    const double2* win = (!second && level >= 1 && !ain) ? D.U : w;
    auto element = [&](int i) {
        double2 u = win[i];
        if (sub) {
            const double2 p = vj[i];
            u.x = fma(-aj, p.x, u.x);
            u.y = fma(-aj, p.y, u.y);
        }
        float cx = 0.f, cy = 0.f;
        int q = 0;
        if (V32) {
            // eight loads in flight before their terms are applied
            for (; q + 8 <= m32; q += 8) {
                float2 v[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) v[r] = V32[(size_t)idx32[q + r] * d + i];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float2 c = coef32[q + r];
                    cx = fmaf(c.x, v[r].x, fmaf(-c.y, v[r].y, cx));
                    cy = fmaf(c.x, v[r].y, fmaf(c.y, v[r].x, cy));
                }
            }
            if (q + 4 <= m32) {
                float2 v[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) v[r] = V32[(size_t)idx32[q + r] * d + i];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float2 c = coef32[q + r];
                    cx = fmaf(c.x, v[r].x, fmaf(-c.y, v[r].y, cx));
                    cy = fmaf(c.x, v[r].y, fmaf(c.y, v[r].x, cy));
                }
                q += 4;
            }
            for (; q < m32; ++q) {
                const float2 v = V32[(size_t)idx32[q] * d + i], c = coef32[q];
                cx = fmaf(c.x, v.x, fmaf(-c.y, v.y, cx));
                cy = fmaf(c.x, v.y, fmaf(c.y, v.x, cy));
            }
        } else {
            for (; q < m32; ++q) {
                const double2 v = Vb[(size_t)idx32[q] * d + i];
                const float2 c = coef32[q];
                const float vx = f64_to_f32_trunc(v.x), vy = f64_to_f32_trunc(v.y);
                cx = fmaf(c.x, vx, fmaf(-c.y, vy, cx));
                cy = fmaf(c.x, vy, fmaf(c.y, vx, cy));
            }
        }
        for (int r = 0; r < m64; ++r) {
            const double2 v = Vb[(size_t)idx64[r] * d + i], c = coef64[r];
            u.x -= fma(c.x, v.x, -c.y * v.y);
            u.y -= fma(c.x, v.y, c.y * v.x);
        }
        if (ain) {
            const double2 p = vj[i];
            u.x = fma(-cA, p.x, u.x);
            u.y = fma(-cA, p.y, u.y);
        }
        u.x -= f32_to_f64_int(cx);
        u.y -= f32_to_f64_int(cy);
        out[i] = u;
        if (S1) {
            S1[i] = u.x + u.y;
            V32_1[i] = make_float2(f64_to_f32_trunc(u.x), f64_to_f32_trunc(u.y));
        }
        acc[0] = fma(u.x, u.x, fma(u.y, u.y, acc[0]));
        em = max(em, max(exp_field(u.x), exp_field(u.y)));
        return u;
    };
    const bool img = D.I != nullptr && level >= 1;  // images for the exact Gram-Schmidt dots
    if ((D.Xf || img) && (second || level < 2)) {
        // Last pass of an exact-integer column: also write the fixed-point
        // image of V_{j+1} that the next H*psi reads, on the exponent efix;
        // with the exact dots, also its 52-bit image I_{j+1} on the same one.
        // The vector's largest exponent is only known at the end of this
        // kernel, so efix bounds it from the inputs: every component of the
        // result is below
        //   2^(E_u - 1022) + |a_j| 2^(E_j - 1022) + sum_k (|Re c_k| + |Im c_k|) 2^(E_k - 1022)
        // (E_u: largest exponent of W, or of V_{j+1} in a second pass), times
        // a margin for the rounding of the FP64 and FP32 arithmetic.
        if (threadIdx.x == 0) {
            const int Eu = second ? C->emax[j + 1] : C->ew;
            double r = 1.0;
            if (!second) r += (fabs(aj) + fabs(cA)) * ldexp(1.0, C->emax[j] - Eu);
            for (int q = 0; q < m32; ++q)
                r += (fabs((double)coef32[q].x) + fabs((double)coef32[q].y)) * ldexp(1.0, C->emax[idx32[q]] - Eu);
            for (int q = 0; q < m64; ++q)
                r += (fabs(coef64[q].x) + fabs(coef64[q].y)) * ldexp(1.0, C->emax[idx64[q]] - Eu);
            r *= 1.0 + 1.0 / 1024.0;
            int ex;
            const double fr = frexp(r, &ex);  // r = fr * 2^ex, fr in [0.5, 1)
            efix_s = Eu + (fr == 0.5 ? ex - 1 : ex);
        }
        __syncthreads();
        const int Ef = efix_s, P = D.fix_pre;
        int4* I1 = img ? D.I + (size_t)(j + 1) * d : nullptr;
        if (D.Xf && img) {
            KG_FOR(i) {
                const double2 u = element(i);
                D.Xf[i] = make_longlong2(fix_term(u.x, Ef, P, 0u), fix_term(u.y, Ef, P, 0u));
                I1[i] = fix_image(u, Ef);
            }
        } else if (D.Xf) {
            KG_FOR(i) {
                const double2 u = element(i);
                D.Xf[i] = make_longlong2(fix_term(u.x, Ef, P, 0u), fix_term(u.y, Ef, P, 0u));
            }
        } else {
            KG_FOR(i) I1[i] = fix_image(element(i), Ef);
        }
        if (blk == 0 && threadIdx.x == 0) {
            if (D.Xf) C->efix = Ef;
            if (img) C->eimg[j + 1] = Ef;
        }
    } else {
        KG_FOR(i) element(i);
    }
    em = block_max_int(em, smi);
    block_sum<1>(acc, 1, sm, bs);
    if (threadIdx.x == 0) bs[1] = (double)em;
    __syncthreads();
    if (grid_finish(bs, 1, D.part, cnt + b, blk, nblk, red, 1) && threadIdx.x == 0) {
        C->emax[j + 1] = (int)red[1];
        const double n = sqrt(red[0]);
        double a = C->alpha[j];
        if (nk) a += C->h[j].x;
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

int launch_update(Krylov& K, int j, int level, bool second, cudaStream_t st) {
    ProfScope ps("update", st);
    const int4* items;
    int n;
    KG_TRY(work_list(K, (const void*)k_update, -1, &items, &n));
    k_update<<<n, kThreads, 0, st>>>(K.desc, items, K.cs, j, level, second ? 1 : 0, K.cnt);
    KG_LAUNCHED();
    return KG_OK;
}

// ------------------------------------------- tridiagonal eigenproblem
// One warp per column.  Implicit symmetric QR with Wilkinson shifts on the
// unreduced blocks of T (Golub and Van Loan, Section 8.3): lane 0 chases the
// bulge and records the Givens rotations of one sweep in shared memory, then
// all lanes apply them to their rows of Q (Q <- Q R_k).  On exit T = Q D Q^T.
//   mode 0 (propagation, Eq. (udelta)), with the column's tau:
//       c_k = beta0 * sum_m Q[k][m] e^{-i lambda_m tau} Q[0][m]
//   mode 1 (ground state, Eq. (eigen)): c_k = Q[k][m0] for the lowest m0,
//       lam0, lam1 = two lowest Ritz values, resest = |b_m Q[m-1][m0]|.
// The stored combination coefficient is c_k * s_k (Lanczos vectors are
// unnormalised).
//
// On this GPU a warp's FP64 instruction occupies the FP64 pipe for many
// cycles even with one active lane, so the serial chase is what costs: each
// rotation takes one reciprocal square root instead of a hypot and two
// divisions, and Q stays in shared memory for m <= 32 (every propagation
// step), so that applying a sweep's rotations does not wait on L2.
constexpr int kTriWarps = 2;
constexpr int kTriSmemQ = 32;

__global__ void __launch_bounds__(32 * kTriWarps) k_tridiag(const ColDesc* desc, ColScalars* cs, int B, int Mcap,
                                                           double* Qall, int mode, const double* taus, int ntau,
                                                           double2* cq) {
    __shared__ double sd[kTriWarps][kMaxMgs], se[kTriWarps][kMaxMgs];
    __shared__ double rc[kTriWarps][kMaxMgs], rs[kTriWarps][kMaxMgs];
    __shared__ int ctl[kTriWarps][4];
    __shared__ double sQ[kTriWarps][kTriSmemQ * kTriSmemQ];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * kTriWarps + warp;
    if (b >= B) return;
    ColScalars* C = cs + b;
    const double tau = desc[b].tau;
    const int m = C->m_eff;
    double* Q = m <= kTriSmemQ ? sQ[warp] : Qall + (size_t)b * Mcap * Mcap;
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
                    // Givens rotation zeroing z against x: r = |(x, z)|
                    const double r2 = fma(x, x, z * z);
                    double c = 1.0, s = 0.0, r = 0.0;
                    if (r2 > 0.0) {
                        const double inv = rsqrt(r2);
                        c = x * inv;
                        s = z * inv;
                        r = r2 * inv;
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
    if (lane == 0 && iter >= max_iter && C->status == KG_OK) C->status = KG_ENOCONV;
    __syncwarp();
    if (mode == 0 || mode == 2) {
        // mode 0: the column's own tau into C->c; mode 2: ntau times
        // (quadrature nodes) into cq[b][t][k], from the same diagonalisation
        const double beta0 = C->beta0;
        double* pc = rc[warp];  // rotation buffers are free now: phases of e^{-i lambda tau}
        double* ps = rs[warp];
        const int nt = mode == 0 ? 1 : ntau;
        for (int t = 0; t < nt; ++t) {
            const double tt = mode == 0 ? tau : taus[(size_t)b * ntau + t];
            __syncwarp();
            for (int mm = lane; mm < m; mm += 32) {
                double sn, cn;
                sincos(d[mm] * tt, &sn, &cn);
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
                if (mode == 0)
                    C->c[k] = make_double2(s * re, s * im);
                else
                    cq[((size_t)b * ntau + t) * Mcap + k] = make_double2(s * re, s * im);
            }
        }
        if (mode == 2)
            for (int t = 0; t < ntau; ++t)
                for (int k = m + lane; k < Mcap; k += 32) cq[((size_t)b * ntau + t) * Mcap + k] = make_double2(0.0, 0.0);
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

// ------------------------------------ step exponential by a Taylor series
// c = beta0 e^{-i T tau} e_1 (times s_k per component), the vector of
// Eq. (udelta), without the eigen-decomposition: the series in (-i T h)
// with h = tau / n_sub and n_sub chosen so that |T h| <= 1/2 (Gershgorin
// bound), 18 terms per sub-step (remainder below 1e-22 of the sum).  One
// warp per column; lane l holds components l and l + 32 (R = 2), so every
// FP64 instruction serves the whole vector -- the eigen-decomposition's
// bulge chase is serial.  Modes 0 and 2 as in k_tridiag.
constexpr int kTaylorTerms = 18;
constexpr int kMaxTaus = 32;  // times per column in one mode-2 launch

template <int R>
__device__ __forceinline__ void tri_apply(const double (&a)[R], const double (&bl)[R], const double (&br)[R],
                                          const double2 (&x)[R], double2 (&y)[R], int lane) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        // x_{k-1} and x_{k+1} for k = lane + 32 r
        double2 xm, xp;
        xm.x = __shfl_up_sync(0xffffffffu, x[r].x, 1);
        xm.y = __shfl_up_sync(0xffffffffu, x[r].y, 1);
        xp.x = __shfl_down_sync(0xffffffffu, x[r].x, 1);
        xp.y = __shfl_down_sync(0xffffffffu, x[r].y, 1);
        const double2 lo = r > 0 ? x[r > 0 ? r - 1 : 0] : make_double2(0.0, 0.0);
        const double2 hi = r + 1 < R ? x[r + 1 < R ? r + 1 : r] : make_double2(0.0, 0.0);
        const double lox = __shfl_sync(0xffffffffu, lo.x, 31), loy = __shfl_sync(0xffffffffu, lo.y, 31);
        const double hix = __shfl_sync(0xffffffffu, hi.x, 0), hiy = __shfl_sync(0xffffffffu, hi.y, 0);
        if (lane == 0) xm = make_double2(lox, loy);
        if (lane == 31) xp = make_double2(hix, hiy);
        y[r].x = fma(a[r], x[r].x, fma(bl[r], xm.x, br[r] * xp.x));
        y[r].y = fma(a[r], x[r].y, fma(bl[r], xm.y, br[r] * xp.y));
    }
}

template <int R>
__global__ void __launch_bounds__(32 * kTriWarps) k_texp(const ColDesc* desc, ColScalars* cs, int B, int Mcap,
                                                        int mode, const double* taus, int ntau, double2* cq) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * kTriWarps + warp;
    if (b >= B) return;
    ColScalars* C = cs + b;
    const int m = C->m_eff;
    if (m == 0) {
        for (int k = lane; k < Mcap; k += 32) C->c[k] = make_double2(0.0, 0.0);
        if (mode == 2)
            for (int t = 0; t < ntau; ++t)
                for (int k = lane; k < Mcap; k += 32) cq[((size_t)b * ntau + t) * Mcap + k] = make_double2(0.0, 0.0);
        return;
    }
    double a[R], bl[R], br[R];
    double g = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int k = lane + 32 * r;
        a[r] = k < m ? C->alpha[k] : 0.0;
        bl[r] = (k < m && k >= 1) ? C->beta[k] : 0.0;      // couples k-1 and k
        br[r] = (k + 1 < m) ? C->beta[k + 1] : 0.0;         // couples k and k+1
        g = fmax(g, fabs(a[r]) + fabs(bl[r]) + fabs(br[r]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
    const double beta0 = C->beta0;
    const int nt = mode == 0 ? 1 : ntau;
    // Several times of one sign (mode 2: quadrature nodes) are taken in order
    // of |tau|, each from the previous result: e^{-iT t_n} e_1 =
    // e^{-iT (t_n - t_{n-1})} e^{-iT t_{n-1}} e_1.  Times of mixed signs
    // restart from e_1.
    int order[kMaxTaus];
    for (int t = 0; t < nt; ++t) order[t] = t;
    if (mode == 2)
        for (int a1 = 1; a1 < nt; ++a1)  // insertion sort by |tau| (nt <= kMaxTaus)
            for (int a2 = a1; a2 > 0 && fabs(taus[(size_t)b * ntau + order[a2]]) <
                                            fabs(taus[(size_t)b * ntau + order[a2 - 1]]); --a2) {
                const int tmp = order[a2];
                order[a2] = order[a2 - 1];
                order[a2 - 1] = tmp;
            }
    double2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = make_double2((lane + 32 * r) == 0 ? 1.0 : 0.0, 0.0);
    double tprev = 0.0;
    for (int tt = 0; tt < nt; ++tt) {
        const int t = order[tt];
        const double tfull = mode == 0 ? desc[b].tau : taus[(size_t)b * ntau + t];
        if (tfull * tprev < 0.0) {  // sign change: start again from e_1
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = make_double2((lane + 32 * r) == 0 ? 1.0 : 0.0, 0.0);
            tprev = 0.0;
        }
        const double tau = tfull - tprev;
        tprev = tfull;
        // a non-finite or absurdly large T (more than kMaxSub sub-steps)
        // cannot be exponentiated this way: report it instead of looping
        const double want = 2.0 * g * fabs(tau);
        if (!(want <= (double)kMaxSub)) {
            if (lane == 0) C->status = KG_ENUMERIC;
            for (int k = lane; k < Mcap; k += 32) C->c[k] = make_double2(0.0, 0.0);
            if (mode == 2)
                for (int t2 = 0; t2 < ntau; ++t2)
                    for (int k = lane; k < Mcap; k += 32) cq[((size_t)b * ntau + t2) * Mcap + k] = make_double2(0.0, 0.0);
            return;
        }
        const int nsub = max(1, (int)ceil(want));
        const double h = tau / nsub;
        for (int sub = 0; sub < nsub; ++sub) {
            double2 term[R], sum[R], y[R];
#pragma unroll
            for (int r = 0; r < R; ++r) term[r] = sum[r] = v[r];
            for (int n = 1; n <= kTaylorTerms; ++n) {
                tri_apply<R>(a, bl, br, term, y, lane);
                const double f = h / n;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    term[r] = make_double2(f * y[r].y, -f * y[r].x);  // (-i h / n) T term
                    sum[r].x += term[r].x;
                    sum[r].y += term[r].y;
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = sum[r];
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = lane + 32 * r;
            if (k < m) {
                const double sc = beta0 * C->scale[k];
                const double2 cv = make_double2(sc * v[r].x, sc * v[r].y);
                if (mode == 0)
                    C->c[k] = cv;
                else
                    cq[((size_t)b * ntau + t) * Mcap + k] = cv;
            } else if (k < Mcap && mode == 2) {
                cq[((size_t)b * ntau + t) * Mcap + k] = make_double2(0.0, 0.0);
            }
        }
    }
}

static int launch_texp(Krylov& K, int mode, const double* taus, int ntau, double2* cq, cudaStream_t st) {
    const int nb = (K.B + kTriWarps - 1) / kTriWarps;
    if (K.M <= 32)
        k_texp<1><<<nb, 32 * kTriWarps, 0, st>>>(K.desc, K.cs, K.B, K.M, mode, taus, ntau, cq);
    else
        k_texp<2><<<nb, 32 * kTriWarps, 0, st>>>(K.desc, K.cs, K.B, K.M, mode, taus, ntau, cq);
    KG_LAUNCHED();
    return KG_OK;
}

int launch_tridiag(Krylov& K, int mode, cudaStream_t st) {
    const int nb = (K.B + kTriWarps - 1) / kTriWarps;
    ProfScope ps("tridiag", st);
    if (mode == 0 && !(K.schedule & 2)) return launch_texp(K, 0, nullptr, 0, nullptr, st);
    k_tridiag<<<nb, 32 * kTriWarps, 0, st>>>(K.desc, K.cs, K.B, K.M, K.Q, mode, nullptr, 0, nullptr);
    KG_LAUNCHED();
    return KG_OK;
}

// ----------------------------------- combination and overlaps
// out = sum_{k<m} c_k V_k  (Eq. (udelta) in the form V x small vector), then
// ||out|| and <ov_a, out> for the column's n_ov overlap vectors, written to
// row cs[b].ov_slot of its overlap table (the slot advances by one).  NOV
// bounds n_ov at compile time so that the accumulators stay in registers.
//
// The Krylov coefficients decay quickly with k.  As in the update, a term
// whose coefficient on the unit vector v_k is below 1e-10 of the largest one
// (which bounds ||out||) is summed in FP32 from the truncated plane; the
// others use three FP64 multiply-adds per element with the Re+Im plane
// (c = p + iq, v = a + ib: T1 = p a, T2 = q b, T3 = (p + q)(a + b),
// Re = T1 - T2, Im = T3 - T1 - T2), or four without it.
template <int NOV>
__global__ void __launch_bounds__(kThreads) k_combine(const ColDesc* desc, const int4* items, ColScalars* cs,
                                                      unsigned* cnt) {
    __shared__ double2 coef[kMaxMgs];
    __shared__ double csum[kMaxMgs];
    __shared__ int idx64[kMaxMgs], idx32[kMaxMgs];
    __shared__ float2 coef32[kMaxMgs];
    __shared__ int n64, n32;
    __shared__ double sm[(kThreads / 32) * (2 * NOV + 2)];
    __shared__ double bs[2 * NOV + 2], red[2 * NOV + 2];
    KG_ITEM();
    const int m = C->m_eff;
    if (threadIdx.x == 0) {
        double cmax = 0.0;
        for (int k = 0; k < m; ++k) {
            const double2 c = C->c[k];
            const double sk = C->scale[k];
            if (sk > 0.0) cmax = fmax(cmax, (fabs(c.x) + fabs(c.y)) / sk);
        }
        int a64 = 0, a32 = 0;
        for (int k = 0; k < m; ++k) {
            const double2 c = C->c[k];
            const double sk = C->scale[k];
            if (D.V32 && sk > 0.0 && (fabs(c.x) + fabs(c.y)) < 1e-10 * cmax * sk) {
                coef32[a32] = make_float2((float)c.x, (float)c.y);
                idx32[a32++] = k;
            } else {
                coef[a64] = c;
                csum[a64] = c.x + c.y;
                idx64[a64++] = k;
            }
        }
        n64 = a64;
        n32 = a32;
    }
    __syncthreads();
    const int m64 = n64, m32 = n32;
    const int d = D.d;
    const int n_ov = D.n_ov;
    const double2* Vb = D.V;
    double2* o = D.out;
    double acc[2 * NOV + 2];
#pragma unroll
    for (int k = 0; k < 2 * NOV + 2; ++k) acc[k] = 0.0;
    const double* Sb = D.S;
    const float2* V32 = D.V32;
    KG_FOR(i) {
        double2 u;
        if (Sb) {
            double t1 = 0.0, t2 = 0.0, t3 = 0.0;
            for (int q = 0; q < m64; ++q) {
                const size_t o_ = (size_t)idx64[q] * d + i;
                const double2 v = Vb[o_];
                const double sv = Sb[o_];
                const double2 c = coef[q];
                t1 = fma(c.x, v.x, t1);
                t2 = fma(c.y, v.y, t2);
                t3 = fma(csum[q], sv, t3);
            }
            u = make_double2(t1 - t2, t3 - t1 - t2);
        } else {
            u = make_double2(0.0, 0.0);
            for (int q = 0; q < m64; ++q) {
                const double2 v = Vb[(size_t)idx64[q] * d + i];
                const double2 c = coef[q];
                u.x = fma(c.x, v.x, fma(-c.y, v.y, u.x));
                u.y = fma(c.x, v.y, fma(c.y, v.x, u.y));
            }
        }
        if (m32) {
            float cx = 0.f, cy = 0.f;
            int q = 0;
            for (; q + 4 <= m32; q += 4) {
                float2 v[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) v[r] = V32[(size_t)idx32[q + r] * d + i];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float2 c = coef32[q + r];
                    cx = fmaf(c.x, v[r].x, fmaf(-c.y, v[r].y, cx));
                    cy = fmaf(c.x, v[r].y, fmaf(c.y, v[r].x, cy));
                }
            }
            for (; q < m32; ++q) {
                const float2 v = V32[(size_t)idx32[q] * d + i], c = coef32[q];
                cx = fmaf(c.x, v.x, fmaf(-c.y, v.y, cx));
                cy = fmaf(c.x, v.y, fmaf(c.y, v.x, cy));
            }
            u.x += (double)cx;
            u.y += (double)cy;
        }
        o[i] = u;
        acc[0] = fma(u.x, u.x, fma(u.y, u.y, acc[0]));
#pragma unroll
        for (int a = 0; a < NOV; ++a) {
            if (a < n_ov) {
                const double2 v = D.ov[(size_t)a * D.ov_stride + i];
                acc[2 + 2 * a] = fma(v.x, u.x, fma(v.y, u.y, acc[2 + 2 * a]));
                acc[3 + 2 * a] = fma(v.x, u.y, fma(-v.y, u.x, acc[3 + 2 * a]));
            }
        }
    }
    const int nv = 2 + 2 * n_ov;
    block_sum<2 * NOV + 2>(acc, nv, sm, bs);
    if (grid_finish(bs, nv, D.part, cnt + b, blk, nblk, red)) {
        const int slot = C->ov_slot;
        for (int a = threadIdx.x; a < n_ov; a += blockDim.x)
            if (slot < D.ov_rows) D.ov_out[(size_t)slot * n_ov + a] = make_double2(red[2 + 2 * a], red[3 + 2 * a]);
        __syncthreads();
        if (threadIdx.x == 0) {
            C->ovnorm = sqrt(red[0]);
            if (n_ov > 0) C->ov_slot = slot + 1;
        }
    }
}

int launch_combine(Krylov& K, cudaStream_t st) {
    int n_ov = 0;
    for (auto& D : K.hdesc) n_ov = std::max(n_ov, D.n_ov);
    if (n_ov > kMaxOv) {
        set_error("at most %d overlap vectors per combination pass", kMaxOv);
        return KG_EINVAL;
    }
    ProfScope ps("combine", st);
    const int4* items;
    int n;
#define KG_COMB(NOV)                                                              \
    do {                                                                          \
        KG_TRY(work_list(K, (const void*)k_combine<NOV>, -1, &items, &n));        \
        k_combine<NOV><<<n, kThreads, 0, st>>>(K.desc, items, K.cs, K.cnt);       \
    } while (0)
    if (n_ov == 0) KG_COMB(0);
    else if (n_ov <= 4) KG_COMB(4);
    else if (n_ov <= 12) KG_COMB(12);
    else KG_COMB(32);
#undef KG_COMB
    KG_LAUNCHED();
    return KG_OK;
}

// -------------------------------------------- ground-state residual
// rq = <x, y> (x normalised), then rnorm = ||y - rq x||.
__global__ void __launch_bounds__(kThreads) k_rq(const double2* x, const double2* y, int d, ColScalars* cs,
                                                 int phase, double* part, unsigned* cnt) {
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
    if (grid_finish(bs, 1, part, cnt, blockIdx.x, gridDim.x, red) && threadIdx.x == 0) {
        if (phase == 0)
            cs->rq = red[0];
        else
            cs->rnorm = sqrt(red[0]);
    }
}

// Coefficients of exp(-i H t) v_0 for ntau times per column (taus[b][t]),
// into cq[b][t][0..M) (already times the scales of the stored vectors).
int launch_tridiag_multi(Krylov& K, const double* taus, int ntau, double2* cq, cudaStream_t st) {
    if (ntau < 1 || ntau > kMaxTaus) {
        set_error("between 1 and %d times per column", kMaxTaus);
        return KG_EINVAL;
    }
    const int nb = (K.B + kTriWarps - 1) / kTriWarps;
    ProfScope ps("tridiag", st);
    if (!(K.schedule & 2)) return launch_texp(K, 2, taus, ntau, cq, st);
    k_tridiag<<<nb, 32 * kTriWarps, 0, st>>>(K.desc, K.cs, K.B, K.M, K.Q, 2, taus, ntau, cq);
    KG_LAUNCHED();
    return KG_OK;
}

// -------------------------------------------------- step sequencing
__global__ void k_set_slots(ColScalars* cs, int B, int value) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) cs[b].ov_slot = value;
}

__global__ void k_reset_status(ColScalars* cs, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) cs[b].status = KG_OK;
}

int launch_reset_status(Krylov& K, cudaStream_t st) {
    k_reset_status<<<(K.B + 127) / 128, 128, 0, st>>>(K.cs, K.B);
    KG_LAUNCHED();
    return KG_OK;
}

int launch_set_slots(Krylov& K, int value, cudaStream_t st) {
    k_set_slots<<<(K.B + 127) / 128, 128, 0, st>>>(K.cs, K.B, value);
    KG_LAUNCHED();
    return KG_OK;
}

int prepare_step(Krylov& K, int reorth) {
    const int4* items;
    int n;
    KG_TRY(prepare_hpsi_lists(K));
    KG_TRY(work_list(K, (const void*)k_colnorm, -1, &items, &n));
    KG_TRY(work_list(K, (const void*)k_update, -1, &items, &n));
    if (reorth >= 1) {
        // every vector count of one step (and of the ground-state restarts)
        for (int nk = 1; nk <= std::min(kChunk, K.M + 1); ++nk) {
            KG_TRY(work_list(K, (const void*)dots_kernel(nk), -1, &items, &n));
            if (use_int_dots(K, false)) KG_TRY(work_list(K, (const void*)int_dots_kernel(nk), -1, &items, &n));
        }
    }
    const void* comb[4] = {(const void*)k_combine<0>, (const void*)k_combine<4>, (const void*)k_combine<12>,
                           (const void*)k_combine<32>};
    for (auto* k : comb) KG_TRY(work_list(K, k, -1, &items, &n));
    return KG_OK;
}

int enqueue_step(Krylov& K, int reorth, cudaStream_t st) {
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
    KG_TRY(launch_tridiag(K, 0, st));
    KG_TRY(launch_combine(K, st));
    return KG_OK;
}

// ------------------------------------------------------ ground state
int ground_state(kg_sector* s, const kg_opts* o) {
    cudaStream_t st = pick_stream(s, o);
    const int d = (int)s->d;
    if (o->M_gs < 2 || o->M_gs > kMaxMgs) {
        set_error("M_gs must be in [2, %d]", kMaxMgs);
        return KG_EINVAL;
    }
    const int M = std::max(1, std::min(o->M_gs, d));
    if (!s->gs) KG_CUDA(cudaMalloc(&s->gs, sizeof(double2) * d));
    Krylov K;
    int rc = krylov_alloc(K, {s}, M, s->nsm, o->schedule);
    if (rc != KG_OK) {
        krylov_free(K);
        return rc;
    }
    auto done = [&](int r) {
        krylov_free(K);
        return r;
    };
    K.hdesc[0].out = s->gs;  // the Ritz vector of each restart goes to the cache
    rc = krylov_upload(K, st);
    const SecView S = s->view();
    double2* V0 = K.vec(0, 0);
    double2* W0 = K.hdesc[0].W;
    double* part = K.hdesc[0].part;
    const int nrq = std::max(1, std::min(K.hdesc[0].nblk_max, (d + kThreads - 1) / kThreads));
    if (rc == KG_OK) rc = launch_random_start(V0, d, o->seed, st);
    ColScalars h;
    bool converged = false;
    for (int r = 0; rc == KG_OK && r < o->max_restarts; ++r) {
        if ((rc = launch_colnorm(K, st)) != KG_OK) break;
        for (int j = 0; j < M && rc == KG_OK; ++j) {
            rc = launch_lanczos_hpsi(K, j, st, !alpha_in_dots(K, 1));
            for (int k0 = 0; rc == KG_OK && k0 <= j; k0 += kChunk)
                rc = launch_reorth_dots(K, j, k0, std::min(kChunk, j + 1 - k0), false, st);
            if (rc == KG_OK) rc = launch_update(K, j, std::max(1, o->reorth), false, st);
            if (rc == KG_OK && o->reorth >= 2) {
                for (int k0 = 0; rc == KG_OK && k0 <= j; k0 += kChunk)
                    rc = launch_reorth_dots(K, j, k0, std::min(kChunk, j + 1 - k0), true, st);
                if (rc == KG_OK) rc = launch_update(K, j, o->reorth, true, st);
            }
        }
        if (rc == KG_OK) rc = launch_tridiag(K, 1, st);
        if (rc == KG_OK) rc = launch_combine(K, st);
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
        if ((rc = launch_hpsi(s, s->gs, W0, st)) != KG_OK) break;
        k_rq<<<nrq, kThreads, 0, st>>>(s->gs, W0, d, K.cs, 0, part, K.cnt);
        count_launch();
        k_rq<<<nrq, kThreads, 0, st>>>(s->gs, W0, d, K.cs, 1, part, K.cnt);
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
        if (cudaMemcpyAsync(V0, s->gs, sizeof(double2) * d, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
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
