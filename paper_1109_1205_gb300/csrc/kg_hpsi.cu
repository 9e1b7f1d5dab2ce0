// kg_hpsi.cu -- the Hamiltonian applied on the fly in the
// occupation-number basis (Section 2, H_jj'; model Hamiltonians of Sections 3
// and 4).  One thread produces one output element y[s], s = i_dn*D_up + i_up:
//
//   y[s] = (e_up[i_up] + e_dn[i_dn] + U(b_up & b_dn)) x[s]
//        + sum_{up hops of i_up}  (+-h_ab) x[i_dn*D_up + j]     (same row)
//        + sum_{down hops of i_dn}(+-h_ab) x[j*D_up + i_up]     (other rows)
//
// Up hops gather inside one row (L1/L2 resident); down hops read whole rows
// at a stride of D_up, so a warp (consecutive i_up, one i_dn) walks the same
// down-hop list and its loads are coalesced.
//
// Hop sums.  The FP64 pipe of this GPU issues about two lanes per clock per
// SM, 64 times fewer than the integer pipe.  When every hop has the same
// amplitude h0 (the Hubbard ring and the SIAM chain), the hop part is h0 times
// a signed sum of gathered components, which is computed exactly on the
// integer pipe: each component becomes the 64-bit fixed-point number
// round(x * 2^(1075 + P - E)), E the largest exponent field of the vector and
// P = 9 - ceil(log2(hops + 1)) the head room, so no sum can overflow.  The
// sum is exact; the only rounding is the conversion of each term, at most
// 2^-57 of the vector's largest component, and one conversion back to FP64.
// Other hoppings (site-dependent or complex amplitudes) use FP64 FMAs.
#include <algorithm>

#include "kg_internal.h"

namespace kg {

__device__ __forceinline__ double flip(double v, uint32_t code) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(code >> 31) << 63));
}

// Fixed-point image of x with the vector's largest exponent field E and
// pre-shift P; the hop sign `neg` (0/1) is applied together with x's own.
__device__ __forceinline__ long long fix_term(double x, int E, int P, uint32_t neg) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffull);
    const unsigned long long m = ((b & 0xfffffffffffffull) | 0x10000000000000ull) << P;
    const int r = min(E - e, 63);
    const unsigned long long half = (1ull << r) >> 1;
    long long v = (long long)((m + half) >> r);
    v = e ? v : 0ll;
    return ((uint32_t)(b >> 63) ^ neg) ? -v : v;
}

template <int MODE>
__device__ __forceinline__ void hop_acc(double2& acc, uint32_t code, double2 xs, const double2* amp) {
    if (MODE == 0) {
        acc.x += flip(xs.x, code);
        acc.y += flip(xs.y, code);
    } else if (MODE == 1) {
        const double a = flip(amp[code & 1023u].x, code);
        acc.x = fma(a, xs.x, acc.x);
        acc.y = fma(a, xs.y, acc.y);
    } else {
        double2 a = amp[code & 1023u];
        a.x = flip(a.x, code);
        a.y = flip(a.y, code);
        acc.x = fma(a.x, xs.x, fma(-a.y, xs.y, acc.x));
        acc.y = fma(a.x, xs.y, fma(a.y, xs.x, acc.y));
    }
}

__device__ __forceinline__ double diag_energy(const SecView& S, int i_dn, int i_up, const double* utab) {
    const uint32_t both = __ldg(S.up_bits + i_up) & __ldg(S.dn_bits + i_dn);
    double diag = __ldg(S.up_e + i_up) + __ldg(S.dn_e + i_dn);
    for (int c = 0; c < S.nchunk; ++c) diag += utab[c * 256 + ((both >> (8 * c)) & 255u)];
    return diag;
}

// Hop part of (H x)[i_dn, i_up].  MODE 0-2: FP64 accumulation (MODE 0 without
// the amplitude, applied by the caller); MODE 3: exact integer accumulation,
// returned in (ix, iy) as fixed-point sums.
template <int MODE>
__device__ __forceinline__ void hop_sum(const SecView& S, const double2* __restrict__ x, int i_dn, int i_up,
                                        const double2* amp, int E, double2& hop, long long& ix, long long& iy) {
    const double2* row = x + (size_t)i_dn * S.Du;
    const int u0 = __ldg(S.up_off + i_up), u1 = __ldg(S.up_off + i_up + 1);
    const int d0 = __ldg(S.dn_off + i_dn), d1 = __ldg(S.dn_off + i_dn + 1);
    if (MODE == 3) {
        const int P = S.fix_pre;
#pragma unroll 4
        for (int e = u0; e < u1; ++e) {
            const uint2 en = __ldg(S.up_ent + e);
            const double2 xs = row[en.x];
            ix += fix_term(xs.x, E, P, en.y >> 31);
            iy += fix_term(xs.y, E, P, en.y >> 31);
        }
#pragma unroll 4
        for (int e = d0; e < d1; ++e) {
            const uint2 en = __ldg(S.dn_ent + e);
            const double2 xs = x[(size_t)en.x * S.Du + i_up];
            ix += fix_term(xs.x, E, P, en.y >> 31);
            iy += fix_term(xs.y, E, P, en.y >> 31);
        }
    } else {
#pragma unroll 4
        for (int e = u0; e < u1; ++e) {
            const uint2 en = __ldg(S.up_ent + e);
            hop_acc<MODE>(hop, en.y, row[en.x], amp);
        }
#pragma unroll 4
        for (int e = d0; e < d1; ++e) {
            const uint2 en = __ldg(S.dn_ent + e);
            hop_acc<MODE>(hop, en.y, x[(size_t)en.x * S.Du + i_up], amp);
        }
    }
}

// 2^(E - 1075 - P): value of one unit of the fixed-point sums.
__device__ __forceinline__ double fix_unit(int E, int P) {
    const long long ex = (long long)E - 52 - P;  // biased exponent of the unit
    return ex > 0 ? __longlong_as_double(ex << 52) : 0.0;
}

__device__ __forceinline__ void stage_tables(const SecView& S, double2* amp, double* utab) {
    for (int k = threadIdx.x; k < S.L * S.L; k += blockDim.x) amp[k] = S.hamp[k];
    for (int k = threadIdx.x; k < S.nchunk * 256; k += blockDim.x) utab[k] = S.Utab[k];
    __syncthreads();
}

// Largest exponent field over the components of x, into *emax (pre-set to 0).
__global__ void __launch_bounds__(kThreads) k_maxexp(const double2* __restrict__ x, int d, int* emax) {
    __shared__ int sm[kThreads / 32];
    int m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        const double2 v = x[i];
        m = max(m, max(exp_field(v.x), exp_field(v.y)));
    }
    m = block_max_int(m, sm);
    if (threadIdx.x == 0) atomicMax(emax, m);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_hpsi(SecView S, const double2* __restrict__ x,
                                                   double2* __restrict__ y, const int* emax) {
    __shared__ double2 amp[kMaxL * kMaxL];
    __shared__ double utab[4 * 256];
    stage_tables(S, amp, utab);
    const int E = (MODE == 3) ? *emax : 0;
    const double unit = (MODE == 3) ? fix_unit(E, S.fix_pre) * S.h0 : 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < S.d; idx += gridDim.x * blockDim.x) {
        int i_dn, i_up;
        split_index(S, idx, i_dn, i_up);
        const double2 xv = x[idx];
        const double diag = diag_energy(S, i_dn, i_up, utab);
        double2 hop = make_double2(0.0, 0.0);
        long long ix = 0, iy = 0;
        hop_sum<MODE>(S, x, i_dn, i_up, amp, E, hop, ix, iy);
        double2 r;
        if (MODE == 3) {
            r.x = fma(diag, xv.x, unit * __ll2double_rn(ix));
            r.y = fma(diag, xv.y, unit * __ll2double_rn(iy));
        } else if (MODE == 0) {
            r.x = fma(diag, xv.x, S.h0 * hop.x);
            r.y = fma(diag, xv.y, S.h0 * hop.y);
        } else {
            r.x = fma(diag, xv.x, hop.x);
            r.y = fma(diag, xv.y, hop.y);
        }
        y[idx] = r;
    }
}

// Lanczos step j for column b of a work-list launch:
//   w = s_j H V_j - b_j s_{j-1} V_{j-1},   a_j = Re <s_j V_j, w>
// (Eq. (recursion) with normalised v_k = s_k V_k).
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_lanczos_hpsi(const ColDesc* desc, const int4* items, ColScalars* cs,
                                                           int j, unsigned* cnt) {
    __shared__ double2 amp[kMaxL * kMaxL];
    __shared__ double utab[4 * 256];
    __shared__ double sm[(kThreads / 32) * 2];
    __shared__ double bs[2], red[2];
    __shared__ SecView S;
    KG_ITEM();
    if (j >= C->m_eff) return;
    if (threadIdx.x == 0) S = *D.sec;
    __syncthreads();
    stage_tables(S, amp, utab);
    const double sj = C->scale[j];
    const double cprev = (j > 0) ? C->beta[j] * C->scale[j - 1] : 0.0;
    const int E = (MODE == 3) ? C->emax[j] : 0;
    const double unit = (MODE == 3) ? fix_unit(E, S.fix_pre) * S.h0 * sj : 0.0;
    const double hs = S.h0 * sj;
    const double2* x = D.V + (size_t)j * D.d;
    const double2* xp = D.V + (size_t)(j > 0 ? j - 1 : 0) * D.d;
    double2* w = D.W;
    double acc[2] = {0.0, 0.0};
    KG_FOR(idx) {
        int i_dn, i_up;
        split_index(S, idx, i_dn, i_up);
        const double2 xv = x[idx];
        const double sdiag = sj * diag_energy(S, i_dn, i_up, utab);
        double2 hop = make_double2(0.0, 0.0);
        long long ix = 0, iy = 0;
        hop_sum<MODE>(S, x, i_dn, i_up, amp, E, hop, ix, iy);
        double2 p = make_double2(0.0, 0.0);
        if (j > 0) p = xp[idx];
        double2 r;
        if (MODE == 3) {
            r.x = fma(sdiag, xv.x, fma(unit, __ll2double_rn(ix), -cprev * p.x));
            r.y = fma(sdiag, xv.y, fma(unit, __ll2double_rn(iy), -cprev * p.y));
        } else if (MODE == 0) {
            r.x = fma(sdiag, xv.x, fma(hs, hop.x, -cprev * p.x));
            r.y = fma(sdiag, xv.y, fma(hs, hop.y, -cprev * p.y));
        } else {
            r.x = fma(sdiag, xv.x, fma(sj, hop.x, -cprev * p.x));
            r.y = fma(sdiag, xv.y, fma(sj, hop.y, -cprev * p.y));
        }
        w[idx] = r;
        acc[0] = fma(xv.x, r.x, fma(xv.y, r.y, acc[0]));  // Re conj(x) r
    }
    acc[0] *= sj;
    block_sum<2>(acc, 1, sm, bs);
    if (grid_finish(bs, 1, D.part, cnt + b, blk, nblk, red)) {
        if (threadIdx.x == 0) {
            const double a = red[0];
            C->alpha[j] = a;
            if (!isfinite(a)) {
                C->status = KG_ENUMERIC;
                C->m_eff = j + 1;
            }
        }
    }
}

int launch_hpsi(const SecView& S, const double2* x, double2* y, cudaStream_t st) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int nb = std::max(1, std::min((S.d + kThreads - 1) / kThreads, nsm * 8));
    if (S.hopmode == 0 && S.fix_pre >= 0) {
        // largest exponent of x first (one extra read of x), then exact hop sums
        static thread_local int* d_emax = nullptr;
        if (!d_emax) KG_CUDA(cudaMalloc(&d_emax, sizeof(int)));
        ProfScope ps("hpsi", st);
        KG_CUDA(cudaMemsetAsync(d_emax, 0, sizeof(int), st));
        k_maxexp<<<std::min(nb, nsm * 4), kThreads, 0, st>>>(x, S.d, d_emax);
        KG_LAUNCHED();
        k_hpsi<3><<<nb, kThreads, 0, st>>>(S, x, y, d_emax);
        KG_LAUNCHED();
        return KG_OK;
    }
    ProfScope ps("hpsi", st);
    if (S.hopmode == 0)
        k_hpsi<0><<<nb, kThreads, 0, st>>>(S, x, y, nullptr);
    else if (S.hopmode == 1)
        k_hpsi<1><<<nb, kThreads, 0, st>>>(S, x, y, nullptr);
    else
        k_hpsi<2><<<nb, kThreads, 0, st>>>(S, x, y, nullptr);
    KG_LAUNCHED();
    return KG_OK;
}

int prepare_hpsi_lists(Krylov& K) {
    bool present[4] = {false, false, false, false};
    for (auto& D : K.hdesc) present[D.mode] = true;
    const void* kerns[4] = {(const void*)k_lanczos_hpsi<0>, (const void*)k_lanczos_hpsi<1>,
                            (const void*)k_lanczos_hpsi<2>, (const void*)k_lanczos_hpsi<3>};
    for (int mode = 0; mode < 4; ++mode) {
        if (!present[mode]) continue;
        const int4* items;
        int n;
        KG_TRY(work_list(K, kerns[mode], mode, &items, &n));
    }
    return KG_OK;
}

int launch_lanczos_hpsi(Krylov& K, int j, cudaStream_t st) {
    bool present[4] = {false, false, false, false};
    for (auto& D : K.hdesc) present[D.mode] = true;
    ProfScope ps("lanczos_hpsi", st);
    for (int mode = 0; mode < 4; ++mode) {
        if (!present[mode]) continue;
        const void* kern = mode == 3   ? (const void*)k_lanczos_hpsi<3>
                           : mode == 0 ? (const void*)k_lanczos_hpsi<0>
                           : mode == 1 ? (const void*)k_lanczos_hpsi<1>
                                       : (const void*)k_lanczos_hpsi<2>;
        const int4* items;
        int n;
        KG_TRY(work_list(K, kern, mode, &items, &n));
        switch (mode) {
            case 3: k_lanczos_hpsi<3><<<n, kThreads, 0, st>>>(K.desc, items, K.cs, j, K.cnt); break;
            case 0: k_lanczos_hpsi<0><<<n, kThreads, 0, st>>>(K.desc, items, K.cs, j, K.cnt); break;
            case 1: k_lanczos_hpsi<1><<<n, kThreads, 0, st>>>(K.desc, items, K.cs, j, K.cnt); break;
            default: k_lanczos_hpsi<2><<<n, kThreads, 0, st>>>(K.desc, items, K.cs, j, K.cnt); break;
        }
        KG_LAUNCHED();
    }
    return KG_OK;
}

}  // namespace kg
