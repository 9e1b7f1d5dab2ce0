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

// Hop part of (H x)[i_dn, i_up] from the fixed-point image Xf of x (all
// components on one exponent, written by the kernel that produced x): the
// same signed sums as the on-the-fly path, without the conversions.
__device__ __forceinline__ void hop_sum_pre(const SecView& S, const longlong2* __restrict__ Xf, int i_dn, int i_up,
                                            long long& ix, long long& iy) {
    // each string's hop list holds its +1-sign hops first, then the -1 ones
    const int u0 = __ldg(S.up_off + i_up), us = __ldg(S.up_split + i_up), u1 = __ldg(S.up_off + i_up + 1);
    const int d0 = __ldg(S.dn_off + i_dn), ds = __ldg(S.dn_split + i_dn), d1 = __ldg(S.dn_off + i_dn + 1);
    const longlong2* row = Xf + (size_t)i_dn * S.Du;
    const longlong2* col = Xf + i_up;
    const unsigned* upx = reinterpret_cast<const unsigned*>(S.up_ent);  // .x of entry e at [2e]
    const unsigned* dnx = reinterpret_cast<const unsigned*>(S.dn_ent);
    long long px = 0, py = 0, nx = 0, ny = 0;
#pragma unroll 4
    for (int e = u0; e < us; ++e) {
        const longlong2 v = row[__ldg(upx + 2 * e)];
        px += v.x;
        py += v.y;
    }
#pragma unroll 4
    for (int e = us; e < u1; ++e) {
        const longlong2 v = row[__ldg(upx + 2 * e)];
        nx += v.x;
        ny += v.y;
    }
#pragma unroll 4
    for (int e = d0; e < ds; ++e) {
        const longlong2 v = col[(size_t)__ldg(dnx + 2 * e) * S.Du];
        px += v.x;
        py += v.y;
    }
#pragma unroll 4
    for (int e = ds; e < d1; ++e) {
        const longlong2 v = col[(size_t)__ldg(dnx + 2 * e) * S.Du];
        nx += v.x;
        ny += v.y;
    }
    ix += px - nx;
    iy += py - ny;
}

// v * 2^(E - 1075 - P) rounded to nearest (ties to even), assembled on the
// integer pipe: the FP64 pipe of this GPU is the scarce one.  |v| < 2^62.
// Falls back to FP64 arithmetic if the result would be subnormal.
__device__ __forceinline__ double fix_to_double(long long v, int E, int P) {
    if (v == 0) return 0.0;
    const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ull;
    unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
    const int n = 63 - __clzll((long long)a);  // position of the leading bit
    int be = n + E - 52 - P;                    // biased exponent of the result
    unsigned long long m;
    if (n > 52) {
        const int s = n - 52;
        m = a >> s;
        const unsigned long long rem = a & ((1ull << s) - 1ull), half = 1ull << (s - 1);
        if (rem > half || (rem == half && (m & 1ull))) ++m;
        if (m >> 53) {
            m >>= 1;
            ++be;
        }
    } else {
        m = a << (52 - n);
    }
    if (be < 1) {
        const long long ex = (long long)E - 52 - P;
        return ex > 0 ? __ll2double_rn(v) * __longlong_as_double(ex << 52) : 0.0;
    }
    return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (m & 0xfffffffffffffull)));
}


__device__ __forceinline__ void stage_amplitudes(const SecView& S, double2* amp) {
    for (int k = threadIdx.x; k < S.L * S.L; k += blockDim.x) amp[k] = S.hamp[k];
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_diag_table(SecView S, double* diag) {
    __shared__ double utab[4 * 256];
    for (int k = threadIdx.x; k < S.nchunk * 256; k += blockDim.x) utab[k] = S.Utab[k];
    __syncthreads();
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < S.d; idx += gridDim.x * blockDim.x) {
        int i_dn, i_up;
        split_index(S, idx, i_dn, i_up);
        diag[idx] = diag_energy(S, i_dn, i_up, utab);
    }
}

int launch_diag_table(const SecView& S, double* diag, cudaStream_t st) {
    const int nb = std::max(1, std::min((S.d + kThreads - 1) / kThreads, 148 * 16));
    k_diag_table<<<nb, kThreads, 0, st>>>(S, diag);
    KG_LAUNCHED();
    return KG_OK;
}

// Per-string and per-byte tables of a sector with on-site offsets added:
// e_up'[i] = e_up[i] + sum over the set bits p of string i of dp[p] (spin up),
// e_dn' likewise with dp[L + p], U'[c][v] = U[c][v] + sum over the set bits
// b of byte v of dp[2L + 8c + b].  H is linear in eps and U, so the diagonal
// built from these tables is that of the offset Hamiltonian.
__global__ void k_drive_tables(SecView S, const double* dp, double* e_up, double* e_dn, double* utab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S.Du) {
        double acc = S.up_e[i];
        for (uint32_t b = S.up_bits[i]; b; b &= b - 1u) acc += dp[__ffs(b) - 1];
        e_up[i] = acc;
    }
    if (i < S.Dd) {
        double acc = S.dn_e[i];
        for (uint32_t b = S.dn_bits[i]; b; b &= b - 1u) acc += dp[S.L + __ffs(b) - 1];
        e_dn[i] = acc;
    }
    if (i < S.nchunk * 256) {
        const int c = i >> 8;
        double acc = S.Utab[i];
        for (uint32_t b = (uint32_t)(i & 255); b; b &= b - 1u) {
            const int site = 8 * c + __ffs(b) - 1;
            if (site < S.L) acc += dp[2 * S.L + site];
        }
        utab[i] = acc;
    }
}

size_t drive_work_doubles(const kg_sector* s) {
    return (size_t)s->d + (size_t)s->Du + (size_t)s->Dd + (size_t)s->nchunk * 256;
}

int launch_drive_diag(const SecView& S, const double* dp, double* work, cudaStream_t st) {
    double* e_up = work + S.d;
    double* e_dn = e_up + S.Du;
    double* utab = e_dn + S.Dd;
    const int n = std::max(std::max(S.Du, S.Dd), S.nchunk * 256);
    k_drive_tables<<<(n + 255) / 256, 256, 0, st>>>(S, dp, e_up, e_dn, utab);
    KG_LAUNCHED();
    SecView T = S;
    T.up_e = e_up;
    T.dn_e = e_dn;
    T.Utab = utab;
    return launch_diag_table(T, work, st);
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

// Fixed-point image of x on the exponent *emax (for the exact hop sums).
__global__ void __launch_bounds__(kThreads) k_tofix(const double2* __restrict__ x, int d, const int* emax, int P,
                                                    longlong2* __restrict__ xf) {
    const int E = *emax;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        const double2 v = x[i];
        xf[i] = make_longlong2(fix_term(v.x, E, P, 0u), fix_term(v.y, E, P, 0u));
    }
}

// y = H x with the hop sums read from the fixed-point image xf of x.
__global__ void __launch_bounds__(kThreads) k_hpsi_pre(SecView S, const double2* __restrict__ x,
                                                       const longlong2* __restrict__ xf, double2* __restrict__ y,
                                                       const int* emax) {
    const int E = *emax;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < S.d; idx += gridDim.x * blockDim.x) {
        int i_dn, i_up;
        split_index(S, idx, i_dn, i_up);
        const double2 xv = x[idx];
        const double diag = __ldg(S.diag + idx);
        long long ix = 0, iy = 0;
        hop_sum_pre(S, xf, i_dn, i_up, ix, iy);
        y[idx] = make_double2(fma(diag, xv.x, S.h0 * fix_to_double(ix, E, S.fix_pre)),
                              fma(diag, xv.y, S.h0 * fix_to_double(iy, E, S.fix_pre)));
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_hpsi(SecView S, const double2* __restrict__ x,
                                                   double2* __restrict__ y, const int* emax) {
    __shared__ double2 amp[kMaxL * kMaxL];
    stage_amplitudes(S, amp);
    const int E = (MODE == 3) ? *emax : 0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < S.d; idx += gridDim.x * blockDim.x) {
        int i_dn, i_up;
        split_index(S, idx, i_dn, i_up);
        const double2 xv = x[idx];
        const double diag = __ldg(S.diag + idx);
        double2 hop = make_double2(0.0, 0.0);
        long long ix = 0, iy = 0;
        hop_sum<MODE>(S, x, i_dn, i_up, amp, E, hop, ix, iy);
        double2 r;
        if (MODE == 3) {
            r.x = fma(diag, xv.x, S.h0 * fix_to_double(ix, E, S.fix_pre));
            r.y = fma(diag, xv.y, S.h0 * fix_to_double(iy, E, S.fix_pre));
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
struct HpsiShared {
    double2 amp[kMaxL * kMaxL];
    double sm[(kThreads / 32) * 2];
    int smi[kThreads / 32];
    double bs[2], red[2];
    SecView S;
};

template <int MODE>
__device__ __forceinline__ void lanczos_hpsi_item(const ColDesc* desc, ColScalars* cs, int j, int with_alpha,
                                                  unsigned* cnt, const int4 it_, HpsiShared& sh) {
    const int b = it_.x, blk = it_.y, nblk = it_.z;
    const ColDesc D = desc[b];
    ColScalars* C = cs + b;
    SecView& S = sh.S;
    double2* amp = sh.amp;
    double *sm = sh.sm, *bs = sh.bs, *red = sh.red;
    int* smi = sh.smi;
    if (j >= C->m_eff) return;
    if (threadIdx.x == 0) S = *D.sec;
    __syncthreads();
    stage_amplitudes(S, amp);
    const double sj = C->scale[j];
    const double cprev = (j > 0) ? C->beta[j] * C->scale[j - 1] : 0.0;
    const int E = (MODE == 3) ? C->emax[j] : 0;
    const double hs = S.h0 * sj;
    // V_j in fixed point, written by the update that produced it (not V_0),
    // used when its exponent bound is tight enough
    const int Ef = C->efix;
    const bool pre = MODE == 3 && j > 0 && D.Xf != nullptr && Ef >= E && Ef - E <= kFixSlack;
    const double2* x = D.V + (size_t)j * D.d;
    const double2* xp = D.V + (size_t)(j > 0 ? j - 1 : 0) * D.d;
    const int E0img = C->eimg[0];
    double2* w = D.W;
    double acc[2] = {0.0, 0.0};
    int ew = 0;
    KG_FOR(idx) {
        int i_dn, i_up;
        split_index(S, idx, i_dn, i_up);
        const double2 xv = x[idx];
        const double sdiag = sj * __ldg(S.diag + idx);
        double2 hop = make_double2(0.0, 0.0);
        long long ix = 0, iy = 0;
        const int Eu = pre ? Ef : E;
        if (MODE == 3 && pre)
            hop_sum_pre(S, D.Xf, i_dn, i_up, ix, iy);
        else
            hop_sum<MODE>(S, x, i_dn, i_up, amp, E, hop, ix, iy);
        double2 p = make_double2(0.0, 0.0);
        if (j > 0) p = xp[idx];
        double2 r;
        if (MODE == 3) {
            r.x = fma(sdiag, xv.x, fma(hs, fix_to_double(ix, Eu, S.fix_pre), -cprev * p.x));
            r.y = fma(sdiag, xv.y, fma(hs, fix_to_double(iy, Eu, S.fix_pre), -cprev * p.y));
        } else if (MODE == 0) {
            r.x = fma(sdiag, xv.x, fma(hs, hop.x, -cprev * p.x));
            r.y = fma(sdiag, xv.y, fma(hs, hop.y, -cprev * p.y));
        } else {
            r.x = fma(sdiag, xv.x, fma(sj, hop.x, -cprev * p.x));
            r.y = fma(sdiag, xv.y, fma(sj, hop.y, -cprev * p.y));
        }
        w[idx] = r;
        if (j == 0 && D.I) D.I[idx] = fix_image(xv, E0img);  // image of V_0 for the exact dots
        if (with_alpha) acc[0] = fma(xv.x, r.x, fma(xv.y, r.y, acc[0]));  // Re conj(x) r
        ew = max(ew, max(exp_field(r.x), exp_field(r.y)));
    }
    acc[0] *= sj;
    ew = block_max_int(ew, smi);
    block_sum<2>(acc, 1, sm, bs);
    if (threadIdx.x == 0) bs[1] = (double)ew;
    __syncthreads();
    if (grid_finish(bs, 1, D.part, cnt + b, blk, nblk, red, 1)) {
        if (threadIdx.x == 0) {
            // without with_alpha, a_j = <v_j, w> comes from the exact dots
            // (their coefficient of v_j), which the update adds to alpha[j]
            const double a = with_alpha ? red[0] : 0.0;
            C->alpha[j] = a;
            C->ew = (int)red[1];
            if (!isfinite(a)) {
                C->status = KG_ENUMERIC;
                C->m_eff = j + 1;
            }
        }
    }
}

// One item per block (one-wave work lists, batches of any mix of sizes).
template <int MODE>
__global__ void __launch_bounds__(kThreads, 4) k_lanczos_hpsi(const ColDesc* desc, const int4* items, ColScalars* cs,
                                                           int j, int with_alpha, unsigned* cnt) {
    __shared__ HpsiShared sh;
    lanczos_hpsi_item<MODE>(desc, cs, j, with_alpha, cnt, items[blockIdx.x], sh);
}

int launch_hpsi(kg_sector* s, const double2* x, double2* y, cudaStream_t st) {
    const SecView S = s->view();
    const int nb = std::max(1, std::min((S.d + kThreads - 1) / kThreads, s->nsm * 8));
    if (S.hopmode == 0 && S.fix_pre >= 0) {
        // largest exponent of x, the fixed-point image of x on it, then exact
        // hop sums that add the image's integers.  The scratch belongs to the
        // sector (allocated once, on the first call), so calls with one
        // sector must be ordered, like every use of a handle.
        if (!s->hp_xf) {
            if (cudaMalloc(&s->hp_emax, 256) != cudaSuccess ||
                cudaMalloc(&s->hp_xf, sizeof(longlong2) * (size_t)S.d) != cudaSuccess) {
                cudaGetLastError();
                cudaFree(s->hp_emax);
                s->hp_emax = nullptr;
                s->hp_xf = nullptr;
                set_error("H*psi scratch of %d elements", S.d);
                return KG_ENOMEM;
            }
        }
        ProfScope ps("hpsi", st);
        KG_CUDA(cudaMemsetAsync(s->hp_emax, 0, sizeof(int), st));
        k_maxexp<<<std::min(nb, s->nsm * 4), kThreads, 0, st>>>(x, S.d, s->hp_emax);
        k_tofix<<<nb, kThreads, 0, st>>>(x, S.d, s->hp_emax, S.fix_pre, s->hp_xf);
        k_hpsi_pre<<<nb, kThreads, 0, st>>>(S, x, s->hp_xf, y, s->hp_emax);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch", __FILE__, __LINE__);
        count_launch(3);
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
        for (int g = 0; g < K.ngroups[mode]; ++g) KG_TRY(work_list(K, kerns[mode], mode, &items, &n, g));
    }
    return KG_OK;
}

int launch_lanczos_hpsi(Krylov& K, int j, cudaStream_t st, bool with_alpha) {
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
        // one launch per group of columns whose gathered vectors fit in L2
        for (int g = 0; g < K.ngroups[mode]; ++g) {
            KG_TRY(work_list(K, kern, mode, &items, &n, g));
            switch (mode) {
                case 3: k_lanczos_hpsi<3><<<n, kThreads, 0, st>>>(K.desc, items, K.cs, j, with_alpha ? 1 : 0, K.cnt); break;
                case 0: k_lanczos_hpsi<0><<<n, kThreads, 0, st>>>(K.desc, items, K.cs, j, with_alpha ? 1 : 0, K.cnt); break;
                case 1: k_lanczos_hpsi<1><<<n, kThreads, 0, st>>>(K.desc, items, K.cs, j, with_alpha ? 1 : 0, K.cnt); break;
                default: k_lanczos_hpsi<2><<<n, kThreads, 0, st>>>(K.desc, items, K.cs, j, with_alpha ? 1 : 0, K.cnt); break;
            }
            KG_LAUNCHED();
        }
    }
    return KG_OK;
}

}  // namespace kg
