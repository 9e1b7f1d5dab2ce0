// kg_hpsi.cu -- a2: the Hamiltonian applied on the fly in the
// occupation-number basis (Section 2, H_jj'; model Hamiltonians of Sections 3
// and 4).  One thread produces one output element y[s], s = i_dn*D_up + i_up:
//
//   y[s] = (e_up[i_up] + e_dn[i_dn] + U(b_up & b_dn)) x[s]
//        + sum_{up hops of i_up}  (+-h_ab) x[i_dn*D_up + j]     (same row)
//        + sum_{down hops of i_dn}(+-h_ab) x[j*D_up + i_up]     (other rows)
//
// Up hops gather inside one row (L1/L2 resident); down hops read whole rows
// at a stride of D_up, so a warp (consecutive i_up, one i_dn) walks the same
// down-hop list and its loads are coalesced.  Fermion signs are applied by
// flipping the IEEE sign bit with integer XOR, and for uniform hopping the
// amplitude multiplies the whole hop sum once, so the FP64 pipe sees one add
// per hop and component.
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

// H x at element (i_dn, i_up); x already loaded as xv.
template <int MODE>
__device__ __forceinline__ double2 hpsi_elem(const SecView& S, const double2* __restrict__ x, int i_dn, int i_up,
                                             double2 xv, const double2* amp, const double* utab) {
    const uint32_t bu = __ldg(S.up_bits + i_up), bd = __ldg(S.dn_bits + i_dn);
    const uint32_t both = bu & bd;
    double diag = __ldg(S.up_e + i_up) + __ldg(S.dn_e + i_dn);
    for (int c = 0; c < S.nchunk; ++c) diag += utab[c * 256 + ((both >> (8 * c)) & 255u)];
    double2 hop = make_double2(0.0, 0.0);
    const double2* row = x + (size_t)i_dn * S.Du;
    const int u0 = __ldg(S.up_off + i_up), u1 = __ldg(S.up_off + i_up + 1);
#pragma unroll 4
    for (int e = u0; e < u1; ++e) {
        const uint2 en = __ldg(S.up_ent + e);
        hop_acc<MODE>(hop, en.y, row[en.x], amp);
    }
    const int d0 = __ldg(S.dn_off + i_dn), d1 = __ldg(S.dn_off + i_dn + 1);
#pragma unroll 4
    for (int e = d0; e < d1; ++e) {
        const uint2 en = __ldg(S.dn_ent + e);
        hop_acc<MODE>(hop, en.y, x[(size_t)en.x * S.Du + i_up], amp);
    }
    if (MODE == 0) {
        return make_double2(fma(diag, xv.x, S.h0 * hop.x), fma(diag, xv.y, S.h0 * hop.y));
    }
    return make_double2(fma(diag, xv.x, hop.x), fma(diag, xv.y, hop.y));
}

__device__ __forceinline__ void stage_tables(const SecView& S, double2* amp, double* utab) {
    for (int k = threadIdx.x; k < S.L * S.L; k += blockDim.x) amp[k] = S.hamp[k];
    for (int k = threadIdx.x; k < S.nchunk * 256; k += blockDim.x) utab[k] = S.Utab[k];
    __syncthreads();
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_hpsi(SecView S, const double2* __restrict__ x,
                                                   double2* __restrict__ y) {
    __shared__ double2 amp[kMaxL * kMaxL];
    __shared__ double utab[4 * 256];
    stage_tables(S, amp, utab);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < S.d; idx += gridDim.x * blockDim.x) {
        int i_dn, i_up;
        split_index(S, idx, i_dn, i_up);
        y[idx] = hpsi_elem<MODE>(S, x, i_dn, i_up, x[idx], amp, utab);
    }
}

// Lanczos step j for column b = blockIdx.y:
//   w = s_j H V_j - b_j s_{j-1} V_{j-1},   a_j = Re <s_j V_j, w>
// (Eq. (recursion) with normalised v_k = s_k V_k).
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_lanczos_hpsi(SecView S, double2* __restrict__ V, size_t colV,
                                                           double2* __restrict__ W, ColScalars* cs, int j,
                                                           double* part, unsigned* cnt, int nblk) {
    __shared__ double2 amp[kMaxL * kMaxL];
    __shared__ double utab[4 * 256];
    __shared__ double sm[(kThreads / 32) * 2];
    __shared__ double bs[2], red[2];
    const int b = blockIdx.y;
    ColScalars* C = cs + b;
    if (j >= C->m_eff) return;
    stage_tables(S, amp, utab);
    const double sj = C->scale[j];
    const double cprev = (j > 0) ? C->beta[j] * C->scale[j - 1] : 0.0;
    const double2* x = V + (size_t)b * colV + (size_t)j * S.d;
    const double2* xp = V + (size_t)b * colV + (size_t)(j > 0 ? j - 1 : 0) * S.d;
    double2* w = W + (size_t)b * S.d;
    double acc[2] = {0.0, 0.0};
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < S.d; idx += gridDim.x * blockDim.x) {
        int i_dn, i_up;
        split_index(S, idx, i_dn, i_up);
        const double2 xv = x[idx];
        double2 r = hpsi_elem<MODE>(S, x, i_dn, i_up, xv, amp, utab);
        r.x *= sj;
        r.y *= sj;
        if (j > 0) {
            const double2 p = xp[idx];
            r.x = fma(-cprev, p.x, r.x);
            r.y = fma(-cprev, p.y, r.y);
        }
        w[idx] = r;
        acc[0] = fma(xv.x, r.x, fma(xv.y, r.y, acc[0]));  // Re conj(x) r
    }
    acc[0] *= sj;
    block_sum<2>(acc, 1, sm, bs);
    if (grid_finish(bs, 1, part + (size_t)b * nblk * kPart, cnt + b, nblk, red)) {
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
    ProfScope ps("hpsi", st);
    switch (S.hopmode) {
        case 0: k_hpsi<0><<<nb, kThreads, 0, st>>>(S, x, y); break;
        case 1: k_hpsi<1><<<nb, kThreads, 0, st>>>(S, x, y); break;
        default: k_hpsi<2><<<nb, kThreads, 0, st>>>(S, x, y); break;
    }
    KG_LAUNCHED();
    return KG_OK;
}

int launch_lanczos_hpsi(const SecView& S, Krylov& K, int j, cudaStream_t st) {
    dim3 grid(K.nblk, K.B);
    ProfScope ps("lanczos_hpsi", st);
    switch (S.hopmode) {
        case 0:
            k_lanczos_hpsi<0><<<grid, kThreads, 0, st>>>(S, K.V, K.colV(), K.W, K.cs, j, K.part, K.cnt, K.nblk);
            break;
        case 1:
            k_lanczos_hpsi<1><<<grid, kThreads, 0, st>>>(S, K.V, K.colV(), K.W, K.cs, j, K.part, K.cnt, K.nblk);
            break;
        default:
            k_lanczos_hpsi<2><<<grid, kThreads, 0, st>>>(S, K.V, K.colV(), K.W, K.cs, j, K.part, K.cnt, K.nblk);
            break;
    }
    KG_LAUNCHED();
    return KG_OK;
}

}  // namespace kg
