// kg_fourier.cu -- the frequency-dependent Green's function from the
// time-dependent one (Section 3: G(omega) by Fourier transformation of G(t),
// the Lorentzian broadening eta entering as the damping e^{-eta t} that makes
// the time integral converge at t_max).  For samples t_k = k dt, k < n_t:
//
//   G(omega_j) = sum_k w_k e^{i (omega_j + i eta) t_k} G(t_k),
//   w_0 = w_{n_t-1} = dt/2, w_k = dt otherwise,
//
// the trapezoidal rule for the integral over [0, (n_t - 1) dt]; zero for one
// sample.  Transforming the particle part G^>(t) gives the particle part of
// Eq. (gomega), transforming -G^<(t) the hole part.
//
// The transform is evaluated directly on the caller's frequency grid: one
// thread per frequency, the samples of one series staged in shared memory
// (every thread reads the same sample: a broadcast), and within each chunk of
// kFtChunk samples a Horner recurrence in z = e^{i (omega + i eta) dt},
//   S = g_0 + z (g_1 + z (g_2 + ...)),
// four FP64 FMAs per sample and frequency.  Each chunk is rotated into place
// by e^{i (omega + i eta) t_c}, computed from sincos/exp at the chunk start,
// so rounding does not build up over long series.  Long series are split
// over blockIdx.z to fill the GPU; a second kernel sums the splits in a fixed
// order (deterministic).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kg_internal.h"

namespace kg {

constexpr int kFtThreads = 128;  // frequencies per block, one per thread
constexpr int kFtTile = 512;     // samples staged in shared memory per pass
constexpr int kFtChunk = 128;    // samples per Horner chunk (one rotation each)
constexpr int kFtMaxSeries = 65535;
constexpr long long kFtMaxSamples = 1ll << 30;

__global__ void __launch_bounds__(kFtThreads) k_fourier(const double2* __restrict__ Gt, int n_t, double dt,
                                                        const double* __restrict__ omega, int n_omega, double eta,
                                                        int tiles_per_split, double2* __restrict__ out) {
    __shared__ double2 g[kFtTile];
    const int j = blockIdx.x * kFtThreads + threadIdx.x;
    const int series = blockIdx.y, split = blockIdx.z;
    const double2* G = Gt + (size_t)series * n_t;
    const double w = j < n_omega ? omega[j] : 0.0;
    double s1, c1;
    sincos(w * dt, &s1, &c1);
    const double r1 = exp(-eta * dt);
    const double zr = r1 * c1, zi = r1 * s1;
    double ar = 0.0, ai = 0.0;
    const int k_begin = split * tiles_per_split * kFtTile;
    const long long k_lim = (long long)k_begin + (long long)tiles_per_split * kFtTile;
    const int k_end = k_lim < n_t ? (int)k_lim : n_t;
    for (int k0 = k_begin; k0 < k_end; k0 += kFtTile) {
        const int len = k_end - k0 < kFtTile ? k_end - k0 : kFtTile;
        __syncthreads();  // the previous tile is consumed
        for (int q = threadIdx.x; q < len; q += kFtThreads) {
            const int k = k0 + q;
            const double wk = (k == 0 || k == n_t - 1) ? 0.5 * dt : dt;
            const double2 v = G[k];
            g[q] = make_double2(wk * v.x, wk * v.y);
        }
        __syncthreads();
        for (int c0 = 0; c0 < len; c0 += kFtChunk) {
            const int cl = len - c0 < kFtChunk ? len - c0 : kFtChunk;
            double sr = 0.0, si = 0.0;
            if (cl == kFtChunk) {
#pragma unroll 16
                for (int q = kFtChunk - 1; q >= 0; --q) {
                    const double2 v = g[c0 + q];
                    const double nr = fma(zr, sr, fma(-zi, si, v.x));
                    const double ni = fma(zr, si, fma(zi, sr, v.y));
                    sr = nr;
                    si = ni;
                }
            } else {
                for (int q = cl - 1; q >= 0; --q) {
                    const double2 v = g[c0 + q];
                    const double nr = fma(zr, sr, fma(-zi, si, v.x));
                    const double ni = fma(zr, si, fma(zi, sr, v.y));
                    sr = nr;
                    si = ni;
                }
            }
            // rotate the chunk to its start time t_c
            const double tc = (double)(k0 + c0) * dt;
            double sa, ca;
            sincos(w * tc, &sa, &ca);
            const double ra = exp(-eta * tc);
            const double pr = ra * ca, pi = ra * sa;
            ar = fma(pr, sr, fma(-pi, si, ar));
            ai = fma(pr, si, fma(pi, sr, ai));
        }
    }
    if (j < n_omega) out[((size_t)split * gridDim.y + series) * n_omega + j] = make_double2(ar, ai);
}

// out[i] = sum over the n_split partial planes of part[s][i], in split order.
__global__ void __launch_bounds__(kThreads) k_fourier_sum(const double2* __restrict__ part, int n_split,
                                                          long long plane, double2* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane;
         i += (long long)gridDim.x * blockDim.x) {
        double r = 0.0, im = 0.0;
        for (int s = 0; s < n_split; ++s) {
            const double2 v = part[(size_t)s * plane + i];
            r += v.x;
            im += v.y;
        }
        out[i] = make_double2(r, im);
    }
}

static int fourier_args(const double* G_t, int n_series, int n_t, double dt, const double* omega, int n_omega,
                        double eta, const double* G_w) {
    if (n_series < 0 || n_series > kFtMaxSeries || n_t < 1 || n_t > kFtMaxSamples || n_omega < 0 ||
        !(dt > 0.0) || !std::isfinite(dt) || !(eta >= 0.0) || !std::isfinite(eta)) {
        set_error("kg_green_fourier: need 0 <= n_series <= %d, 1 <= n_t <= 2^30, n_omega >= 0, finite dt > 0 and "
                  "finite eta >= 0", kFtMaxSeries);
        return KG_EINVAL;
    }
    if (n_series > 0 && n_omega > 0) {
        if (!G_t || !omega || !G_w) {
            set_error("kg_green_fourier: NULL buffer");
            return KG_EINVAL;
        }
        for (int j = 0; j < n_omega; ++j)
            if (!std::isfinite(omega[j])) {
                set_error("kg_green_fourier: omega[%d] is not finite", j);
                return KG_EINVAL;
            }
    }
    return KG_OK;
}

static int green_fourier(const double* G_t, int n_series, int n_t, double dt, const double* omega, int n_omega,
                         double eta, cudaStream_t st, double* G_w) {
    KG_TRY(fourier_args(G_t, n_series, n_t, dt, omega, n_omega, eta, G_w));
    if (n_series == 0 || n_omega == 0) return KG_OK;
    const long long plane = (long long)n_series * n_omega;
    if (n_t == 1) {  // the integral over an empty interval
        std::memset(G_w, 0, sizeof(double2) * (size_t)plane);
        return KG_OK;
    }
    int dev = 0, nsm = 148;
    KG_CUDA(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int n_wtiles = (n_omega + kFtThreads - 1) / kFtThreads;
    const int n_tiles = (int)((n_t + kFtTile - 1) / kFtTile);
    const long long base = (long long)n_wtiles * n_series;
    // Split count: the resident blocks of an SM share its FP64 pipe, so an
    // SM's time is the number of tiles its blocks hold, and the launch ends
    // with the busiest SM, ceil(blocks / nsm) blocks of tiles_per_split tiles
    // (plus a small per-block cost).  Take the split count that minimises
    // this, the fewest splits among equals, over at most a few waves, with at
    // least 4 blocks (16 warps) per SM where the series is long enough: the
    // Horner chains need that many warps to keep the FP64 pipe busy.
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fourier, kFtThreads, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long long max_split = std::max(1LL, std::min<long long>(n_tiles, 4LL * per_sm * nsm / base + 1));
    const long long min_split = std::min(max_split, (4LL * nsm + base - 1) / base);
    int n_split = 1, tiles_per_split = n_tiles;
    double best = -1.0;
    for (int pass = 0; pass < 2 && best < 0.0; ++pass)
        for (long long ns = pass == 0 ? min_split : 1; ns <= max_split; ++ns) {
            const int tps = (int)((n_tiles + ns - 1) / ns);
            if ((n_tiles + tps - 1) / tps != ns) continue;  // would leave a split empty
            const long long busiest = (base * ns + nsm - 1) / nsm;
            const double cost = (double)busiest * (tps + 0.05);
            if (best < 0.0 || cost < best) {
                best = cost;
                n_split = (int)ns;
                tiles_per_split = tps;
            }
        }

    // device copies: the series, the frequencies, the partial planes, the result
    const size_t b_gt = sizeof(double2) * (size_t)n_series * n_t;
    const size_t b_om = (sizeof(double) * (size_t)n_omega + 255) & ~(size_t)255;
    const size_t b_out = sizeof(double2) * (size_t)plane;
    const size_t b_part = n_split > 1 ? b_out * n_split : 0;
    const size_t o_om = (b_gt + 255) & ~(size_t)255, o_out = o_om + b_om, o_part = o_out + ((b_out + 255) & ~(size_t)255);
    char* buf = nullptr;
    if (cudaMallocAsync((void**)&buf, o_part + b_part, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("kg_green_fourier: cannot allocate %zu bytes on the device", o_part + b_part);
        return KG_ENOMEM;
    }
    const double2* d_gt = reinterpret_cast<const double2*>(buf);
    const double* d_om = reinterpret_cast<const double*>(buf + o_om);
    double2* d_out = reinterpret_cast<double2*>(buf + o_out);
    double2* d_part = n_split > 1 ? reinterpret_cast<double2*>(buf + o_part) : d_out;
    int rc = KG_OK;
    cudaError_t e = cudaMemcpyAsync(buf, G_t, b_gt, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf + o_om, omega, sizeof(double) * n_omega, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "kg_green_fourier: copy in", __FILE__, __LINE__);
    if (rc == KG_OK) {
        ProfScope ps("fourier", st);
        k_fourier<<<dim3(n_wtiles, n_series, n_split), kFtThreads, 0, st>>>(d_gt, n_t, dt, d_om, n_omega, eta,
                                                                           tiles_per_split, d_part);
        int launched = 1;
        if (n_split > 1) {
            const int nb = (int)std::max(1LL, std::min<long long>((plane + kThreads - 1) / kThreads, 4LL * nsm));
            k_fourier_sum<<<nb, kThreads, 0, st>>>(d_part, n_split, plane, d_out);
            launched = 2;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "kernel launch", __FILE__, __LINE__);
        else count_launch(launched);
    }
    if (rc == KG_OK) {
        e = cudaMemcpyAsync(G_w, d_out, b_out, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "kg_green_fourier: copy out", __FILE__, __LINE__);
    }
    cudaFreeAsync(buf, st);
    e = cudaStreamSynchronize(st);
    if (rc == KG_OK && e != cudaSuccess) rc = cuda_fail(e, "kg_green_fourier", __FILE__, __LINE__);
    return rc;
}

}  // namespace kg

extern "C" int kg_green_fourier(const double* G_t, int n_series, int n_t, double dt, const double* omega,
                                int n_omega, double eta, void* stream, double* G_w) {
    return kg::green_fourier(G_t, n_series, n_t, dt, omega, n_omega, eta, (cudaStream_t)stream, G_w);
}
