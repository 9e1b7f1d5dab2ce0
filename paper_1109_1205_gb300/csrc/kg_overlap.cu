// kg_overlap.cu -- overlaps of caller-held vectors: batched inner products
//     G[b][a] = <x_a | y_b> = sum_i conj(x_a[i]) y_b[i]
// the overlaps from which the Green's functions are assembled (Section 3,
// Eq. (psigreen); Section 4, step (iv): G^<(t,t') = i <Psi_a'(t')|Psi_a(t)>).
// One launch covers all n_y columns (blockIdx.y); each block accumulates the
// n_x dot products of its slice in registers, and a deterministic last-block
// reduction over a partial-sum scratch writes G.
#include <algorithm>
#include <map>
#include <mutex>

#include "kg_internal.h"

namespace kg {

template <int NX>
__global__ void __launch_bounds__(kThreads) k_inner(const double2* __restrict__ X, int n_x,
                                                    const double2* __restrict__ Y, int d, double* part,
                                                    unsigned* cnt, int pstride, double2* G, int g_stride) {
    __shared__ double sm[(kThreads / 32) * 2 * NX];
    __shared__ double bs[2 * NX], red[2 * NX];
    const int b = blockIdx.y;
    const double2* y = Y + (size_t)b * d;
    double acc[2 * NX];
#pragma unroll
    for (int k = 0; k < 2 * NX; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        const double2 u = y[i];
#pragma unroll
        for (int a = 0; a < NX; ++a) {
            if (a < n_x) {
                const double2 v = X[(size_t)a * d + i];
                acc[2 * a] = fma(v.x, u.x, fma(v.y, u.y, acc[2 * a]));
                acc[2 * a + 1] = fma(v.x, u.y, fma(-v.y, u.x, acc[2 * a + 1]));
            }
        }
    }
    block_sum<2 * NX>(acc, 2 * n_x, sm, bs);
    if (grid_finish(bs, 2 * n_x, part + (size_t)b * pstride, cnt + b, blockIdx.x, gridDim.x, red)) {
        for (int a = threadIdx.x; a < n_x; a += blockDim.x)
            G[(size_t)b * g_stride + a] = make_double2(red[2 * a], red[2 * a + 1]);
    }
}

// Launches k_inner with `per_col` blocks per column over the given scratch
// (partials: n_y rows of per_col*kPart doubles; counters: n_y, all zero).
static int launch_inner(const double2* X, int n_x, const double2* Y, int n_y, int d, int per_col, double* part,
                        unsigned* cnt, double2* G, int g_stride, cudaStream_t st) {
    ProfScope ps("inner", st);
    const dim3 grid(per_col, n_y);
    const int pst = per_col * kPart;
    if (n_x <= 4)
        k_inner<4><<<grid, kThreads, 0, st>>>(X, n_x, Y, d, part, cnt, pst, G, g_stride);
    else if (n_x <= 8)
        k_inner<8><<<grid, kThreads, 0, st>>>(X, n_x, Y, d, part, cnt, pst, G, g_stride);
    else if (n_x <= 16)
        k_inner<16><<<grid, kThreads, 0, st>>>(X, n_x, Y, d, part, cnt, pst, G, g_stride);
    else
        k_inner<32><<<grid, kThreads, 0, st>>>(X, n_x, Y, d, part, cnt, pst, G, g_stride);
    KG_LAUNCHED();
    return KG_OK;
}

static int check_inner_args(const void* X, int n_x, const void* Y, int n_y, long long d, const void* G) {
    if (!X || !Y || !G || n_x < 1 || n_x > kMaxOv || n_y < 1 || d < 1 || d >= 0x7fffffffLL) {
        set_error("kg_overlaps: need 1 <= n_x <= %d, n_y >= 1, 1 <= d < 2^31 and non-NULL pointers", kMaxOv);
        return KG_EINVAL;
    }
    return KG_OK;
}

static int blocks_per_column(int n_y, long long d) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int want = std::max(1, (nsm * 4) / n_y);
    return (int)std::max(1LL, std::min<long long>(want, (d + kThreads - 1) / kThreads));
}

// Library-owned scratch for kg_overlaps, one grow-only buffer per device.
struct InnerScratch {
    double* part = nullptr;
    unsigned* cnt = nullptr;
    size_t part_len = 0, cnt_len = 0;
};

static int inner_scratch(int dev, size_t part_len, size_t cnt_len, InnerScratch** out) {
    static std::mutex mu;
    static std::map<int, InnerScratch> bufs;
    std::lock_guard<std::mutex> lk(mu);
    InnerScratch& s = bufs[dev];
    if (s.part_len < part_len) {
        cudaFree(s.part);
        s.part = nullptr;
        s.part_len = 0;
        KG_CUDA(cudaMalloc(&s.part, sizeof(double) * part_len));
        s.part_len = part_len;
    }
    if (s.cnt_len < cnt_len) {
        cudaFree(s.cnt);
        s.cnt = nullptr;
        s.cnt_len = 0;
        KG_CUDA(cudaMalloc(&s.cnt, sizeof(unsigned) * cnt_len));
        KG_CUDA(cudaMemset(s.cnt, 0, sizeof(unsigned) * cnt_len));
        s.cnt_len = cnt_len;
    }
    *out = &s;
    return KG_OK;
}

int launch_inner_lib(const double2* X, int n_x, const double2* Y, int n_y, int d, double2* G, int g_stride,
                     cudaStream_t st) {
    KG_TRY(check_inner_args(X, n_x, Y, n_y, d, G));
    const int per_col = blocks_per_column(n_y, d);
    int dev = 0;
    KG_CUDA(cudaGetDevice(&dev));
    InnerScratch* s = nullptr;
    KG_TRY(inner_scratch(dev, (size_t)n_y * per_col * kPart, (size_t)n_y, &s));
    return launch_inner(X, n_x, Y, n_y, d, per_col, s->part, s->cnt, G, g_stride, st);
}

}  // namespace kg

extern "C" int kg_overlaps(const double* X_dev, int n_x, const double* Y_dev, int n_y, long long d, double* G_dev,
                           void* stream) {
    using namespace kg;
    return launch_inner_lib(reinterpret_cast<const double2*>(X_dev), n_x, reinterpret_cast<const double2*>(Y_dev), n_y,
                            (int)d, reinterpret_cast<double2*>(G_dev), n_x, (cudaStream_t)stream);
}

// ------------------------------------------- no-allocation variant
// Some callers cannot allocate device memory at call time: code under a fixed
// device-memory budget or with a memory pool that must not grow, and code
// that must not hit the allocator's implicit synchronisation.  kg_overlaps_noalloc serves them with
// the same kernel as kg_overlaps, its partial sums and tickets held in fixed
// arrays of this library's device image instead of allocated memory.
namespace kg {

constexpr int kNoAllocCols = 64;    // largest n_y accepted
constexpr int kNoAllocRows = 2048;  // partial-sum rows of kPart doubles (1,179,648 bytes)

static __device__ __align__(256) double g_noalloc_part[kNoAllocRows * kPart];
static __device__ __align__(256) unsigned g_noalloc_cnt[kNoAllocCols];

// Device addresses of the arrays on one device.  In host code the symbols are
// host-side stand-ins, so the addresses come from cudaGetSymbolAddress, once
// per device, with that device current.
struct NoAllocPtrs {
    double* part = nullptr;
    unsigned* cnt = nullptr;
};

static int noalloc_ptrs(NoAllocPtrs* out) {
    static std::mutex mu;
    static std::map<int, NoAllocPtrs> cache;
    int dev = 0;
    KG_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it == cache.end()) {
        NoAllocPtrs p;
        KG_CUDA(cudaGetSymbolAddress((void**)&p.part, g_noalloc_part));
        KG_CUDA(cudaGetSymbolAddress((void**)&p.cnt, g_noalloc_cnt));
        it = cache.emplace(dev, p).first;
    }
    *out = it->second;
    return KG_OK;
}

// The tickets must start at zero; device code names the array directly.
__global__ void k_noalloc_clear() {
    for (int i = threadIdx.x; i < kNoAllocCols; i += blockDim.x) g_noalloc_cnt[i] = 0u;
}

}  // namespace kg

extern "C" int kg_overlaps_noalloc(const double* X_dev, int n_x, const double* Y_dev, int n_y, long long d,
                                   double* G_dev, void* stream) {
    using namespace kg;
    KG_TRY(check_inner_args(X_dev, n_x, Y_dev, n_y, d, G_dev));
    if (n_y > kNoAllocCols) {
        set_error("kg_overlaps_noalloc: n_y = %d exceeds its fixed scratch limit of %d columns", n_y, kNoAllocCols);
        return KG_EINVAL;
    }
    NoAllocPtrs p;
    KG_TRY(noalloc_ptrs(&p));
    const int per_col = std::min(blocks_per_column(n_y, d), kNoAllocRows / n_y);
    cudaStream_t st = (cudaStream_t)stream;
    k_noalloc_clear<<<1, kNoAllocCols, 0, st>>>();
    KG_LAUNCHED();
    return launch_inner(reinterpret_cast<const double2*>(X_dev), n_x, reinterpret_cast<const double2*>(Y_dev), n_y,
                        (int)d, per_col, p.part, p.cnt, reinterpret_cast<double2*>(G_dev), n_x, st);
}
