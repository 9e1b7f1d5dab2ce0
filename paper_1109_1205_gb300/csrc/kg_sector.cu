// kg_sector.cu -- sector construction (occupation-number basis with N_up and
// N_dn conserved, Section 2 and Section 4 of the paper), the c / c^dag maps
// between neighbouring sectors (Section 3 Eq. (psit), Section 4 step (iii)),
// and small vector utilities.
//
// Spin strings are ranked in the combinatorial number system: the string with
// set bits p_0 < p_1 < ... < p_{N-1} has rank sum_k C(p_k, k+1).  This is the
// position of the string in ascending numeric order among L-bit words of
// popcount N, so the state index s = i_dn * D_up + i_up is the order of the
// full occupation word (down bits above up bits).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <atomic>

#include "kg_internal.h"

namespace kg {

__constant__ uint32_t c_binom[kMaxL + 1][kMaxL + 1];

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    set_error("%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? KG_ENOMEM : KG_ECUDA;
}

static thread_local bool t_capturing = false;
void set_capturing(bool on) { t_capturing = on; }
// launches recorded into a graph are counted when the graph is replayed
void count_launch(unsigned long long n) {
    if (!t_capturing) g_launches += n;
}
unsigned long long launch_count() { return g_launches.load(); }
const char* last_error() { return g_last_error.c_str(); }

static uint64_t host_binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

static int upload_binomials() {
    static std::once_flag once;
    static int status = KG_OK;
    std::call_once(once, [] {
        uint32_t tab[kMaxL + 1][kMaxL + 1];
        for (int n = 0; n <= kMaxL; ++n)
            for (int k = 0; k <= kMaxL; ++k) tab[n][k] = (uint32_t)host_binom(n, k);
        cudaError_t e = cudaMemcpyToSymbol(c_binom, tab, sizeof tab);
        if (e != cudaSuccess) status = cuda_fail(e, "binomial table upload", __FILE__, __LINE__);
    });
    return status;
}

// ----------------------------------------------------------- basis kernels
__device__ __forceinline__ uint32_t rank_string(uint32_t b) {
    uint32_t r = 0;
    int j = 1;
    while (b) {
        const int p = __ffs(b) - 1;
        r += c_binom[p][j];
        ++j;
        b &= b - 1u;
    }
    return r;
}

__device__ __forceinline__ uint32_t unrank_string(uint32_t r, int L, int N) {
    uint32_t b = 0;
    int k = N;
    for (int p = L - 1; p >= 0 && k > 0; --p) {
        const uint32_t c = c_binom[p][k];
        if (r >= c) {
            b |= 1u << p;
            r -= c;
            --k;
        }
    }
    return b;
}

// bits strictly between positions a and b
__device__ __forceinline__ uint32_t between_mask(int a, int b) {
    const int lo = min(a, b), hi = max(a, b);
    const uint32_t below_hi = (hi >= 32) ? 0xffffffffu : ((1u << hi) - 1u);
    const uint32_t upto_lo = (lo >= 31) ? 0xffffffffu : ((2u << lo) - 1u);
    return below_hi & ~upto_lo;
}

__global__ void k_unrank(int L, int N, int D, uint32_t* bits) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < D) bits[i] = unrank_string((uint32_t)i, L, N);
}

// Gather form of the hopping: for target string s, term h_ab c^dag_a c_b
// reaches s from source j = s - a + b when a is occupied and b empty in s.
__global__ void k_hop_count(int L, int D, const uint32_t* bits, const uint32_t* hnz, int* cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    const uint32_t s = bits[i];
    const uint32_t full = (L == 32) ? 0xffffffffu : ((1u << L) - 1u);
    int c = 0;
    for (uint32_t occ = s; occ; occ &= occ - 1u) {
        const int a = __ffs(occ) - 1;
        c += __popc(hnz[a] & ~s & full);
    }
    cnt[i] = c;
}

// Entries of string i: the hops with fermion sign +1 first, then those with
// -1 from split[i] on, so that sign-uniform loops can skip the sign test.
__global__ void k_hop_fill(int L, int D, const uint32_t* bits, const uint32_t* hnz, const int* off,
                           uint2* ent, int* split) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    const uint32_t s = bits[i];
    const uint32_t full = (L == 32) ? 0xffffffffu : ((1u << L) - 1u);
    int e = off[i];
    for (uint32_t want = 0; want < 2; ++want) {
        if (want == 1) split[i] = e;
        for (uint32_t occ = s; occ; occ &= occ - 1u) {
            const int a = __ffs(occ) - 1;
            for (uint32_t emp = hnz[a] & ~s & full; emp; emp &= emp - 1u) {
                const int b = __ffs(emp) - 1;
                const uint32_t neg = __popc(s & between_mask(a, b)) & 1u;
                if (neg != want) continue;
                const uint32_t src = (s & ~(1u << a)) | (1u << b);
                ent[e++] = make_uint2(rank_string(src), (neg << 31) | (uint32_t)(a * L + b));
            }
        }
    }
}

__global__ void k_single_energy(int L, int D, const uint32_t* bits, const double* eps_eff, double* e) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    double acc = 0.0;
    for (uint32_t s = bits[i]; s; s &= s - 1u) acc += eps_eff[__ffs(s) - 1];
    e[i] = acc;
}

static int build_spin(SpinTables& T, int L, int N, const uint32_t* d_hnz, const double* eps_eff_host,
                      cudaStream_t st) {
    T.N = N;
    T.D = (int)host_binom(L, N);
    const int D = T.D, nb = (D + 255) / 256;
    KG_CUDA(cudaMalloc(&T.bits, sizeof(uint32_t) * D));
    KG_CUDA(cudaMalloc(&T.off, sizeof(int) * (D + 1)));
    KG_CUDA(cudaMalloc(&T.e, sizeof(double) * D));
    k_unrank<<<nb, 256, 0, st>>>(L, N, D, T.bits);
    KG_LAUNCHED();
    int* d_cnt = nullptr;
    KG_CUDA(cudaMalloc(&d_cnt, sizeof(int) * D));
    k_hop_count<<<nb, 256, 0, st>>>(L, D, T.bits, d_hnz, d_cnt);
    KG_LAUNCHED();
    std::vector<int> cnt(D), off(D + 1);
    KG_CUDA(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int) * D, cudaMemcpyDeviceToHost, st));
    KG_CUDA(cudaStreamSynchronize(st));
    cudaFree(d_cnt);
    long long acc = 0;
    int mx = 0;
    for (int i = 0; i < D; ++i) {
        off[i] = (int)acc;
        acc += cnt[i];
        mx = cnt[i] > mx ? cnt[i] : mx;
    }
    off[D] = (int)acc;
    if (acc > 0x7fffffffLL) {
        set_error("hop table too large");
        return KG_ENOMEM;
    }
    T.nnz = acc;
    T.max_row = mx;
    KG_CUDA(cudaMemcpyAsync(T.off, off.data(), sizeof(int) * (D + 1), cudaMemcpyHostToDevice, st));
    KG_CUDA(cudaMalloc(&T.ent, sizeof(uint2) * (acc > 0 ? acc : 1)));
    KG_CUDA(cudaMalloc(&T.split, sizeof(int) * D));
    if (acc > 0) {
        k_hop_fill<<<nb, 256, 0, st>>>(L, D, T.bits, d_hnz, T.off, T.ent, T.split);
        KG_LAUNCHED();
    } else {
        KG_CUDA(cudaMemsetAsync(T.split, 0, sizeof(int) * D, st));
    }
    double* d_eps = nullptr;
    KG_CUDA(cudaMalloc(&d_eps, sizeof(double) * L));
    KG_CUDA(cudaMemcpyAsync(d_eps, eps_eff_host, sizeof(double) * L, cudaMemcpyHostToDevice, st));
    k_single_energy<<<nb, 256, 0, st>>>(L, D, T.bits, d_eps, T.e);
    KG_LAUNCHED();
    KG_CUDA(cudaStreamSynchronize(st));
    cudaFree(d_eps);
    return KG_OK;
}

static void free_spin(SpinTables& T) {
    cudaFree(T.bits);
    cudaFree(T.off);
    cudaFree(T.ent);
    cudaFree(T.split);
    cudaFree(T.e);
    T = SpinTables();
}

int sector_build(int L, int nu, int nd, const double* h_re, const double* h_im, const double* eps,
                 const double* U, kg_sector** out) {
    if (!out) {
        set_error("out is NULL");
        return KG_EINVAL;
    }
    *out = nullptr;
    if (L < 1 || L > kMaxL || nu < 0 || nd < 0 || nu > L || nd > L || !h_re || !eps || !U) {
        set_error("invalid sector (L=%d, n_up=%d, n_dn=%d) or NULL parameter array", L, nu, nd);
        return KG_EINVAL;
    }
    for (int k = 0; k < L * L; ++k)
        if (!std::isfinite(h_re[k]) || (h_im && !std::isfinite(h_im[k]))) {
            set_error("hopping element %d is not finite", k);
            return KG_EINVAL;
        }
    for (int k = 0; k < 2 * L; ++k)
        if (!std::isfinite(eps[k]) || (k < L && !std::isfinite(U[k]))) {
            set_error("eps or U element %d is not finite", k);
            return KG_EINVAL;
        }
    double hmax = 0.0;
    for (int k = 0; k < L * L; ++k) hmax = fmax(hmax, fabs(h_re[k]) + (h_im ? fabs(h_im[k]) : 0.0));
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            const double dr = h_re[i * L + j] - h_re[j * L + i];
            const double di = h_im ? h_im[i * L + j] + h_im[j * L + i] : 0.0;
            if (fabs(dr) + fabs(di) > 1e-14 * fmax(1.0, hmax)) {
                set_error("hopping matrix is not Hermitian at (%d,%d)", i, j);
                return KG_EINVAL;
            }
        }
    const long long d = (long long)host_binom(L, nu) * (long long)host_binom(L, nd);
    if (d >= 0x7fffffffLL) {
        set_error("sector dimension %lld exceeds 2^31-1", d);
        return KG_ENOMEM;
    }
    KG_TRY(upload_binomials());

    kg_sector* s = new kg_sector();
    s->L = L;
    s->nu = nu;
    s->nd = nd;
    s->d = d;
    s->h_re.assign(h_re, h_re + L * L);
    s->h_im.assign(L * L, 0.0);
    if (h_im) s->h_im.assign(h_im, h_im + L * L);
    s->eps.assign(eps, eps + 2 * L);
    s->U.assign(U, U + L);
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->device);
    int rc = KG_OK;
    auto fail = [&](int r) {
        sector_free(s);
        return r;
    };
    {
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__));
        e = cudaEventCreateWithFlags(&s->fence, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaEventCreate", __FILE__, __LINE__));
    }
    // hopping classification and tables
    std::vector<uint32_t> hnz(kMaxL, 0u);
    bool any_im = false, uniform = true, first = true;
    double h0 = 0.0;
    for (int a = 0; a < L; ++a)
        for (int b = 0; b < L; ++b) {
            if (a == b) continue;
            const double re = h_re[a * L + b], im = s->h_im[a * L + b];
            if (re == 0.0 && im == 0.0) continue;
            hnz[a] |= 1u << b;
            if (im != 0.0) any_im = true;
            if (first) {
                h0 = re;
                first = false;
            } else if (re != h0) {
                uniform = false;
            }
        }
    s->hopmode = any_im ? 2 : (uniform ? 0 : 1);
    s->h0 = first ? 0.0 : h0;
    std::vector<double2> hamp(L * L);
    for (int k = 0; k < L * L; ++k) hamp[k] = make_double2(h_re[k], s->h_im[k]);
    s->nchunk = (L + 7) / 8;
    std::vector<double> utab(s->nchunk * 256, 0.0);
    for (int c = 0; c < s->nchunk; ++c)
        for (int v = 0; v < 256; ++v) {
            double acc = 0.0;
            for (int t = 0; t < 8; ++t)
                if (((v >> t) & 1) && 8 * c + t < L) acc += U[8 * c + t];
            utab[c * 256 + v] = acc;
        }
    std::vector<double> eps_up(L), eps_dn(L);
    for (int i = 0; i < L; ++i) {
        eps_up[i] = eps[i] + h_re[i * L + i];
        eps_dn[i] = eps[L + i] + h_re[i * L + i];
    }
    uint32_t* d_hnz = nullptr;
    {
        cudaError_t e = cudaMalloc(&d_hnz, sizeof(uint32_t) * kMaxL);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    }
    cudaMemcpy(d_hnz, hnz.data(), sizeof(uint32_t) * kMaxL, cudaMemcpyHostToDevice);
    rc = build_spin(s->up, L, nu, d_hnz, eps_up.data(), s->stream);
    if (rc == KG_OK) rc = build_spin(s->dn, L, nd, d_hnz, eps_dn.data(), s->stream);
    cudaFree(d_hnz);
    if (rc != KG_OK) return fail(rc);
    s->Du = s->up.D;
    s->Dd = s->dn.D;
    if (cudaMalloc(&s->hamp, sizeof(double2) * L * L) != cudaSuccess ||
        cudaMalloc(&s->Utab, sizeof(double) * utab.size()) != cudaSuccess) {
        set_error("device allocation of sector tables failed");
        return fail(KG_ENOMEM);
    }
    cudaMemcpy(s->hamp, hamp.data(), sizeof(double2) * L * L, cudaMemcpyHostToDevice);
    cudaMemcpy(s->Utab, utab.data(), sizeof(double) * utab.size(), cudaMemcpyHostToDevice);
    if (cudaMalloc(&s->diag, sizeof(double) * s->d) != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of the diagonal table failed (%lld states)", s->d);
        return fail(KG_ENOMEM);
    }
    rc = launch_diag_table(s->view(), s->diag, s->stream);
    if (rc == KG_OK && cudaStreamSynchronize(s->stream) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "diagonal table", __FILE__, __LINE__);
    if (rc != KG_OK) return fail(rc);
    *out = s;
    return KG_OK;
}

void sector_free(kg_sector* s) {
    if (!s) return;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) sector_free(s->nb[a][b]);
    free_spin(s->up);
    free_spin(s->dn);
    cudaFree(s->hamp);
    cudaFree(s->Utab);
    cudaFree(s->diag);
    cudaFree(s->gs);
    cudaFree(s->hp_emax);
    cudaFree(s->hp_xf);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->fence) cudaEventDestroy(s->fence);
    delete s;
}

int neighbour(kg_sector* s, int spin, int dagger, kg_sector** out) {
    *out = nullptr;
    if (spin < 0 || spin > 1) {
        set_error("spin must be 0 or 1");
        return KG_EINVAL;
    }
    dagger = dagger ? 1 : 0;
    const int nu = s->nu + (spin == 0 ? (dagger ? 1 : -1) : 0);
    const int nd = s->nd + (spin == 1 ? (dagger ? 1 : -1) : 0);
    if (nu < 0 || nd < 0 || nu > s->L || nd > s->L) {
        set_error("neighbour sector (%d,%d) does not exist", nu, nd);
        return KG_EINVAL;
    }
    if (!s->nb[spin][dagger]) {
        kg_sector* n = nullptr;
        KG_TRY(sector_build(s->L, nu, nd, s->h_re.data(), s->h_im.data(), s->eps.data(), s->U.data(), &n));
        n->is_child = true;
        s->nb[spin][dagger] = n;
    }
    *out = s->nb[spin][dagger];
    return KG_OK;
}

// A caller's stream is used as given.  Without one, work runs on the
// sector's own non-blocking stream (which graphs can capture), ordered after
// everything already queued on the legacy default stream.
cudaStream_t pick_stream(const kg_sector* s, const kg_opts* o) {
    if (o && o->stream) return (cudaStream_t)o->stream;
    cudaEventRecord(s->fence, 0);
    cudaStreamWaitEvent(s->stream, s->fence, 0);
    return s->stream;
}

// --------------------------------------------------------- c / c^dag
// Target-side gather: every element of the destination sector looks up the
// one source element it can come from.
__global__ void k_cop(int L, int site, int spin, int dagger, int nu_src, int Du_dst, int d_dst, int Du_src,
                      const uint32_t* __restrict__ dst_up, const uint32_t* __restrict__ dst_dn,
                      const double2* __restrict__ x, double2* __restrict__ y) {
    const uint32_t bit = 1u << site;
    const uint32_t below = bit - 1u;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d_dst; t += gridDim.x * blockDim.x) {
        const int t_dn = t / Du_dst, t_up = t - t_dn * Du_dst;
        const uint32_t bs = spin == 0 ? __ldg(dst_up + t_up) : __ldg(dst_dn + t_dn);
        const bool present = (bs & bit) != 0u;
        double2 v = make_double2(0.0, 0.0);
        if (present == (dagger != 0)) {
            const uint32_t src = dagger ? (bs & ~bit) : (bs | bit);
            const uint32_t r = rank_string(src);
            unsigned neg = __popc(bs & below) & 1u;
            if (spin == 1) neg ^= (unsigned)(nu_src & 1);
            const size_t si = spin == 0 ? (size_t)t_dn * Du_src + r : (size_t)r * Du_src + t_up;
            v = x[si];
            if (neg) {
                v.x = -v.x;
                v.y = -v.y;
            }
        }
        y[t] = v;
    }
}

int launch_cop(const kg_sector* src, const kg_sector* dst, int site, int spin, int dagger, const double2* x,
               double2* y, cudaStream_t st) {
    const int d = (int)dst->d;
    const int nb = std::min((d + 255) / 256, dst->nsm * 8);
    ProfScope ps("cop", st);
    k_cop<<<nb, 256, 0, st>>>(src->L, site, spin, dagger, src->nu, dst->Du, d, src->Du, dst->up.bits,
                              dst->dn.bits, x, y);
    KG_LAUNCHED();
    return KG_OK;
}

// ------------------------------------------------------------ utilities
// Start vector of the ground-state search: real uniform[-1,1) entries from
// the SplitMix64 generator (Steele, Lea, Flood 2014) keyed by (seed, index).
__global__ void k_random_start(double2* v, int d, unsigned long long seed) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        v[i] = make_double2(2.0 * u - 1.0, 0.0);
    }
}

int launch_random_start(double2* v, int d, unsigned long long seed, cudaStream_t st) {
    k_random_start<<<std::min((d + 255) / 256, 1024), 256, 0, st>>>(v, d, seed);
    KG_LAUNCHED();
    return KG_OK;
}

__global__ void k_scale_copy(double2* dst, const double2* src, int d, double s) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        const double2 v = src[i];
        dst[i] = make_double2(s * v.x, s * v.y);
    }
}

int launch_scale_copy(double2* dst, const double2* src, int d, double s, cudaStream_t st) {
    k_scale_copy<<<std::min((d + 255) / 256, 2048), 256, 0, st>>>(dst, src, d, s);
    KG_LAUNCHED();
    return KG_OK;
}

}  // namespace kg

kg::SecView kg_sector::view() const {
    kg::SecView v;
    v.L = L;
    v.Du = Du;
    v.Dd = Dd;
    v.d = (int)d;
    v.up_bits = up.bits;
    v.dn_bits = dn.bits;
    v.up_off = up.off;
    v.up_ent = up.ent;
    v.up_split = up.split;
    v.dn_split = dn.split;
    v.up_e = up.e;
    v.dn_off = dn.off;
    v.dn_ent = dn.ent;
    v.dn_e = dn.e;
    v.hamp = hamp;
    v.Utab = Utab;
    v.diag = diag;
    v.nchunk = nchunk;
    v.hopmode = hopmode;
    v.h0 = h0;
    {
        // head room for the exact hop sums: the hops of one element plus one
        const int maxhops = up.max_row + dn.max_row;
        int hb = 0;
        while ((1 << hb) < maxhops + 1) ++hb;
        v.fix_pre = 9 - hb;  // negative: no integer hop sums for this sector
    }
    {
        int l = 0;
        while ((1LL << l) < (long long)Du) ++l;
        v.du_l = l;
        v.du_m = (uint32_t)((((unsigned long long)1 << 32) * ((1ULL << l) - (unsigned long long)Du)) / (unsigned long long)Du + 1ULL);
    }
    return v;
}
