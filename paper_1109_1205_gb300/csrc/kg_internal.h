// kg_internal.h -- shared declarations of the CUDA implementation of
// libkrylovgf (not part of the public ABI; see include/krylovgf.h).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "krylovgf.h"

namespace kg {

constexpr int kMaxL = 32;      // spin strings are 32-bit words
constexpr int kMaxM = 64;      // Krylov dimension of one propagation step
constexpr int kMaxMgs = 256;   // Krylov dimension of one ground-state restart
constexpr int kChunk = 24;     // complex dot products accumulated per pass
constexpr int kMaxOv = 32;     // overlap vectors fused into the combination pass
constexpr int kPart = 72;      // doubles per block in a partial-sum row
constexpr int kThreads = 256;  // threads per block of the streaming kernels
constexpr int kMaxSub = 1 << 17;  // largest sub-step count of a step exponential
// H*psi gathers each input component about once per hop; a launch covers a
// group of columns whose inputs together fit in this much L2 (of 129 MB).
constexpr long long kHpsiGroupBytes = 72ll << 20;

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
void count_launch(unsigned long long n = 1);

#define KG_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return kg::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define KG_LAUNCHED()                                                   \
    do {                                                                \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return kg::cuda_fail(e_, "kernel launch", __FILE__, __LINE__); \
        kg::count_launch();                                             \
    } while (0)

#define KG_TRY(call)                        \
    do {                                    \
        int r_ = (call);                    \
        if (r_ != KG_OK) return r_;         \
    } while (0)

// ------------------------------------------------------- sector (device)
// One spin species: the D strings with N of L bits set, in rank order, and
// the CSR list of allowed hops.  For string s, entry e = (j, code) says that
// h_ab c^dag_a c_b maps string j onto s, a = (code & 1023) / L, b = code % L
// (within the low 10 bits), with fermion sign (-1)^(code >> 31).
struct SpinTables {
    int D = 0, N = 0;
    long long nnz = 0;
    int max_row = 0;
    uint32_t* bits = nullptr;  // [D]
    int* off = nullptr;        // [D + 1]
    uint2* ent = nullptr;      // [nnz], per string the +1-sign hops first
    int* split = nullptr;      // [D] first entry of string i with sign -1
    double* e = nullptr;       // [D]  sum over occupied i of (eps_i + h_ii)
};

// Read-only view of a sector, passed by value to kernels.
struct SecView {
    int L, Du, Dd, d;
    const uint32_t* up_bits;
    const uint32_t* dn_bits;
    const int* up_off;
    const uint2* up_ent;
    const int* up_split;  // first entry of each string's -1-sign hops
    const int* dn_split;
    const double* up_e;
    const int* dn_off;
    const uint2* dn_ent;
    const double* dn_e;
    const double2* hamp;  // [L*L] hopping amplitudes h_ab
    const double* Utab;   // [nchunk * 256] U summed over the set bits of a byte
    const double* diag;   // [d] diagonal of H (eps, h_ii and U terms) per state
    int nchunk;
    int hopmode;          // 0: all hops share the real amplitude h0; 1: real; 2: complex
    double h0;
    int fix_pre;          // P: left pre-shift of fixed-point hop terms (9 - headroom bits)
    uint32_t du_m;        // s / D_up = (umulhi(s, du_m) + s) >> du_l   (s < 2^31)
    int du_l;
};

}  // namespace kg

struct kg_sector {
    int L = 0, nu = 0, nd = 0;
    int Du = 0, Dd = 0;
    long long d = 0;
    std::vector<double> h_re, h_im, eps, U;
    int hopmode = 1;
    double h0 = 0.0;
    kg::SpinTables up, dn;
    double2* hamp = nullptr;
    double* Utab = nullptr;
    double* diag = nullptr;  // [d] diagonal of H
    int nchunk = 1;
    kg_sector* nb[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [spin][dagger]
    bool is_child = false;
    cudaStream_t stream = nullptr;   // the library's own stream (graph capture)
    cudaEvent_t fence = nullptr;     // orders it after the legacy default stream
    int device = 0;
    int nsm = 148;
    bool has_gs = false;
    double E0 = 0.0, resid = 0.0, gap = 0.0;
    double2* gs = nullptr;  // [d] cached ground state (unit norm)
    // scratch of the standalone H*psi (exact hop sums): the largest exponent
    // and the fixed-point image of the input, allocated on first use
    int* hp_emax = nullptr;
    longlong2* hp_xf = nullptr;
    kg::SecView view() const;
};

namespace kg {

// --------------------------------------------------- Krylov workspace
// Per-column scalars of the Lanczos recursion, Eq. (recursion), kept on the
// device so that a whole propagation step runs without a host round trip.
struct ColScalars {
    double alpha[kMaxMgs];      // a_k (diagonal of T)
    double beta[kMaxMgs + 1];   // b_k (beta[k] couples vectors k-1 and k)
    double scale[kMaxMgs + 1];  // 1/||V_k||: stored Lanczos vectors are unnormalised
    double2 h[kMaxMgs + 1];     // Gram-Schmidt coefficients of the current pass
    double2 c[kMaxMgs];         // combination coefficients (already times scale)
    int emax[kMaxMgs + 1];      // largest biased FP64 exponent among the components of V_k
    int eimg[kMaxMgs + 1];      // exponent bound of the fixed-point image I_k (exact dots)
    double beta0;               // norm of the start vector
    double lam0, lam1, resest;  // ground-state Ritz value, next one, residual estimate
    double rq, rnorm;           // Rayleigh quotient and residual of a Ritz vector
    double ovnorm;              // norm of the last combined vector
    int m_eff;                  // Krylov dimension reached (smaller after a breakdown)
    int status;                 // KG_OK, KG_ENUMERIC or KG_ENOCONV
    int ov_slot;                // overlap rows written so far
    int ew;                     // largest exponent field of the last H*psi output W
    int efix;                   // exponent of the fixed-point image Xf of the newest V_k
    int pad;
};

// One column of a Krylov batch.  Columns are independent vectors, each with
// its own sector (dimension, tables), its own Lanczos basis and step tau;
// the device copy is read by every kernel of a step.
struct ColDesc {
    const SecView* sec;     // this column's sector (device copy)
    double2* V;             // [M+1][d] Lanczos vectors (unnormalised)
    double* S;              // [M+1][d] Re + Im of each component of V_k (or null)
    float2* V32;            // [M+1][d] V_k truncated to FP32 (or null)
    int4* I;                // [M+1][d] V_k in 52-bit fixed point on eimg[k], split
                            // into 26-bit halves {x_hi, x_lo, y_hi, y_lo} (or null)
    longlong2* Xf;          // [d] fixed-point image of the next H*psi input (or null)
    double2* W;             // [d] H v workspace
    double2* U;             // [d] W - a_j v_j, left by the Gram-Schmidt dots
    double* part;           // [nblk_max][kPart] partial sums of this column
    double2* out;           // where the combination writes (V_0 by default)
    const double2* ov;      // n_ov overlap vectors, stride ov_stride
    double2* ov_out;        // overlap rows [ov_rows][n_ov]
    long long ov_stride;
    double tau;             // propagation step of this column
    int d, n_ov, ov_rows, nblk_max;
    int mode;               // hop sums: 0 FP64 uniform, 1 real, 2 complex, 3 exact integer
    int Du, Dd, fix_pre;    // row length, row count, fixed-point pre-shift of the sector
    int pad;
};

// B columns of (possibly) different sectors.  Every streaming kernel runs over
// a work list of (column, block, blocks of that column) items sized from the
// kernel's occupancy and each column's dimension, so that one launch of a
// phase covers every column of the batch in about one wave.
struct Krylov {
    int B = 0, M = 0, nsm = 148;
    int schedule = 0;               // kg_opts.schedule bits (hop sums, step exponential)
    long long total_d = 0;
    double wave_scale = 1.0;        // work-list size relative to one wave (tuned)
    std::vector<ColDesc> hdesc;     // host copy (device addresses)
    std::vector<SecView> hsec;
    ColDesc* desc = nullptr;        // [B]
    SecView* secs = nullptr;        // [B]
    ColScalars* cs = nullptr;       // [B]
    unsigned* cnt = nullptr;        // [B]
    double* Q = nullptr;            // [B][M*M] eigenvectors of T
    double2* Vbuf = nullptr;
    double* Sbuf = nullptr;         // planes of the Gram-Schmidt kernels (optional)
    float2* V32buf = nullptr;
    int4* Ibuf = nullptr;           // fixed-point images of the exact Gram-Schmidt dots
    longlong2* Xfbuf = nullptr;     // fixed-point H*psi inputs of exact-integer columns
    double2* Wbuf = nullptr;
    double* partbuf = nullptr;
    std::map<long long, std::pair<int4*, int>> lists;
    std::vector<int> group;         // H*psi launch group of each column (per mode)
    int ngroups[4] = {0, 0, 0, 0};  // groups per hop-sum mode
    double2* vec(int b, int k) const { return hdesc[b].V + (size_t)k * hdesc[b].d; }
    int dim(int b) const { return hdesc[b].d; }
};

// One column per entry of `cols` (sectors may repeat).  schedule: the
// kg_opts.schedule bits (bit 0: FP64 hop sums instead of the exact integer
// sums for sectors with uniform hopping; bit 1: step exponential through the
// eigen-decomposition of T instead of the Taylor series).
// planes = false leaves out the optional Gram-Schmidt planes (S, V32).
int krylov_alloc(Krylov& K, const std::vector<const kg_sector*>& cols, int M, int nsm, int schedule,
                 bool planes = true);
// Device bytes krylov_alloc takes for these columns (an upper estimate).
size_t krylov_bytes(const std::vector<const kg_sector*>& cols, int M, bool planes, int schedule = 0);
int krylov_upload(Krylov& K, cudaStream_t st);  // after editing hdesc (tau, out, overlaps)
void krylov_free(Krylov& K);
int work_list(Krylov& K, const void* kern, int mode, const int4** items, int* n, int group = -1);

// ----------------------------------------------------------- launchers
// y = H x (plain); exact-hop-sum sectors use the sector's own scratch.
int launch_hpsi(kg_sector* s, const double2* x, double2* y, cudaStream_t st);
// Lanczos H*psi: w = s_j H V_j - b_j s_{j-1} V_{j-1} for every column, with the
// partial sums of a_j = <v_j, w> reduced on the device.
// with_alpha = false leaves a_j to the exact Gram-Schmidt dots (alpha_in_dots).
int launch_lanczos_hpsi(Krylov& K, int j, cudaStream_t st, bool with_alpha = true);
// True when the first Gram-Schmidt pass of level `reorth` runs the exact
// integer dots, which then also give a_j = <v_j, w> (their coefficient of
// v_j): H*psi skips its FP64 dot and the update subtracts a_j v_j.
bool alpha_in_dots(const Krylov& K, int reorth);
// start of a step: beta0 = ||V_0||, scale[0], largest exponent, m_eff = M.
int launch_colnorm(Krylov& K, cudaStream_t st);
// Reorthogonalisation: h_k = <v_k, w - a_j v_j> (first pass) or
// h_k = <v_k, V_{j+1}> (second pass) for k in [k0, k0 + nk).
int launch_reorth_dots(Krylov& K, int j, int k0, int nk, bool second, cudaStream_t st);
// Lanczos update: V_{j+1} = w - a_j v_j - sum_k h_k v_k (or in place for the
// second pass), then b_{j+1} = ||V_{j+1}||, scale, breakdown test.
// The Lanczos space (colnorm, then M iterations of H*psi, Gram-Schmidt and
// update) of every column's V_0, without the combination step.
int build_space(Krylov& K, int reorth, cudaStream_t st);
// level: the reorthogonalisation level (0, 1, 2); second: the second pass.
// diag[s] = e_up[i_up] + e_dn[i_dn] + sum of U over doubly occupied sites.
int launch_diag_table(const SecView& S, double* diag, cudaStream_t st);
// Driven Hamiltonians: work = [d] diagonal, then scratch tables (in doubles,
// drive_work_doubles of them).  launch_drive_diag writes into work[0, d) the
// diagonal of H with the on-site offsets dp = [eps_up (L), eps_dn (L), U (L)]
// (device) added to the sector's eps and U.
size_t drive_work_doubles(const kg_sector* s);
int launch_drive_diag(const SecView& S, const double* dp, double* work, cudaStream_t st);
// Points every column's sector view at `diag` (device, [d] of its sector),
// before a StepRunner is initialised for K.
int krylov_set_diag(Krylov& K, const double* diag);
int launch_update(Krylov& K, int j, int level, bool second, cudaStream_t st);
// Tridiagonal step: T = Q D Q^T on the device; mode 0: c = beta0 Q e^{-i D tau} Q^T e_1
// with each column's tau; mode 1: ground-state Ritz pair (lam0, c = q_0).
int launch_tridiag(Krylov& K, int mode, cudaStream_t st);
// The same for several times at once: cq[b][t][k] = coefficients of
// exp(-i H taus[b][t]) v_0 in the stored basis (adjoint quadrature nodes).
int launch_tridiag_multi(Krylov& K, const double* taus, int ntau, double2* cq, cudaStream_t st);
// Combination and overlaps: out = sum_k c_k V_k per column; ||out||; overlaps <ov_a, out>.
int launch_combine(Krylov& K, cudaStream_t st);
// Overlaps: G[b*g_stride + a] = <x_a | y_b> (kg_overlap.cu), library scratch.
int launch_inner_lib(const double2* X, int n_x, const double2* Y, int n_y, int d, double2* G, int g_stride,
                     cudaStream_t st);
// y = c / c^dag x between neighbouring sectors.
int launch_cop(const kg_sector* src, const kg_sector* dst, int site, int spin, int dagger,
               const double2* x, double2* y, cudaStream_t st);
// utilities
int launch_random_start(double2* v, int d, unsigned long long seed, cudaStream_t st);
int launch_scale_copy(double2* dst, const double2* src, int d, double s, cudaStream_t st);

// ------------------------------------------------------------ drivers
int sector_build(int L, int nu, int nd, const double* h_re, const double* h_im, const double* eps,
                 const double* U, kg_sector** out);
void sector_free(kg_sector* s);
int neighbour(kg_sector* s, int spin, int dagger, kg_sector** out);
cudaStream_t pick_stream(const kg_sector* s, const kg_opts* o);

// One propagation step exp(-i H tau_b) of every column b of K, starting from
// V[b][0] and leaving the result at desc[b].out (V[b][0] unless changed),
// with the overlaps configured in the column descriptors.
int enqueue_step(Krylov& K, int reorth, cudaStream_t st);
// Builds every work list a step uses (device allocations) so that the step
// can then be captured into a graph, where allocation is not allowed.
int prepare_step(Krylov& K, int reorth);
int prepare_hpsi_lists(Krylov& K);
// Sets the overlap row counter of every column.
int launch_set_slots(Krylov& K, int value, cudaStream_t st);
// Clears every column's status (KG_OK); the kernels only ever raise it, so a
// non-finite value met in any step of a call stays reported until this runs.
int launch_reset_status(Krylov& K, cudaStream_t st);

// Replays the launch sequence of one propagation step, as a CUDA graph when
// allowed (the sequence is fixed: iteration counts and early exits after a
// breakdown are decided on the device).
struct StepRunner {
    Krylov* K = nullptr;
    int reorth = 1;
    cudaGraphExec_t exec = nullptr;
    size_t nodes = 0;
    bool graph = false;
    int init(Krylov& k, int reorth_mode, cudaStream_t st, bool use_graph);
    int run(cudaStream_t st);
    void release();
};

int ground_state(kg_sector* s, const kg_opts* o);
int green_equilibrium(kg_sector* s, const int* orb, int n_orb, double dt, int n_steps, const kg_opts* o,
                      double* G_gtr, double* G_les);
int green_equilibrium_batched(kg_sector* const* s, int n_inst, const int* orb, int n_orb, double dt, int n_steps,
                              const kg_opts* o, double* G_gtr, double* G_les, int* status);
int gram(const double2* X, int nv, int d, int nsm, std::vector<std::complex<double>>& G, cudaStream_t st);
int green_equilibrium_vjp(kg_sector* s, const int* orb, int n_orb, double dt, int n_steps, const kg_opts* o,
                          int checkpoint, const double* dGgtr, const double* dGles, double* g_eps, double* g_hre,
                          double* g_him, double* g_U);
// dparams (host, or null for the quench): a driven H(t) after t = 0, the
// on-site offsets at the Gauss nodes of every internal step,
// [(n_t - 1) n_sub][2][3L] (eps_up, eps_dn, U).
int keldysh_create(kg_sector* ini, kg_sector* fin, const int* orb, int n_orb, double dt, int n_t,
                   const kg_opts* o, kg_keldysh** out, const double* dparams = nullptr);
void keldysh_free(kg_keldysh* X);
int keldysh_row(kg_keldysh* X, int k, double* G_les_kk, double* G_gtr_kk);
int keldysh_gram(kg_keldysh* X, double* G_les, double* G_gtr);
int keldysh_phi(kg_keldysh* X, int k, double* phi_host, const double* phi_in);
int keldysh_plan(const kg_keldysh* X, int* phi_on_host, int* stores_kept, int* planes, long long* budget);
int green_keldysh(kg_sector* ini, kg_sector* fin, const int* orb, int n_orb, double dt, int n_t,
                  const kg_opts* o, double* G_les, double* G_gtr, const double* dparams = nullptr);
int green_four_time(kg_sector* ini, kg_sector* fin, const int* ops, double dt, int n_t, const kg_opts* o, double* G);
int green_mixed(kg_sector* ini, kg_sector* fin, const int* orb, int n_orb, double dt, int n_t, double mu, double dtau,
                int n_tau, const kg_opts* o, double* G_right, double* G_left);
int green_matsubara_steps(kg_sector* s, const int* orb, int n_orb, double mu, double dtau, int n_steps,
                          const kg_opts* o, double* G_plus, double* G_minus);
int necpt_occupations(kg_sector* ini, kg_sector* fin, int L_b, double T_b, double V, double dt, int n_t, double beta,
                      int n_tau, const kg_opts* o, double* n_out);
int propagate(kg_sector* s, double2* x, double dt, int n_steps, const kg_opts* o);
void set_capturing(bool on);
bool profiling();

// Opt-in per-kernel timing: while the profiler is on, every launcher brackets
// its launch with CUDA events on the launch stream (graphs are not used).
struct ProfScope {
    int slot = -1;
    cudaStream_t st = nullptr;
    ProfScope(const char* name, cudaStream_t s);
    ~ProfScope();
};
int profile_start();
int profile_stop();
int profile_count();
int profile_get(int i, char* name, int len, long long* launches, double* ms);
int probe_fp64(double* tflops, cudaStream_t st);
unsigned long long launch_count();
const char* last_error();

}  // namespace kg

// ----------------------------------------------------- device helpers
#ifdef __CUDACC__
namespace kg {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ double2 cdotmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}

// s / D_up and s % D_up without a hardware divide (multiply-high method).
__device__ __forceinline__ void split_index(const SecView& S, int s, int& i_dn, int& i_up) {
    i_dn = (int)((__umulhi((unsigned)s, S.du_m) + (unsigned)s) >> S.du_l);
    i_up = s - i_dn * S.Du;
}

// FP32 -> FP64 (exact) on the integer pipe; subnormal inputs give 0.
__device__ __forceinline__ double f32_to_f64_int(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e8 = (b >> 23) & 0xffu;
    if (e8 == 0u) return 0.0;
    const unsigned e11 = e8 == 0xffu ? 0x7ffu : e8 + 896u;
    const unsigned hi = (b & 0x80000000u) | (e11 << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// FP64 -> FP32 by truncation on the integer pipe (no FP64 instruction):
// exponent rebias and the top 23 mantissa bits; |x| < 2^-126 gives 0.  Used
// only for correction terms whose size makes the truncation negligible.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;
    const unsigned bits = (hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    return e > 0 ? __uint_as_float(bits) : 0.0f;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums nv doubles over the block.  v: this thread's values; sm: shared
// scratch of (blockDim/32)*nv doubles; on return out[0..nv) (shared) holds
// the block totals (valid for all threads).
template <int NV>
__device__ __forceinline__ void block_sum(const double (&v)[NV], int nv, double* sm, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if (k < nv) {
            double s = warp_sum(v[k]);
            if (lane == 0) sm[warp * nv + k] = s;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sm[w * nv + k];
        out[k] = s;
    }
    __syncthreads();
}

// A block of a work-list launch: its column b, its index blk among the nblk
// blocks of that column, the column descriptor D and scalars C.
#define KG_ITEM()                                   \
    const int4 it_ = items[blockIdx.x];             \
    const int b = it_.x, blk = it_.y, nblk = it_.z; \
    const ColDesc D = desc[b];                      \
    ColScalars* C = cs + b
#define KG_FOR(i) for (int i = blk * blockDim.x + threadIdx.x; i < D.d; i += nblk * blockDim.x)

// Block maximum of an int (valid in thread 0 only).
__device__ __forceinline__ int block_max_int(int v, int* sm) {
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    int m = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, sm[w]);
    __syncthreads();
    return m;
}

// Biased exponent field of an FP64 value (0 for zero).
__device__ __forceinline__ int exp_field(double x) {
    return (int)(((unsigned)__double2hiint(x) >> 20) & 0x7ffu);
}

// Fixed-point image round(x * 2^(1075 + P - E)) of x, for E at least the
// exponent field of x (so |result| < 2^(53 + P)); `neg` (0/1) flips the sign
// together with x's own.  Exponent field 0 (zero, subnormal) gives 0.
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

// round(x * 2^(1074 - E)) for E at least the exponent field of x, so that
// |x| < 2^(E - 1022) and |result| < 2^52: a 52-bit fixed-point number whose
// unit is 2^-52 of the bound.  Zero and subnormal x give 0.  Integer pipe
// only (round half away from zero on the magnitude).
__device__ __forceinline__ long long fix52(double x, int E) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffull);
    const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;  // x = m 2^(e - 1075)
    const int r = min(E + 1 - e, 63);                                              // >= 1
    long long v = (long long)((m + (1ull << (r - 1))) >> r);
    v = e ? v : 0ll;
    return (b >> 63) ? -v : v;
}

// The two 26-bit halves of a 52-bit fixed-point number: v = hi 2^26 + lo,
// lo in [0, 2^26), |hi| <= 2^26.
__device__ __forceinline__ int fix_hi(long long v) { return (int)(v >> 26); }
__device__ __forceinline__ int fix_lo(long long v) { return (int)(v & 0x3ffffffll); }

__device__ __forceinline__ int4 fix_image(double2 u, int E) {
    const long long x = fix52(u.x, E), y = fix52(u.y, E);
    return make_int4(fix_hi(x), fix_lo(x), fix_hi(y), fix_lo(y));
}

// The fixed-point image of V_{j+1} is written by the update with an exponent
// bound known before the vector exists; H*psi uses it when the bound exceeds
// the vector's true largest exponent by at most kFixSlack bits (each bit
// costs one bit of the fixed-point sums' precision, which has P >= 4 bits to
// spare over FP64), and converts on the fly otherwise.
constexpr int kFixSlack = 4;

// Deterministic reduction over the nblk blocks of one column (block `row`).
// Each block stores its nv + nmax totals (bsum, in shared memory) into its
// row of part; the last block to arrive (atomic ticket) combines the rows in
// a fixed order into red (shared): values [0, nv) are summed, values
// [nv, nv + nmax) max-reduced.  It resets the ticket and returns true; other
// blocks return false.
__device__ __forceinline__ bool grid_finish(const double* bsum, int nv, double* part, unsigned* cnt, int row,
                                            int nblk, double* red, int nmax = 0) {
    __shared__ unsigned ticket;
    const int nt = nv + nmax;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) part[(size_t)row * kPart + k] = bsum[k];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(cnt, 1u);
    __syncthreads();
    if (ticket != (unsigned)(nblk - 1)) return false;
    __threadfence();
    // value k is combined by one warp: lanes take blocks lane, lane+32, ...
    // then a fixed shuffle tree -- the order does not depend on timing.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < nt; k += nw) {
        if (k < nv) {
            double s = 0.0;
            for (int b = lane; b < nblk; b += 32) s += __ldcg(part + (size_t)b * kPart + k);
            s = warp_sum(s);
            if (lane == 0) red[k] = s;
        } else {
            double s = 0.0;
            for (int b = lane; b < nblk; b += 32) s = fmax(s, __ldcg(part + (size_t)b * kPart + k));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
            if (lane == 0) red[k] = s;
        }
    }
    if (threadIdx.x == 0) *cnt = 0u;
    __syncthreads();
    return true;
}

}  // namespace kg
#endif
