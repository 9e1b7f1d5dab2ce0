// kg_oracle.cpp -- plain, slow FP64 CPU oracle for the Krylov-space
// Green's-function method (Balzer, Gdaniec, Potthoff).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code;
// it exists so that tests/, the smoke check and the bench's CPU baseline can
// check the CUDA path against an independent implementation.  It shares no
// code, table or helper with the CUDA library.
//
// What it computes, and from which passage:
//   * occupation-number basis with N_up, N_dn conserved (Section 2, H_jj' in
//     the occupation-number basis; Section 4, N and S_z good quantum numbers):
//     all 2L-bit states with the right popcounts, sorted, found by binary
//     search (no combinatorial ranking here on purpose);
//   * H*psi written out term by term in second quantisation with
//     Jordan-Wigner signs (Section 2; model Hamiltonians of Section 3 and 4);
//   * c and c^dag maps between sectors (Section 3 Eq. (psit), Section 4
//     step (iii));
//   * ground state: Lanczos recursion, Eq. (recursion), with full
//     Gram-Schmidt reorthogonalisation (Section 3, the remark on
//     reorthogonalisation), T diagonalised by cyclic Jacobi (Eq. (tdiag)),
//     Ritz vector Eq. (eigen), restarted until the true residual is small;
//   * exp(-i H tau) psi by a Chebyshev expansion with Bessel coefficients
//     (Tal-Ezer and Kosloff 1984) -- a different algorithm from the
//     GPU's Krylov propagation of Eq. (udelta), used as the exact reference.
//
// Mode ordering: mode m = sigma*L + i (all up orbitals, then all down).
// A basis state is the 64-bit word with bit m = n_m; the state is
// c^dag_{m1} c^dag_{m2} ... |vac> with m1 < m2 < ...
// Vectors are complex<double> arrays (interleaved re, im).

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <random>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cd;

struct ko_model {
    int L, nu, nd;
    std::vector<cd> h;        // h[i*L+j] = h_ij (Hermitian)
    std::vector<double> eps;  // eps[s*L+i]
    std::vector<double> U;    // U[i]
    std::vector<uint64_t> basis;
    double lo, hi;            // Gershgorin bounds of the spectrum
};

static inline int popc64(uint64_t x) { return __builtin_popcountll(x); }

// Parity of the number of occupied modes below m (Jordan-Wigner string).
static inline double jw_sign(uint64_t st, int m) {
    uint64_t below = (m == 0) ? 0ULL : (st & ((1ULL << m) - 1ULL));
    return (popc64(below) & 1) ? -1.0 : 1.0;
}

// c_m |st>: returns false when mode m is empty.
static bool op_c(uint64_t st, int m, uint64_t* out, double* sg) {
    if (!((st >> m) & 1ULL)) return false;
    *sg = jw_sign(st, m);
    *out = st & ~(1ULL << m);
    return true;
}

// c^dag_m |st>: returns false when mode m is occupied.
static bool op_cdag(uint64_t st, int m, uint64_t* out, double* sg) {
    if ((st >> m) & 1ULL) return false;
    *sg = jw_sign(st, m);
    *out = st | (1ULL << m);
    return true;
}

static long find_state(const ko_model* M, uint64_t st) {
    auto it = std::lower_bound(M->basis.begin(), M->basis.end(), st);
    if (it == M->basis.end() || *it != st) return -1;
    return (long)(it - M->basis.begin());
}

static double diag_energy(const ko_model* M, uint64_t st) {
    const int L = M->L;
    double e = 0.0;
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < L; ++i)
            if ((st >> (s * L + i)) & 1ULL) e += M->eps[s * L + i] + M->h[i * L + i].real();
    for (int i = 0; i < L; ++i)
        if (((st >> i) & 1ULL) && ((st >> (L + i)) & 1ULL)) e += M->U[i];
    return e;
}

// y = H x in the gather form: for output state s, every hopping term
// h_ij c^dag_i c_j connects s to s' = c^dag_j c_i s, with
// <s| c^dag_i c_j |s'> equal to the product of the two JW signs.
static void hpsi_impl(const ko_model* M, const cd* x, cd* y) {
    const long d = (long)M->basis.size();
    const int L = M->L;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < d; ++s) {
        const uint64_t st = M->basis[s];
        cd acc = diag_energy(M, st) * x[s];
        for (int sg = 0; sg < 2; ++sg)
            for (int i = 0; i < L; ++i)
                for (int j = 0; j < L; ++j) {
                    if (i == j) continue;
                    const cd hij = M->h[i * L + j];
                    if (hij == cd(0.0, 0.0)) continue;
                    uint64_t t1, t2;
                    double s1, s2;
                    if (!op_c(st, sg * L + i, &t1, &s1)) continue;
                    if (!op_cdag(t1, sg * L + j, &t2, &s2)) continue;
                    const long k = find_state(M, t2);
                    acc += hij * (s1 * s2) * x[k];
                }
        y[s] = acc;
    }
}

static void gershgorin(ko_model* M) {
    const long d = (long)M->basis.size();
    const int L = M->L;
    double lo = 1e300, hi = -1e300;
    for (long s = 0; s < d; ++s) {
        const uint64_t st = M->basis[s];
        const double c = diag_energy(M, st);
        double r = 0.0;
        for (int sg = 0; sg < 2; ++sg)
            for (int i = 0; i < L; ++i)
                for (int j = 0; j < L; ++j) {
                    if (i == j || M->h[i * L + j] == cd(0.0, 0.0)) continue;
                    uint64_t t1, t2;
                    double s1, s2;
                    if (!op_c(st, sg * L + i, &t1, &s1)) continue;
                    if (!op_cdag(t1, sg * L + j, &t2, &s2)) continue;
                    r += std::abs(M->h[i * L + j]);
                }
        lo = std::min(lo, c - r);
        hi = std::max(hi, c + r);
    }
    if (d == 0) { lo = 0; hi = 0; }
    M->lo = lo;
    M->hi = hi;
}

// Dot products and norms: each thread sums one fixed contiguous slice, the
// slice sums are added in slice order, so the result does not depend on
// timing (only on the thread count).
static cd vdot(const cd* a, const cd* b, long n) {
#ifdef _OPENMP
    const int nt = omp_get_max_threads();
#else
    const int nt = 1;
#endif
    std::vector<cd> part(nt, cd(0.0, 0.0));
#pragma omp parallel num_threads(nt)
    {
#ifdef _OPENMP
        const int t = omp_get_thread_num();
#else
        const int t = 0;
#endif
        const long lo = n * t / nt, hi = n * (t + 1) / nt;
        cd s(0.0, 0.0);
        for (long i = lo; i < hi; ++i) s += std::conj(a[i]) * b[i];
        part[t] = s;
    }
    cd s(0.0, 0.0);
    for (const cd& p : part) s += p;
    return s;
}

static double vnorm(const cd* a, long n) { return std::sqrt(vdot(a, a, n).real()); }

// y -= c * x
static void vaxpy(cd c, const cd* x, cd* y, long n) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) y[i] -= c * x[i];
}

// Cyclic Jacobi eigenvalue algorithm for a dense real symmetric matrix
// (Golub and Van Loan, Section 8.5).  A (n x n, row-major) is destroyed;
// on return w holds the eigenvalues and Z the eigenvectors as columns.
static void jacobi_eigen(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& Z) {
    Z.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
    double fro = 0.0;
    for (double v : A) fro += v * v;
    for (int sweep = 0; sweep < 200; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off <= 1e-34 * fro || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q of A
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q of A
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double zkp = Z[(size_t)k * n + p], zkq = Z[(size_t)k * n + q];
                    Z[(size_t)k * n + p] = c * zkp - s * zkq;
                    Z[(size_t)k * n + q] = s * zkp + c * zkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

extern "C" {

ko_model* ko_model_new(int L, int nu, int nd, const double* h_re, const double* h_im,
                       const double* eps, const double* U) {
    if (L < 1 || L > 24 || nu < 0 || nd < 0 || nu > L || nd > L) return nullptr;
    ko_model* M = new ko_model();
    M->L = L; M->nu = nu; M->nd = nd;
    M->h.resize((size_t)L * L);
    for (int k = 0; k < L * L; ++k) M->h[k] = cd(h_re[k], h_im ? h_im[k] : 0.0);
    M->eps.assign(eps, eps + 2 * L);
    M->U.assign(U, U + L);
    std::vector<uint64_t> ups, dns;
    for (uint64_t x = 0; x < (1ULL << L); ++x) {
        if (popc64(x) == nu) ups.push_back(x);
        if (popc64(x) == nd) dns.push_back(x);
    }
    M->basis.reserve(ups.size() * dns.size());
    for (uint64_t b : dns)
        for (uint64_t a : ups) M->basis.push_back(a | (b << L));
    std::sort(M->basis.begin(), M->basis.end());
    gershgorin(M);
    return M;
}

void ko_model_free(ko_model* M) { delete M; }

long ko_model_dim(const ko_model* M) { return (long)M->basis.size(); }

void ko_model_basis(const ko_model* M, uint64_t* out) {
    std::memcpy(out, M->basis.data(), M->basis.size() * sizeof(uint64_t));
}

void ko_model_bounds(const ko_model* M, double* lo, double* hi) { *lo = M->lo; *hi = M->hi; }

int ko_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ko_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

void ko_hpsi(const ko_model* M, const double* x, double* y) {
    hpsi_impl(M, reinterpret_cast<const cd*>(x), reinterpret_cast<cd*>(y));
}

// y = c_{site,spin} x (dagger = 0) or c^dag_{site,spin} x (dagger = 1); y lives
// in dst's sector, which must be the neighbouring one.  Returns 0 or -1.
// The sector Hamiltonian as a dense row-major d x d matrix: the same terms as
// ko_hpsi, each written to its own entry H[s][k] (one hopping term links a
// pair of states at most, so every entry is a single term or the diagonal).
void ko_dense_h(const ko_model* M, double* out_) {
    cd* out = reinterpret_cast<cd*>(out_);
    const long d = (long)M->basis.size();
    const int L = M->L;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < d; ++s) {
        cd* row = out + s * d;
        for (long k = 0; k < d; ++k) row[k] = cd(0.0, 0.0);
        const uint64_t st = M->basis[s];
        row[s] = diag_energy(M, st);
        for (int sg = 0; sg < 2; ++sg)
            for (int i = 0; i < L; ++i)
                for (int j = 0; j < L; ++j) {
                    if (i == j) continue;
                    const cd hij = M->h[i * L + j];
                    if (hij == cd(0.0, 0.0)) continue;
                    uint64_t t1, t2;
                    double s1, s2;
                    if (!op_c(st, sg * L + i, &t1, &s1)) continue;
                    if (!op_cdag(t1, sg * L + j, &t2, &s2)) continue;
                    row[find_state(M, t2)] += hij * (s1 * s2);
                }
    }
}

int ko_apply_cop(const ko_model* src, const ko_model* dst, int site, int spin, int dagger,
                 const double* x_, double* y_) {
    if (src->L != dst->L) return -1;
    const int dnu = (spin == 0) ? (dagger ? 1 : -1) : 0;
    const int dnd = (spin == 1) ? (dagger ? 1 : -1) : 0;
    if (dst->nu != src->nu + dnu || dst->nd != src->nd + dnd) return -1;
    const cd* x = reinterpret_cast<const cd*>(x_);
    cd* y = reinterpret_cast<cd*>(y_);
    const long dd = (long)dst->basis.size();
    for (long k = 0; k < dd; ++k) y[k] = 0.0;
    const int m = spin * src->L + site;
    for (size_t s = 0; s < src->basis.size(); ++s) {
        uint64_t t;
        double sg;
        const bool ok = dagger ? op_cdag(src->basis[s], m, &t, &sg) : op_c(src->basis[s], m, &t, &sg);
        if (!ok) continue;
        const long k = find_state(dst, t);
        if (k < 0) return -1;
        y[k] += sg * x[s];
    }
    return 0;
}

// Lanczos ground state with full reorthogonalisation and Ritz restarts.
// Returns 0 when the residual ||H psi - E0 psi|| <= tol*max(1,|E0|), 1 when
// max_restarts were used up (E0, psi, resid hold the last iterate).
int ko_ground_state(const ko_model* M, int K, int max_restarts, double tol, unsigned long long seed,
                    double* E0, double* psi_out, double* resid) {
    const long d = (long)M->basis.size();
    if (d == 0) return -1;
    std::mt19937_64 gen(seed);
    std::uniform_real_distribution<double> uni(-1.0, 1.0);
    std::vector<cd> v(d);
    for (long i = 0; i < d; ++i) v[i] = cd(uni(gen), 0.0);
    {
        const double nv = vnorm(v.data(), d);
        for (auto& z : v) z /= nv;
    }
    std::vector<cd> w(d), u(d), Hu(d);
    int status = 1;
    for (int r = 0; r < max_restarts; ++r) {
        std::vector<std::vector<cd>> V;
        std::vector<double> alpha, beta(1, 0.0);
        V.push_back(v);
        const int kmax = (int)std::min<long>(K, d);
        for (int j = 0; j < kmax; ++j) {
            hpsi_impl(M, V[j].data(), w.data());
            const double a = vdot(V[j].data(), w.data(), d).real();
            vaxpy(a, V[j].data(), w.data(), d);
            if (j > 0) vaxpy(beta[j], V[j - 1].data(), w.data(), d);
            for (int pass = 0; pass < 2; ++pass)
                for (int k = 0; k <= j; ++k) vaxpy(vdot(V[k].data(), w.data(), d), V[k].data(), w.data(), d);
            alpha.push_back(a);
            const double b = vnorm(w.data(), d);
            if (j + 1 == kmax || b <= 1e-13 * (std::fabs(a) + beta[j] + 1e-300)) break;
            beta.push_back(b);
            std::vector<cd> nv(d);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < d; ++i) nv[i] = w[i] / b;
            V.push_back(nv);
        }
        const int m = (int)alpha.size();
        std::vector<double> T((size_t)m * m, 0.0), ev, Z;
        for (int i = 0; i < m; ++i) T[(size_t)i * m + i] = alpha[i];
        for (int i = 1; i < m; ++i) T[(size_t)i * m + i - 1] = T[(size_t)(i - 1) * m + i] = beta[i];
        jacobi_eigen(T, m, ev, Z);
        int i0 = 0;
        for (int i = 1; i < m; ++i)
            if (ev[i] < ev[i0]) i0 = i;
        for (long i = 0; i < d; ++i) u[i] = 0.0;
        for (int k = 0; k < m; ++k) vaxpy(-Z[(size_t)k * m + i0], V[k].data(), u.data(), d);
        const double nu_ = vnorm(u.data(), d);
        for (auto& z : u) z /= nu_;
        hpsi_impl(M, u.data(), Hu.data());
        const double rq = vdot(u.data(), Hu.data(), d).real();
        for (long i = 0; i < d; ++i) w[i] = Hu[i] - rq * u[i];
        const double rn = vnorm(w.data(), d);
        *E0 = rq;
        *resid = rn;
        std::memcpy(psi_out, u.data(), d * sizeof(cd));
        if (rn <= tol * std::max(1.0, std::fabs(rq))) { status = 0; break; }
        v = u;
    }
    return status;
}

// y = exp(-i H tau) x by the Chebyshev expansion
//   exp(-i H tau) = exp(-i b tau) sum_k (2 - delta_k0) (-i)^k J_k(a tau) T_k((H - b)/a)
// with [b - a, b + a] enclosing the spectrum (Gershgorin bounds, widened).
// Returns the number of Chebyshev terms used.
int ko_propagate(const ko_model* M, const double* x_, double tau, double* y_) {
    const long d = (long)M->basis.size();
    const cd* x = reinterpret_cast<const cd*>(x_);
    cd* y = reinterpret_cast<cd*>(y_);
    const double a = 0.5 * (M->hi - M->lo) * 1.01 + 1e-8;
    const double b = 0.5 * (M->hi + M->lo);
    const double z = a * tau;
    const double az = std::fabs(z);
    const cd step = (z >= 0) ? cd(0.0, -1.0) : cd(0.0, 1.0);  // (-i sgn z)
    std::vector<cd> t0(x, x + d), t1(d), t2(d), tmp(d);
    // T_1 = (H - b)/a x
    hpsi_impl(M, t0.data(), tmp.data());
    for (long i = 0; i < d; ++i) t1[i] = (tmp[i] - b * t0[i]) / a;
    const double j0 = std::cyl_bessel_j(0.0, az);
    cd ph = step;
    cd c1 = 2.0 * ph * std::cyl_bessel_j(1.0, az);
    for (long i = 0; i < d; ++i) y[i] = j0 * t0[i] + c1 * t1[i];
    int k = 1, small = 0;
    while (true) {
        ++k;
        hpsi_impl(M, t1.data(), tmp.data());
        ph *= step;
        const double jk = std::cyl_bessel_j((double)k, az);
        const cd ck = 2.0 * ph * jk;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < d; ++i) {
            t2[i] = 2.0 * (tmp[i] - b * t1[i]) / a - t0[i];
            y[i] += ck * t2[i];
        }
        std::swap(t0, t1);
        std::swap(t1, t2);
        if (k > az && std::fabs(jk) < 1e-18) {
            if (++small >= 2) break;
        } else {
            small = 0;
        }
        if (k > 100000) break;
    }
    const cd g = std::exp(cd(0.0, -b * tau));
    for (long i = 0; i < d; ++i) y[i] *= g;
    return k + 1;
}

}  // extern "C"
