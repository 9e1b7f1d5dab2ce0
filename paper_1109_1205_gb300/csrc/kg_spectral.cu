// kg_spectral.cu -- the conventional Lanczos Green's function (Section 2,
// Eqs. (gomega), (resolv), (gapprox)): for a diagonal orbital alpha, the
// resolvent of H restricted to the n-dimensional Krylov space of
// c^dag_alpha |0> (particle part) or c_alpha |0> (hole part).  In that basis
// the resolvent is the (0,0) element of the inverse of a tridiagonal matrix,
// i.e. a continued fraction in the Lanczos coefficients a_j, b_j:
//
//   G^>(w) = b_0^2 / (z - a_0 - b_1^2 / (z - a_1 - b_2^2 / ...)),  z = w + i eta + E0
//   G^<(w) = b_0^2 / (z' + a_0 - b_1^2 / (z' + a_1 - ...)),        z' = w + i eta - E0
//
// with b_0 = ||c^dag |0>|| (or ||c |0>||).  This is the n-pole sum of
// Eq. (gapprox) over the Ritz pairs of the Lanczos run, summed without
// diagonalising.  The Lanczos runs of all requested orbitals and both kinds
// are one Krylov batch on the GPU (the kernels of the propagation, with full
// reorthogonalisation); the continued fractions, O(n) per frequency, are
// evaluated on the host.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "kg_internal.h"

namespace kg {

namespace {
struct LzCol {
    int a, dagger;
    kg_sector* nb;
};
}  // namespace

// The n-step Lanczos runs (full reorthogonalisation) from c^dag_a|0> and
// c_a|0> of every requested orbital, as one Krylov batch; the ground state is
// computed first if needed.  cl lists the runs (a part whose neighbour sector
// does not exist is left out), h their coefficients.
static int lanczos_columns(kg_sector* s, const int* orb, int n_orb, int n, const kg_opts* o, std::vector<LzCol>& cl,
                           std::vector<ColScalars>& h) {
    if (!orb || n_orb < 1 || n < 1 || n > kMaxMgs - 1 || o->reorth < 0 || o->reorth > 2 || o->schedule < 0 ||
        o->schedule > 7) {
        set_error("bad arguments to the Lanczos runs (need orbitals and 1 <= n <= %d)", kMaxMgs - 1);
        return KG_EINVAL;
    }
    for (int a = 0; a < n_orb; ++a)
        if (orb[2 * a] < 0 || orb[2 * a] >= s->L || (orb[2 * a + 1] != 0 && orb[2 * a + 1] != 1)) {
            set_error("orbital %d out of range", a);
            return KG_EINVAL;
        }
    if (!s->has_gs) KG_TRY(ground_state(s, o));
    cudaStream_t st = pick_stream(s, o);
    std::vector<const kg_sector*> cols;
    cl.clear();
    for (int a = 0; a < n_orb; ++a)
        for (int dagger = 1; dagger >= 0; --dagger) {
            kg_sector* nb = nullptr;
            if (neighbour(s, orb[2 * a + 1], dagger, &nb) != KG_OK) continue;  // empty/full band: that part is 0
            cl.push_back({a, dagger, nb});
            cols.push_back(nb);
        }
    h.assign(cl.size(), ColScalars());
    if (cl.empty()) return KG_OK;
    Krylov K;
    KG_TRY(krylov_alloc(K, cols, n, s->nsm, o->schedule));
    int rc = KG_OK;
    for (size_t b = 0; rc == KG_OK && b < cl.size(); ++b)
        rc = launch_cop(s, cl[b].nb, orb[2 * cl[b].a], orb[2 * cl[b].a + 1], cl[b].dagger, s->gs, K.vec((int)b, 0),
                        st);
    if (rc == KG_OK) rc = build_space(K, std::max(1, o->reorth), st);
    if (rc == KG_OK && (cudaMemcpyAsync(h.data(), K.cs, sizeof(ColScalars) * h.size(), cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
        rc = cuda_fail(cudaGetLastError(), "Lanczos coefficients", __FILE__, __LINE__);
    krylov_free(K);
    if (rc != KG_OK) return rc;
    for (auto& c : h)
        if (c.status == KG_ENUMERIC) {
            set_error("non-finite value in the Lanczos run");
            return KG_ENUMERIC;
        }
    return KG_OK;
}

int green_lanczos(kg_sector* s, const int* orb, int n_orb, int n, const double* omega, int n_omega, double eta,
                  const kg_opts* o, double* G_gtr, double* G_les, double* coef) {
    if (n_omega < 0 || (n_omega > 0 && !omega) || !(eta >= 0.0) || (n_omega > 0 && (!G_gtr || !G_les))) {
        set_error("bad arguments to the Lanczos Green's function (need eta >= 0 and output buffers)");
        return KG_EINVAL;
    }
    std::vector<LzCol> cl;
    std::vector<ColScalars> h;
    KG_TRY(lanczos_columns(s, orb, n_orb, n, o, cl, h));
    const double E0 = s->E0;
    // coefficients out: [n_orb][kind: 0 = particle, 1 = hole][a_0..a_{n-1}, b_0..b_{n-1}],
    // zero beyond the Krylov dimension reached (and for a missing kind)
    if (coef) std::fill(coef, coef + (size_t)n_orb * 2 * 2 * n, 0.0);
    for (int k = 0; k < 2 * n_orb * n_omega; ++k) {
        G_gtr[k] = 0.0;
        G_les[k] = 0.0;
    }
    for (size_t b = 0; b < cl.size(); ++b) {
        const ColScalars& c = h[b];
        const int m = c.m_eff, a = cl[b].a, dagger = cl[b].dagger;
        if (coef) {
            double* row = coef + ((size_t)a * 2 + (dagger ? 0 : 1)) * 2 * n;
            for (int j = 0; j < m; ++j) {
                row[j] = c.alpha[j];
                row[n + j] = j == 0 ? c.beta0 : c.beta[j];
            }
        }
        if (m == 0) continue;  // c|0> = 0
        double* G = dagger ? G_gtr : G_les;
        const double b02 = c.beta0 * c.beta0;
        for (int w = 0; w < n_omega; ++w) {
            // bottom-up evaluation of the continued fraction
            const std::complex<double> z = dagger ? std::complex<double>(omega[w] + E0, eta)
                                                  : std::complex<double>(omega[w] - E0, eta);
            const double sg = dagger ? -1.0 : 1.0;  // z - a_j (particle) or z + a_j (hole)
            std::complex<double> tail(0.0, 0.0);
            for (int j = m - 1; j >= 1; --j) tail = c.beta[j] * c.beta[j] / (z + sg * c.alpha[j] - tail);
            const std::complex<double> g = b02 / (z + sg * c.alpha[0] - tail);
            G[2 * ((size_t)a * n_omega + w)] = g.real();
            G[2 * ((size_t)a * n_omega + w) + 1] = g.imag();
        }
    }
    return KG_OK;
}

// Eigenvalues theta_k and first eigenvector components q0_k = Q_{0k} of the
// symmetric tridiagonal T (diagonal alpha[0..m-1], off-diagonal beta[1..m-1],
// beta[j] coupling j-1 and j), by cyclic Jacobi rotations on the dense m x m
// matrix: each rotation in the (p,q) plane, tan(phi) = t the smaller root of
// t^2 + 2 t cot(2 phi) - 1 = 0 with cot(2 phi) = (T_qq - T_pp) / (2 T_pq),
// zeroes T_pq; the first row of the accumulated rotations gives q0.  Sweeps
// until the off-diagonal part is below 1e-30 of the Frobenius norm (m <= 255,
// host, O(m^3) per sweep).
static void tridiag_eigen(const double* alpha, const double* beta, int m, std::vector<double>& theta,
                          std::vector<double>& q0) {
    std::vector<double> A((size_t)m * m, 0.0);
    double norm2 = 0.0;
    for (int j = 0; j < m; ++j) {
        A[(size_t)j * m + j] = alpha[j];
        norm2 += alpha[j] * alpha[j];
        if (j > 0) {
            A[(size_t)j * m + j - 1] = A[(size_t)(j - 1) * m + j] = beta[j];
            norm2 += 2.0 * beta[j] * beta[j];
        }
    }
    q0.assign(m, 0.0);
    q0[0] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) off += 2.0 * A[(size_t)p * m + q] * A[(size_t)p * m + q];
        if (off <= 1e-30 * norm2) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[(size_t)p * m + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
                const double cot2 = (aqq - app) / (2.0 * apq);
                const double t = std::fabs(cot2) > 1e150 ? 0.5 / cot2
                                                          : (cot2 >= 0.0 ? 1.0 : -1.0) /
                                                                (std::fabs(cot2) + std::sqrt(cot2 * cot2 + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                A[(size_t)p * m + p] = app - t * apq;
                A[(size_t)q * m + q] = aqq + t * apq;
                A[(size_t)p * m + q] = A[(size_t)q * m + p] = 0.0;
                for (int r = 0; r < m; ++r) {
                    if (r == p || r == q) continue;
                    const double arp = A[(size_t)r * m + p], arq = A[(size_t)r * m + q];
                    A[(size_t)r * m + p] = A[(size_t)p * m + r] = c * arp - sn * arq;
                    A[(size_t)r * m + q] = A[(size_t)q * m + r] = sn * arp + c * arq;
                }
                const double qp = q0[p], qq = q0[q];
                q0[p] = c * qp - sn * qq;
                q0[q] = sn * qp + c * qq;
            }
    }
    theta.resize(m);
    for (int k = 0; k < m; ++k) theta[k] = A[(size_t)k * m + k];
}

// The zero-temperature Matsubara function of H (Section 4, after step (iv):
// G^M is the equilibrium Green's function of the initial-state Hamiltonian,
// which either Lanczos route of the paper can compute), by the conventional
// route: the n-step Lanczos runs from c^dag_a|0> and
// c_a|0>, their Ritz pairs (theta_k, Q_{0k}) (Eq. (eigen)), and
//   G^M_aa(+tau) = -b0^2 sum_k Q_{0k}^2 e^{-(theta_k - E0 - mu) tau},
//   G^M_aa(-tau) = +b0'^2 sum_k Q'_{0k}^2 e^{-(theta'_k - E0 + mu) tau}.
int green_matsubara(kg_sector* s, const int* orb, int n_orb, int n, double mu, const double* tau, int n_tau,
                    const kg_opts* o, double* G_plus, double* G_minus) {
    if (n_tau < 0 || (n_tau > 0 && (!tau || !G_plus || !G_minus)) || !std::isfinite(mu)) {
        set_error("bad arguments to the Matsubara function (need finite mu and output buffers)");
        return KG_EINVAL;
    }
    for (int j = 0; j < n_tau; ++j)
        if (!(tau[j] >= 0.0) || !std::isfinite(tau[j])) {
            set_error("tau[%d] must be finite and >= 0", j);
            return KG_EINVAL;
        }
    std::vector<LzCol> cl;
    std::vector<ColScalars> h;
    KG_TRY(lanczos_columns(s, orb, n_orb, n, o, cl, h));
    const double E0 = s->E0;
    std::fill(G_plus, G_plus + (size_t)n_orb * n_tau, 0.0);
    std::fill(G_minus, G_minus + (size_t)n_orb * n_tau, 0.0);
    std::vector<double> theta, q0;
    for (size_t b = 0; b < cl.size(); ++b) {
        const ColScalars& c = h[b];
        const int m = c.m_eff, a = cl[b].a, dagger = cl[b].dagger;
        if (m == 0) continue;  // c|0> = 0
        tridiag_eigen(c.alpha, c.beta, m, theta, q0);
        const double b02 = c.beta0 * c.beta0;
        const double shift = dagger ? E0 + mu : E0 - mu;
        double* G = (dagger ? G_plus : G_minus) + (size_t)a * n_tau;
        for (int j = 0; j < n_tau; ++j) {
            double acc = 0.0;
            for (int k = 0; k < m; ++k) acc += q0[k] * q0[k] * std::exp(-(theta[k] - shift) * tau[j]);
            G[j] = dagger ? -b02 * acc : b02 * acc;
        }
    }
    return KG_OK;
}

}  // namespace kg

extern "C" int kg_green_matsubara(kg_sector* s, const int* orb, int n_orb, int n, double mu, const double* tau,
                                  int n_tau, const kg_opts* o, double* G_plus, double* G_minus) {
    if (!s) {
        kg::set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    if (!o) {
        kg_opts_default(&tmp);
        o = &tmp;
    }
    return kg::green_matsubara(s, orb, n_orb, n, mu, tau, n_tau, o, G_plus, G_minus);
}

extern "C" int kg_green_lanczos(kg_sector* s, const int* orb, int n_orb, int n, const double* omega, int n_omega,
                                double eta, const kg_opts* o, double* G_gtr, double* G_les, double* coef) {
    if (!s) {
        kg::set_error("NULL sector");
        return KG_EINVAL;
    }
    kg_opts tmp;
    if (!o) {
        kg_opts_default(&tmp);
        o = &tmp;
    }
    return kg::green_lanczos(s, orb, n_orb, n, omega, n_omega, eta, o, G_gtr, G_les, coef);
}
