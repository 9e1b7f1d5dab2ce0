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
#include <complex>
#include <vector>

#include "kg_internal.h"

namespace kg {

int green_lanczos(kg_sector* s, const int* orb, int n_orb, int n, const double* omega, int n_omega, double eta,
                  const kg_opts* o, double* G_gtr, double* G_les, double* coef) {
    if (!orb || n_orb < 1 || n < 1 || n > kMaxMgs - 1 || n_omega < 0 || (n_omega > 0 && !omega) ||
        !(eta >= 0.0) || (n_omega > 0 && (!G_gtr || !G_les)) || o->reorth < 0 || o->reorth > 2 ||
        o->schedule < 0 || o->schedule > 3) {
        set_error("bad arguments to the Lanczos Green's function (need 1 <= n <= %d, eta >= 0)", kMaxMgs - 1);
        return KG_EINVAL;
    }
    for (int a = 0; a < n_orb; ++a)
        if (orb[2 * a] < 0 || orb[2 * a] >= s->L || (orb[2 * a + 1] != 0 && orb[2 * a + 1] != 1)) {
            set_error("orbital %d out of range", a);
            return KG_EINVAL;
        }
    if (!s->has_gs) KG_TRY(ground_state(s, o));
    cudaStream_t st = pick_stream(s, o);
    const double E0 = s->E0;
    // columns: (orbital a, kind) for every existing neighbour sector
    struct Col {
        int a, dagger;
        kg_sector* nb;
    };
    std::vector<Col> cl;
    std::vector<const kg_sector*> cols;
    for (int a = 0; a < n_orb; ++a)
        for (int dagger = 1; dagger >= 0; --dagger) {
            kg_sector* nb = nullptr;
            if (neighbour(s, orb[2 * a + 1], dagger, &nb) != KG_OK) continue;  // empty/full band: that part is 0
            cl.push_back({a, dagger, nb});
            cols.push_back(nb);
        }
    std::vector<ColScalars> h(cl.size());
    if (!cl.empty()) {
        Krylov K;
        KG_TRY(krylov_alloc(K, cols, n, s->nsm, o->schedule));
        int rc = KG_OK;
        for (size_t b = 0; rc == KG_OK && b < cl.size(); ++b)
            rc = launch_cop(s, cl[b].nb, orb[2 * cl[b].a], orb[2 * cl[b].a + 1], cl[b].dagger, s->gs,
                            K.vec((int)b, 0), st);
        if (rc == KG_OK) rc = build_space(K, std::max(1, o->reorth), st);
        if (rc == KG_OK && (cudaMemcpyAsync(h.data(), K.cs, sizeof(ColScalars) * h.size(), cudaMemcpyDeviceToHost,
                                            st) != cudaSuccess ||
                            cudaStreamSynchronize(st) != cudaSuccess))
            rc = cuda_fail(cudaGetLastError(), "Lanczos coefficients", __FILE__, __LINE__);
        krylov_free(K);
        if (rc != KG_OK) return rc;
        for (auto& c : h)
            if (c.status == KG_ENUMERIC) {
                set_error("non-finite value in the Lanczos run");
                return KG_ENUMERIC;
            }
    }
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

}  // namespace kg

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
