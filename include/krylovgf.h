/*
 * krylovgf.h -- C ABI of libkrylovgf, a GB300 (sm_103a) implementation of the
 * Krylov-space method for the zero-temperature single-particle Green's
 * function of Balzer, Gdaniec and Potthoff ("Krylov-space approach to the
 * equilibrium and the nonequilibrium single-particle Green's function").
 *
 * Conventions shared by every call
 * --------------------------------
 * Model (Sections 3 and 4 of the paper, written for one spin-conserving
 * hopping matrix):
 *     H = sum_sigma sum_{i != j} h_ij c^dag_{i sigma} c_{j sigma}
 *         + sum_{i sigma} (eps_{i sigma} + h_ii) n_{i sigma}
 *         + sum_i U_i n_{i up} n_{i dn}
 * The paper writes the hopping as -T sum c^dag c, so callers pass h_ij = -T.
 * A local field H_field = -h (n_up - n_dn) (Eq. (hfi)) is passed through eps.
 *
 * Sector and basis (Section 2: H_jj' in the occupation-number basis; Section 4:
 * particle number and S_z as good quantum numbers): a sector is (L, N_up,
 * N_dn) with D_up = C(L, N_up) up strings and D_dn = C(L, N_dn) down strings.
 * A spin string's index is its rank in ascending numeric order among the
 * L-bit words with that popcount (the combinatorial number system).  The
 * state index is  s = i_dn * D_up + i_up  (i_up fastest), dimension
 * d = D_up * D_dn.  Fermion order: all up orbitals (site order), then all
 * down orbitals; c^dag_{i sigma} carries the sign (-1)^(number of occupied
 * orbitals before (i, sigma)).
 *
 * Vectors are complex FP64, interleaved (re, im): a vector of dimension d is
 * 2*d doubles.  "_dev" pointers are device memory of the current CUDA device,
 * "_host" pointers host memory; the caller owns both.  The library owns every
 * buffer it allocates behind a handle, until the handle is freed.
 *
 * Orbitals are passed as n_orb pairs orb[2a] = site, orb[2a+1] = spin (0 up,
 * 1 down).  Green's functions are complex FP64 arrays (interleaved) with the
 * orbital pair innermost: G[...][a][a'] = G_{a a'}.
 *
 * Every call returns KG_OK (0) or a negative status; no exception and no
 * abort crosses this boundary.  kg_last_error() gives a message for the most
 * recent failure on the calling thread.  One handle must not be used by two
 * threads at once.  Calls are stream-ordered on opts->stream (or the
 * sector's own stream when it is NULL) and return after the results they
 * write to host memory are complete.
 */
#ifndef KRYLOVGF_H
#define KRYLOVGF_H

#ifdef __cplusplus
extern "C" {
#endif

#define KG_OK          0
#define KG_EINVAL     (-1)  /* bad argument, bad sector pair, bad call order   */
#define KG_ENOMEM     (-2)  /* device or host allocation failed / too large    */
#define KG_ENOCONV    (-3)  /* ground state not converged in max_restarts      */
#define KG_EDEGEN     (-4)  /* ground state (near) degenerate: gap < 1e-8      */
#define KG_EBREAKDOWN (-5)  /* informational: Krylov space became invariant    */
#define KG_ENUMERIC   (-6)  /* NaN or Inf met in a norm or dot product         */
#define KG_ETIMEOUT   (-7)  /* a bounded device wait ran out                   */
#define KG_ECUDA      (-8)  /* a CUDA runtime call failed                      */

typedef struct kg_sector kg_sector;
typedef struct kg_keldysh kg_keldysh;

/* Solver options.  kg_opts_default() fills the defaults shown. */
typedef struct kg_opts {
    int M;              /* Krylov dimension n per propagation step, 1..64 (20)  */
    int M_gs;           /* Krylov dimension per ground-state restart, 2..256 (100) */
    int max_restarts;   /* ground-state restarts (200)                         */
    double tol_resid;   /* ground state: stop when ||H0 - E0 0|| <=
                           tol_resid * max(1, |E0|) (1e-12)                    */
    int reorth;         /* 0: three-term recurrence only; 1: plus one full
                           Gram-Schmidt pass against every stored Lanczos
                           vector; 2: plus two passes (1)                       */
    int mem_budget_mb;  /* device memory, in MiB, that a Keldysh calculation
                           may plan for; 0 = the free memory at creation (0) */
    int schedule;       /* bit 0: H*psi hop sums in FP64 always, instead of
                           exact 64-bit integer sums when all hops share one
                           amplitude; bit 1: each propagation step's
                           exponential e^{-iT tau} e_1 through the eigen-
                           decomposition of T (Section 3, Eq. (udelta)),
                           instead of the scaled Taylor series of the same
                           vector; bit 2: Gram-Schmidt dot products in FP64
                           (three multiply-adds per complex product) instead
                           of exact integer products of 52-bit fixed-point
                           images of the Lanczos vectors (0)                     */
    int use_graphs;     /* replay each propagation step as a CUDA graph (1)    */
    double dt_internal; /* Keldysh: Krylov step inside one grid step; 0 = dt   */
    unsigned long long seed; /* ground-state start vector seed (1234)         */
    void* stream;       /* cudaStream_t for all work; NULL = the sector's own
                           stream, ordered after work already queued on the
                           legacy default stream                               */
} kg_opts;

void kg_opts_default(kg_opts* o);

/* ---- sector basis and ranking ------------------------------------------
 * Builds the (L, n_up, n_dn) sector of H (Section 2, occupation-number basis
 * with N and S_z conserved) on the device: the spin strings by unranking in
 * the combinatorial number system, the per-spin hop tables (source rank and
 * fermion sign of every allowed c^dag_a c_b), the single-spin diagonal
 * energies and the U table.
 *   h_re, h_im : L*L row-major host arrays, h[i*L+j] = h_ij, Hermitian;
 *                h_im may be NULL (real hopping).
 *   eps        : 2*L host array, eps[sigma*L + i].
 *   U          : L host array.
 * Limits: 1 <= L <= 32, 0 <= n_up, n_dn <= L, d < 2^31.  Returns KG_EINVAL
 * for bad sizes or non-Hermitian h, KG_ENOMEM when the tables do not fit.
 * *out receives a handle that owns all device memory; free with
 * kg_free_sector (which also frees the neighbour sectors it built). */
int kg_build_sector(int L, int n_up, int n_dn, const double* h_re, const double* h_im,
                    const double* eps, const double* U, kg_sector** out);
void kg_free_sector(kg_sector* s);

/* Dimensions of the sector (any pointer may be NULL). */
int kg_sector_dims(const kg_sector* s, long long* dim, long long* D_up, long long* D_dn);

/* Copies the unranked spin strings (bit i = site i occupied) to host arrays
 * of D_up and D_dn entries: the device result of the combinatorial unranking. */
int kg_sector_strings(const kg_sector* s, unsigned int* up_host, unsigned int* dn_host);

/* ---- H*psi --------------------------------------------------------------
 * y = H x on the device (Section 2, the matrix H_jj' applied on the fly:
 * hopping by bit flips with popcount fermion signs, diagonal eps and U).
 * x_dev, y_dev: complex vectors of dimension d, must not overlap.
 * stream: cudaStream_t; NULL means CUDA's legacy default stream.
 * Asynchronous (stream-ordered).  When all hops of the sector share one
 * amplitude, the hop sums are exact 64-bit integer sums of a fixed-point
 * image of x, held in 16 d bytes of scratch that the sector owns (allocated
 * by the first such call, freed with the sector): calls with one sector must
 * therefore be ordered (one stream, or synchronised), as for any handle. */
int kg_hpsi(kg_sector* s, const double* x_dev, double* y_dev, void* stream);

/* ---- c / c^dag sector maps ------------------------------------------
 * y = c_{site,spin} x (dagger = 0) or y = c^dag_{site,spin} x (dagger = 1),
 * mapping sector (N_up, N_dn) to the neighbouring sector with N_spin -/+ 1
 * (Section 3, the state c^dag_a' |0> of Eq. (psit); Section 4, step (iii)).
 * x_dev has the dimension of s, y_dev that of the neighbour sector (query it
 * with kg_neighbour_dim).  Returns KG_EINVAL if the neighbour does not exist
 * (N_spin would leave [0, L]).  stream as for kg_hpsi.  Asynchronous. */
int kg_neighbour_dim(kg_sector* s, int spin, int dagger, long long* dim);
int kg_apply_cop(kg_sector* s, int site, int spin, int dagger, const double* x_dev, double* y_dev,
                 void* stream);

/* ---- overlaps of caller-held vectors -----------------------------------
 * G[b][a] = <x_a | y_b> = sum_i conj(x_a[i]) y_b[i] for the n_x vectors
 * X_dev (complex, [n_x][d] row-major) and the n_y vectors Y_dev ([n_y][d]):
 * the inner products from which the Green's functions are assembled
 * (Section 3, Eq. (psigreen); Section 4, step (iv)).  G_dev: device,
 * complex [n_y][n_x].  Limits: 1 <= n_x <= 32, n_y >= 1, 1 <= d < 2^31.
 * The reduction is deterministic (fixed order for a given device and size).
 * Partial sums live in a library-owned, grow-only scratch buffer per device
 * (allocated on first use), so calls must not run concurrently on one
 * device.  stream as for kg_hpsi.  Asynchronous. */
int kg_overlaps(const double* X_dev, int n_x, const double* Y_dev, int n_y, long long d, double* G_dev,
                void* stream);

/* The same overlaps for callers that cannot allocate device memory at call
 * time: code that runs under a fixed device-memory budget or with a memory
 * pool that must not grow, or where the allocator's implicit synchronisation
 * is not acceptable.  The paper has no counterpart; this is a deployment
 * variant.  It allocates nothing: its scratch is a fixed 1.2 MB array in the
 * library's device image (every GPU that loads the library holds it until the
 * process exits).  Limits as for kg_overlaps plus n_y <= 64; larger n_y is
 * rejected with KG_EINVAL.  The first call on a device looks up the scratch
 * address (cudaGetSymbolAddress) and should come before any stream capture.
 * All calls share the scratch: calls that overlap on the GPU race, so issue
 * them on one stream or otherwise order them. */
int kg_overlaps_noalloc(const double* X_dev, int n_x, const double* Y_dev, int n_y, long long d, double* G_dev,
                        void* stream);

/* ---- ground state -------------------------------------------------
 * Lanczos ground state of the sector (Section 2: recursion Eq. (recursion)
 * with full reorthogonalisation, T of Eq. (tmatrix) diagonalised on the
 * device, Eq. (tdiag), Ritz vector Eq. (eigen)), restarted from the Ritz
 * vector until ||H|0> - E0|0>|| <= tol_resid*max(1,|E0|).  The ground state
 * stays cached in the handle for the Green's-function calls.
 * E0, resid, gap: host outputs (gap = second-lowest minus lowest Ritz value
 * of the last restart, an estimate; any may be NULL).
 * Returns KG_ENOCONV after max_restarts, KG_EDEGEN when gap < 1e-8. */
int kg_ground_state(kg_sector* s, const kg_opts* o, double* E0, double* resid, double* gap);

/* Copies the cached ground state (complex, dimension d) to psi; to_host != 0
 * means psi is host memory, else device memory.  KG_EINVAL before
 * kg_ground_state. */
int kg_copy_ground_state(kg_sector* s, double* psi, int to_host);

/* ---- Krylov propagation ------------------------------------------
 * x <- exp(-i H dt)^n_steps x in place on the device (Section 3, Eqs.
 * (newstate) and (udelta): one Lanczos space of dimension opts->M per step,
 * T diagonalised on the device, exp(-i D dt) applied in the small space,
 * the new state formed as V Q e^{-iD dt} Q^T e_1 ||x||).  dt < 0 propagates
 * backward, exp(+i H |dt|).  Returns when x_dev holds the result. */
int kg_propagate(kg_sector* s, double* x_dev, double dt, int n_steps, const kg_opts* o);

/* ---- equilibrium Green's function ---------------------------
 * Section 3, Eqs. (psit)/(psigreen) with eta = 0, and the hole part given
 * after Eq. (gomega); for t_k = k*dt, k = 0..n_steps:
 *   G_gtr[k][a][a'] = -i e^{+i E0 t_k} <c^dag_a 0| e^{-iH t_k} |c^dag_a' 0>
 *   G_les[k][a][a'] = +i e^{-i E0 t_k} <c_a' 0| e^{+iH t_k} |c_a 0>
 * (the retarded G is G_gtr - G_les).  Runs kg_ground_state first if needed.
 * G_gtr, G_les: host, complex [(n_steps+1)][n_orb][n_orb].  Entries of
 * opposite spins are zero. */
int kg_green_equilibrium(kg_sector* s, const int* orb, int n_orb, double dt, int n_steps,
                         const kg_opts* o, double* G_gtr, double* G_les);

/* ---- equilibrium Green's function on a fine output grid ---------------
 * Section 3, Eq. (udelta) evaluated at several times per Krylov space: the
 * same G as kg_green_equilibrium on t_k = k*dt, k = 0..n_steps, but each
 * Krylov space (of dimension o->M, built from psi(t)) serves the `fine` times
 * t + q*dt, q = 1..fine (the last one also starts the next space), so there
 * are n_steps/fine Krylov builds instead of n_steps.  The Krylov step is
 * fine*dt: o->M must be large enough for it (the error of one step falls as
 * (w fine dt / 2)^M / M! with w the spectral width of H).  1 <= fine <= 32;
 * output as for kg_green_equilibrium. */
int kg_green_equilibrium_fine(kg_sector* s, const int* orb, int n_orb, double dt, int n_steps, int fine,
                              const kg_opts* o, double* G_gtr, double* G_les);

/* ---- time-dependent Lanczos with restarts ------------------------------
 * Section 3, Fig. 1 (Eqs. (newstate) and (udelta)): the equilibrium G of
 * kg_green_equilibrium on t_k = k dt, k = 0..f*q, with one Krylov space of
 * dimension n (full reorthogonalisation as opts->reorth) built every restart
 * interval Delta t = q dt: inside an interval every output time comes from
 * the same space through the eigen-decomposition of its tridiagonal matrix,
 * and the state at the interval's end starts the next space.  f = 1 is the
 * conventional Lanczos Green's function written in time (Eq. (res)); the
 * paper's Fig. 1 uses n = 100, dt = 0.01, t_max = 1000 and f = 1, 100, 1000.
 * 1 <= n <= 255, f >= 1, q >= 1, f*q <= 2^28, dt > 0 (KG_EINVAL otherwise).
 * G_gtr, G_les: host, complex [(f*q+1)][n_orb][n_orb]. */
int kg_green_restarted(kg_sector* s, const int* orb, int n_orb, int n, int f, int q, double dt, const kg_opts* o,
                       double* G_gtr, double* G_les);

/* ---- conventional Lanczos Green's function (frequency domain) ----------
 * Section 2, Eqs. (gomega), (resolv) and (gapprox): for each diagonal orbital
 * alpha = (site, spin), an n-step Lanczos run (full reorthogonalisation) from
 * c^dag_alpha |0> gives the n-pole particle part and one from c_alpha |0> the
 * hole part, evaluated as continued fractions in the Lanczos coefficients:
 *   G_gtr[a][w] = <0| c_a (omega_w + i eta - H + E0)^{-1} c^dag_a |0>,
 *   G_les[a][w] = <0| c^dag_a (omega_w + i eta + H - E0)^{-1} c_a |0>,
 * so that G_gtr + G_les is the retarded function of Eq. (gomega) with the
 * broadening eta, and A(w) = -Im(G_gtr + G_les)/pi the spectral function.
 * Runs kg_ground_state first if needed.
 *   orb: host int[2 n_orb] (site, spin) pairs; 1 <= n <= 255; eta >= 0.
 *   omega: host double[n_omega]; G_gtr, G_les: host complex [n_orb][n_omega].
 *   coef: host double[n_orb][2][2n] or NULL -- for each orbital, the particle
 *     (index 0) and hole (1) coefficients a_0..a_{n-1}, b_0..b_{n-1}
 *     (b_0 the norm of the start vector, b_j coupling j-1 and j), zero beyond
 *     the Krylov dimension reached.
 * A part whose neighbour sector does not exist (full or empty band) is zero. */
int kg_green_lanczos(kg_sector* s, const int* orb, int n_orb, int n, const double* omega, int n_omega,
                     double eta, const kg_opts* o, double* G_gtr, double* G_les, double* coef);

/* ---- zero-temperature Matsubara function (conventional Lanczos route) ----
 * Section 4, after step (iv): the Matsubara Green's function is the
 * equilibrium Green's function of the (initial-state) Hamiltonian on the
 * imaginary branch.  With K = H - mu N and the ground state |0> of s:
 *   G_plus[a][j]  = G^M_aa(+tau_j) = -<0| c_a e^{-(H - E0 - mu) tau_j} c^dag_a |0>,
 *   G_minus[a][j] = G^M_aa(-tau_j) = +<0| c^dag_a e^{-(H - E0 + mu) tau_j} c_a |0>,
 * evaluated from the n-step Lanczos runs of kg_green_lanczos (the same GPU
 * batch) through the Ritz pairs of each tridiagonal matrix (Eq. (eigen)),
 * found on the host by cyclic Jacobi rotations.  Exact when the Krylov space
 * exhausts the sector; otherwise the error falls faster than exponentially
 * in n at fixed tau.  mu should lie between the removal and addition
 * energies (E0 - E0(N-1) <= mu <= E0(N+1) - E0) for decaying functions.
 *   orb: host int[2 n_orb] (site, spin) pairs; 1 <= n <= 255; mu finite;
 *   tau: host double[n_tau], each finite and >= 0;
 *   G_plus, G_minus: host double[n_orb][n_tau] (real: diagonal orbitals).
 * Runs kg_ground_state first if needed.  A part whose neighbour sector does
 * not exist is zero. */
int kg_green_matsubara(kg_sector* s, const int* orb, int n_orb, int n, double mu, const double* tau, int n_tau,
                       const kg_opts* o, double* G_plus, double* G_minus);

/* ---- zero-temperature Matsubara function on a tau grid ------------------
 * The same G^M as kg_green_matsubara, for every orbital pair of one spin, on
 * tau_k = k dtau, k = 0..n_steps, by imaginary-time Krylov steps: each vector
 * c^dag_b|0> (c_b|0>) is carried from tau to tau + dtau by Eq. (udelta) with
 * the exponential e^{-(T - s) dtau} of the step's Lanczos matrix, s = E0 + mu
 * (E0 - mu); o->M sets the Krylov dimension of a step.
 *   G_plus[k][a][b]  = G^M_ab(+tau_k) = -<0| c_a e^{-(H - E0 - mu) tau_k} c^dag_b |0>,
 *   G_minus[k][a][b] = G^M_ab(-tau_k) = +<0| c^dag_b e^{-(H - E0 + mu) tau_k} c_a |0>,
 * host, complex [(n_steps+1)][n_orb][n_orb]; entries of opposite spins are
 * zero.  n_steps >= 0, dtau > 0 and mu finite (KG_EINVAL otherwise).  Runs
 * kg_ground_state first if needed.  Every step checks the a-posteriori
 * estimate b_M dtau |[e^{-(T - s) dtau} e_1]_{M-1}| of its relative error and
 * returns KG_ENOCONV above 1e-11: the step must keep dtau times the spectral
 * spread of H small against M (the error falls like (w dtau / 2)^M / M!, so
 * for example M = 20 takes w dtau up to about 8). */
int kg_green_matsubara_steps(kg_sector* s, const int* orb, int n_orb, double mu, double dtau, int n_steps,
                             const kg_opts* o, double* G_plus, double* G_minus);

/* ---- G(omega) from G(t): the damped Fourier transform ---------------------
 * Section 3: the frequency-dependent Green's function obtained from the
 * time-dependent one by Fourier transformation, the Lorentzian broadening eta
 * entering as the damping e^{-eta t} (time-dependent Lanczos route, Fig. 1).
 * For each of n_series series sampled at t_k = k dt, k = 0..n_t-1:
 *   G_w[s][j] = sum_k w_k exp(i (omega_j + i eta) t_k) G_t[s][k],
 * w_0 = w_{n_t-1} = dt/2 and w_k = dt otherwise (trapezoidal rule on
 * [0, (n_t-1) dt]; all zero when n_t = 1).  The transform of the particle
 * part G^>(t) of kg_green_equilibrium is the particle part of Eq. (gomega)
 * (G_gtr of kg_green_lanczos, exact in the limit dt -> 0, t_max -> inf), the
 * transform of -G^<(t) the hole part.  Evaluated directly on the caller's
 * frequencies (no FFT grid), FP64, deterministic.
 *   G_t: host, complex [n_series][n_t];  omega: host double[n_omega], finite;
 *   G_w: host, complex [n_series][n_omega] (caller-owned, written);
 *   0 <= n_series <= 65535, 1 <= n_t <= 2^30, n_omega >= 0, dt > 0, eta >= 0
 *   (KG_EINVAL otherwise; KG_ENOMEM when the device copies do not fit).
 * stream as for kg_hpsi; returns after the result is on the host.  Device
 * memory is stream-ordered scratch (cudaMallocAsync), freed before return. */
int kg_green_fourier(const double* G_t, int n_series, int n_t, double dt, const double* omega, int n_omega,
                     double eta, void* stream, double* G_w);

/* ---- batched equilibrium Green's functions ----------------------------
 * The equilibrium Green's functions of n_inst independent sectors (for
 * example the repeated impurity solves of DMFT/VCA-type embedding schemes,
 * Section 1), computed together: after each instance's ground state, the
 * columns of all instances -- of different dimensions -- are propagated in
 * the same launches (one CUDA graph per time step, work lists sized to fill
 * the GPU, a work-list scale chosen by a short timing run).  Same orbitals,
 * dt and n_steps for all instances.
 *   G_gtr, G_les: host, complex [n_inst][n_steps+1][n_orb][n_orb];
 *   status: host int[n_inst] (may be NULL): KG_OK, or the error of that
 *           instance's ground state (KG_ENOCONV, KG_EDEGEN, ...) or
 *           KG_ENUMERIC; the G of a failed instance is left zero.
 * Returns KG_OK unless an argument is invalid or the device fails. */
int kg_green_equilibrium_batched(kg_sector* const* s, int n_inst, const int* orb, int n_orb, double dt,
                                 int n_steps, const kg_opts* o, double* G_gtr, double* G_les, int* status);

/* ---- adjoint of the equilibrium Green's function ----------------------
 * Vector-Jacobian product of kg_green_equilibrium with respect to the
 * Hamiltonian parameters (not in the paper; built on the structure of its
 * propagation, Section 3).  For a real loss L of the returned G, the caller
 * passes the cotangents dG_gtr, dG_les (host, complex [n_steps+1][n_orb]
 * [n_orb], entry = dL/dRe G + i dL/dIm G; either may be NULL = zero) and
 * receives, on the host,
 *   g_eps[sigma*L + i] = dL/d eps_{i sigma},     g_U[i] = dL/dU_i,
 *   g_hre[i*L + j] = dL/dRe h_ij  (h_ji = conj(h_ij) tied, so symmetric;
 *                    the diagonal is dL/dh_ii = sum over spins of g_eps),
 *   g_him[i*L + j] = dL/dIm h_ij  (antisymmetric),
 * for the bonds of the model (pairs i != j with h_ij != 0, whose hops the
 * sector tables hold) and the diagonal; entries of pairs absent from the
 * model are returned as zero (a caller that needs the derivative with respect
 * to a new bond passes that bond with a tiny nonzero amplitude).
 * Method: adjoint states propagated backward with the same Krylov steps,
 * Frechet derivative of each step by 10-point Gauss-Legendre quadrature with
 * node vectors from that step's Krylov spaces, ground-state terms by
 * Hellmann-Feynman and one projected conjugate-gradient solve.  Forward
 * states are checkpointed every `checkpoint` steps (0 = 20) and recomputed.
 * The quadrature is exact to rounding when |dt| times the spectral width of
 * the sectors is below about 3.  Other arguments as for
 * kg_green_equilibrium. */
int kg_green_equilibrium_vjp(kg_sector* s, const int* orb, int n_orb, double dt, int n_steps, const kg_opts* o,
                             int checkpoint, const double* dG_gtr, const double* dG_les, double* g_eps,
                             double* g_hre, double* g_him, double* g_U);

/* ---- nonequilibrium (Keldysh) Green's function -----------------------
 * Section 4, steps (i)-(iv): |0> = ground state of H_ini; Phi(t) =
 * e^{-iH t}|0> with H = H_fin; Psi_a(t) = e^{iHt} c_a Phi(t) and
 * chi_a(t) = e^{iHt} c^dag_a Phi(t); then for t_k = k*dt, k < n_t,
 *   G_les[k][l][a][a'] = +i <Psi_a'(t_l) | Psi_a(t_k)>
 *   G_gtr[k][l][a][a'] = -i <chi_a(t_k) | chi_a'(t_l)>.
 * H_ini and H_fin must have the same (L, N_up, N_dn), else KG_EINVAL.
 * opts->dt_internal splits every grid step into round(dt/dt_internal)
 * Krylov steps.  G_les, G_gtr: host, complex [n_t][n_t][n_orb][n_orb]. */
int kg_green_keldysh(kg_sector* H_ini, kg_sector* H_fin, const int* orb, int n_orb, double dt,
                     int n_t, const kg_opts* o, double* G_les, double* G_gtr);

/* The same computation in stages, so that a caller can schedule the rows of
 * step (iii) itself.  kg_keldysh_create runs steps (i) and (ii) and keeps
 * Phi(t_k) for all k.  kg_keldysh_row runs step (iii) for one time index k
 * -- every Psi_a(t_k) and chi_a(t_k) of the orbital list, batched -- stores
 * them, and writes the time-diagonal block G(t_k, t_k) (host, complex
 * [n_orb][n_orb] each; either pointer may be NULL).  kg_keldysh_gram runs
 * step (iv) over all stored rows (rows never computed give KG_EINVAL) into
 * arrays shaped like kg_green_keldysh's.
 *
 * Memory plan (decided at creation against opts->mem_budget_mb, or the free
 * device memory): Phi(t_k) stays on the device when it fits beside the
 * largest (spin, kind) block's columns and Krylov workspace, else it is kept
 * in host memory (pinned when possible) and one Phi(t_k) at a time is copied
 * to the device.  When the columns of all blocks do not fit together, rows
 * still return their time-diagonal blocks but keep no columns, and
 * kg_keldysh_gram returns KG_EINVAL: kg_green_keldysh then computes the whole
 * grid one block at a time (one block's columns and workspace resident).
 * The Krylov workspaces drop their Gram-Schmidt planes (same results, slower)
 * when the planes do not fit.  kg_keldysh_plan reports the decisions:
 * phi_on_host 0 (device), 1 (pinned host) or 2 (pageable host); stores_kept
 * 1 when kg_keldysh_gram is available; planes 1 when the staged rows use
 * them; budget the byte budget planned against (any pointer may be NULL). */
int kg_keldysh_create(kg_sector* H_ini, kg_sector* H_fin, const int* orb, int n_orb, double dt,
                      int n_t, const kg_opts* o, kg_keldysh** out);
int kg_keldysh_row(kg_keldysh* K, int k, double* G_les_kk, double* G_gtr_kk);
int kg_keldysh_gram(kg_keldysh* K, double* G_les, double* G_gtr);
int kg_keldysh_plan(const kg_keldysh* K, int* phi_on_host, int* stores_kept, int* planes, long long* budget);
/* ---- driven Hamiltonian after the quench ----------------------------------
 * Section 6 (outlook): a Hamiltonian with a general time dependence after
 * t = 0, propagated by a higher-order commutator-free exponential integrator.
 * H(t) = H_fin + sum_{i,sigma} de_{i sigma}(t) n_{i sigma}
 *              + sum_i dU_i(t) n_{i up} n_{i dn}
 * (on-site energy and interaction offsets; hoppings fixed).  Every grid step
 * is split into n_sub = max(1, round(dt / opts->dt_internal)) internal steps
 * of h = dt / n_sub (n_sub = 1 when dt_internal <= 0), each propagated by the
 * fourth-order commutator-free step with two exponentials,
 *   U(t + h, t) = e^{-i h (a1 A_1 + a2 A_2)} e^{-i h (a2 A_1 + a1 A_2)},
 * A_{1,2} = H(t + (1/2 -+ sqrt(3)/6) h), a1 = (3 - 2 sqrt(3))/12,
 * a2 = (3 + 2 sqrt(3))/12 (right factor first), each exponential one Krylov
 * step of h/2 with opts->M vectors; the error of G falls as h^4.
 * dparams: host, [(n_t - 1) n_sub][2][3L] doubles: for internal step s and
 * node j (the two times above, t = s h) the offsets de_{i up} (L values),
 * de_{i dn} (L), dU_i (L).  It may be NULL only when n_t == 1.  G_les and
 * G_gtr as in kg_green_keldysh, with Phi(t_k) = U(t_k, 0)|0>, Psi_a(t_k) =
 * U(t_k, 0)^dag c_a Phi(t_k), chi_a(t_k) = U(t_k, 0)^dag c^dag_a Phi(t_k).
 * Constant offsets reproduce kg_green_keldysh for H_fin with the offsets
 * added.  KG_EINVAL for a non-finite offset or the kg_green_keldysh cases.
 * kg_keldysh_create_td is the staged form (rows, Gram, plan, Phi as for
 * kg_keldysh_create). */
int kg_green_keldysh_td(kg_sector* H_ini, kg_sector* H_fin, const int* orb, int n_orb, double dt, int n_t,
                        const double* dparams, const kg_opts* o, double* G_les, double* G_gtr);
int kg_keldysh_create_td(kg_sector* H_ini, kg_sector* H_fin, const int* orb, int n_orb, double dt, int n_t,
                         const double* dparams, const kg_opts* o, kg_keldysh** out);

/* ---- four-time correlation functions -------------------------------------
 * Section 6 (outlook): higher-order Green's functions with four independent
 * time arguments, by the Krylov steps of Section 4.  After the quench,
 *   G[k1][k2][k3][k4] = <0| A1(t1) A2(t2) A3(t3) A4(t4) |0>,  t_k = k dt, k < n_t,
 * A(t) = e^{iHt} A e^{-iHt} with H = H_fin, |0> the ground state of H_ini
 * (H_ini = H_fin gives the equilibrium function).  ops: host, 12 ints, the
 * four operators as (site, spin, dagger) with dagger 1 for c^dag, 0 for c.
 * Computed as <L(t1,t2) | R(t3,t4)> with R = e^{iH t3} A3 e^{-iH(t3-t4)} A4
 * Phi(t4) and L = e^{iH t2} A2^dag e^{-iH(t2-t1)} A1^dag Phi(t1), Phi(t) =
 * e^{-iHt}|0>; every grid step is round(dt / opts->dt_internal) Krylov
 * steps (one when dt_internal <= 0).  Device memory: Phi on n_t times and
 * 2 n_t^2 vectors of the target sector, plus Krylov workspaces of n_t
 * columns (KG_ENOMEM when they do not fit).  G: host complex [n_t]^4,
 * zero when the operators change the particle numbers.  KG_EINVAL for a bad
 * operator, n_t < 1, negative or non-finite dt, or sectors that differ. */
int kg_green_four_time(kg_sector* H_ini, kg_sector* H_fin, const int* ops, double dt, int n_t, const kg_opts* o,
                       double* G);

/* ---- nonequilibrium cluster-perturbation theory ---------------------------
 * Section 5, Eq. (cpteq) with the bath of Eqs. (gb1), (gb2): the cluster of
 * H_ini / H_fin (L sites; its last site L-1) coupled by the hopping V to the
 * first site of a non-interacting chain of L_b sites with hopping -T_b
 * (on-site energies and chemical potential 0; a half-filled, particle-hole
 * symmetric bath).  G = (G'^{-1} - V)^{-1} is solved on the contour
 * 0 -> t_max -> 0 -> -i beta, t_max = (n_t - 1) dt, discretised by the
 * trapezoidal rule on t_k = k dt and tau_j = j beta / n_tau (2 n_t + n_tau + 1
 * points, at most 3072).  The cluster functions at inverse temperature beta
 * are built from the zero-temperature components of this library
 * (kg_green_keldysh, kg_green_mixed, kg_green_matsubara_steps with mu = 0,
 * opts as given) plus the antiperiodic tails of the imaginary branch; terms of
 * relative size e^{-beta gap} of the cluster are dropped, so beta must be
 * large against the inverse gap.  The bath integrated out, the coupled site's
 * contour equation is solved by an LU factorisation on the device.
 * n_out: host, [2][n_t][L] doubles, n_out[s][k][i] = n_{i s}(t_k) = -i
 * G^<_{ii}(t_k, t_k) of the coupled system (spin s = 0 up, 1 down).
 * KG_EINVAL for bad sizes (L_b < 1, n_t < 1, n_tau < 2, dt < 0, beta <= 0,
 * non-finite values, too many contour points) or differing sectors;
 * KG_ENUMERIC if the contour matrix is singular; the errors of the component
 * calls otherwise.  Discretisation error: second order in dt and dtau. */
int kg_necpt_occupations(kg_sector* H_ini, kg_sector* H_fin, int L_b, double T_b, double V, double dt, int n_t,
                         double beta, int n_tau, const kg_opts* o, double* n_out);

/* ---- mixed components on the imaginary branch ---------------------------
 * Section 4, the remark after step (iv): the components of the contour
 * Green's function with one time on the imaginary branch, at zero
 * temperature with the initial ground state |0> of H_ini and K = H_ini - mu N
 * there (the imaginary time later on the contour):
 *   G_right[k][j][a][a'] = G^right_{aa'}(t_k, tau_j) = +i <xi_a'(tau_j) | Psi_a(t_k)>,
 *   G_left[j][k][a][a']  = G^left_{aa'}(tau_j, t_k)  = -i <zeta_a(tau_j) | chi_a'(t_k)>,
 * xi_a(tau) = e^{-(H_ini - E0 + mu) tau} c_a|0>, zeta_a(tau) =
 * e^{-(H_ini - E0 - mu) tau} c^dag_a|0> on tau_j = j dtau, j = 0..n_tau (the
 * imaginary-time Krylov steps of kg_green_matsubara_steps, o->M vectors per
 * step), and Psi_a, chi_a the step-(iii) columns of kg_green_keldysh on
 * t_k = k dt, k < n_t.  G_right: host complex [n_t][n_tau+1][n_orb][n_orb];
 * G_left: host complex [n_tau+1][n_t][n_orb][n_orb].  KG_EINVAL for bad
 * arguments (as kg_green_keldysh, plus n_tau >= 0, finite dtau > 0 and mu),
 * KG_ENOMEM when the Keldysh columns of all blocks do not fit together (see
 * the memory plan below). */
int kg_green_mixed(kg_sector* H_ini, kg_sector* H_fin, const int* orb, int n_orb, double dt, int n_t, double mu,
                   double dtau, int n_tau, const kg_opts* o, double* G_right, double* G_left);

/* Host copy of Phi(t_k) (complex, dimension d), and the reverse: replaces
 * the stored Phi(t_k) by a host vector (used to time a row end to end). */
int kg_keldysh_get_phi(kg_keldysh* K, int k, double* phi_host);
int kg_keldysh_set_phi(kg_keldysh* K, int k, const double* phi_host);
void kg_keldysh_free(kg_keldysh* K);

/* ---- measurement (not part of the method) ---------------------------------
 * kg_profile_start/stop bracket a region in which every kernel launch of
 * this library is timed with CUDA events on its launch stream (CUDA graphs
 * are not used while profiling).  After stop, kg_profile_count entries are
 * available: kernel name (copied into name[len]), number of launches and
 * total milliseconds.  kg_probe_fp64 runs a dependent-FMA-free FP64 kernel on
 * the current device and reports the FMA throughput in TFLOP/s (2 flops per
 * FMA); stream as for kg_hpsi. */
int kg_profile_start(void);
int kg_profile_stop(void);
int kg_profile_count(void);
int kg_profile_get(int i, char* name, int len, long long* launches, double* ms);
int kg_probe_fp64(double* tflops, void* stream);

/* ---- utilities ----------------------------------------------------------- */
const char* kg_strerror(int code);
const char* kg_last_error(void);

/* Number of kernel launches this library has issued since load (graph
 * replays count their kernels); a counter for benchmark bookkeeping. */
unsigned long long kg_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* KRYLOVGF_H */
