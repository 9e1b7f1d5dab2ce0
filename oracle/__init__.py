"""CPU FP64 oracle for the Krylov-space Green's-function method.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline legs of bench.py may import this package.  The CUDA library never
calls it, and it shares no code, table or helper with the CUDA path.

The heavy loops live in kg_oracle.cpp (basis, H*psi, c/c^dag, Lanczos ground
state, Chebyshev propagator).  This module assembles the Green's functions
exactly as the paper defines them:

* equilibrium, Section 3, Eqs. (psit) and (psigreen), plus the hole part
  given after Eq. (gomega):
      G^>_{aa'}(t) = -i e^{+i E0 t} < c^dag_a 0 | e^{-iHt} | c^dag_a' 0 >
      G^<_{aa'}(t) = +i e^{-i E0 t} < c_a' 0 | e^{+iHt} | c_a 0 >
  (eta = 0; the retarded function is G^> - G^< for t >= 0);
* nonequilibrium, Section 4, steps (i)-(iv):
      |0> = ground state of H_ini, Phi(t) = e^{-iHt}|0>,
      Psi_a(t) = e^{iHt} c_a Phi(t),  chi_a(t) = e^{iHt} c^dag_a Phi(t),
      G^<_{aa'}(t,t') = i <Psi_a'(t') | Psi_a(t)>,
      G^>_{aa'}(t,t') = -i <chi_a(t) | chi_a'(t')>;
* G(omega) from G(t): the damped Fourier transform of Section 3 (trapezoidal
  rule on the sampled times);
* the Matsubara and mixed components named after step (iv) of Section 4, at
  zero temperature with a chemical potential mu on the imaginary branch
  (imaginary-time propagators from dense eigen-decompositions, small sectors);
* the NE-CPT of Section 5 (Eq. (cpteq), the bath of Eqs. (gb1), (gb2)) on a
  trapezoidal Keldysh-Matsubara contour;
* the two directions of the outlook in Section 6: a driven H(t) by the
  fourth-order commutator-free exponential step, and four-time correlation
  functions.

Every propagation here is a Chebyshev expansion over the whole interval
(never the GPU's restarted Krylov steps), so the two sides are independent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kg_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libkgoracle.so")
_lib = None


def build(force=False):
    """Compile the C++ oracle into oracle/_build/libkgoracle.so with g++."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.ko_model_new.restype = P
    lib.ko_model_new.argtypes = [I, I, I, P, P, P, P]
    lib.ko_model_free.argtypes = [P]
    lib.ko_model_dim.restype = ctypes.c_long
    lib.ko_model_dim.argtypes = [P]
    lib.ko_model_basis.argtypes = [P, P]
    lib.ko_model_bounds.argtypes = [P, P, P]
    lib.ko_num_threads.restype = I
    lib.ko_set_num_threads.argtypes = [I]
    lib.ko_hpsi.argtypes = [P, P, P]
    lib.ko_dense_h.argtypes = [P, P]
    lib.ko_apply_cop.restype = I
    lib.ko_apply_cop.argtypes = [P, P, I, I, I, P, P]
    lib.ko_ground_state.restype = I
    lib.ko_ground_state.argtypes = [P, I, I, D, ctypes.c_ulonglong, P, P, P]
    lib.ko_propagate.restype = I
    lib.ko_propagate.argtypes = [P, P, D, P]
    _lib = lib
    return lib


def num_threads():
    return _load().ko_num_threads()


def set_num_threads(n):
    _load().ko_set_num_threads(int(n))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Sector:
    """One (N_up, N_dn) sector of a model (see workloads.make_model)."""

    def __init__(self, model, n_up=None, n_dn=None):
        lib = _load()
        self.model = model
        self.L = model["L"]
        self.n_up = model["n_up"] if n_up is None else n_up
        self.n_dn = model["n_dn"] if n_dn is None else n_dn
        self._h_re = np.ascontiguousarray(model["h"].real, dtype=np.float64)
        self._h_im = np.ascontiguousarray(model["h"].imag, dtype=np.float64)
        self._eps = np.ascontiguousarray(model["eps"], dtype=np.float64)
        self._U = np.ascontiguousarray(model["U"], dtype=np.float64)
        self.h = lib.ko_model_new(self.L, self.n_up, self.n_dn, _ptr(self._h_re), _ptr(self._h_im),
                                  _ptr(self._eps), _ptr(self._U))
        if not self.h:
            raise ValueError("invalid sector")
        self.dim = int(lib.ko_model_dim(self.h))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ko_model_free(self.h)
            self.h = None

    def basis(self):
        out = np.empty(self.dim, dtype=np.uint64)
        _load().ko_model_basis(self.h, _ptr(out))
        return out

    def bounds(self):
        lo, hi = ctypes.c_double(), ctypes.c_double()
        _load().ko_model_bounds(self.h, ctypes.byref(lo), ctypes.byref(hi))
        return lo.value, hi.value

    def hpsi(self, x):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.empty_like(x)
        _load().ko_hpsi(self.h, _ptr(x), _ptr(y))
        return y

    def neighbour(self, spin, dagger):
        du = (1 if dagger else -1) if spin == 0 else 0
        dd = (1 if dagger else -1) if spin == 1 else 0
        nu, nd = self.n_up + du, self.n_dn + dd
        if nu < 0 or nd < 0 or nu > self.L or nd > self.L:
            return None
        return Sector(self.model, nu, nd)

    def apply_cop(self, dst, site, spin, dagger, x):
        """y = c_{site,spin} x (dagger False) or c^dag x, y in sector dst."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.empty(dst.dim, dtype=np.complex128)
        rc = _load().ko_apply_cop(self.h, dst.h, site, spin, 1 if dagger else 0, _ptr(x), _ptr(y))
        if rc != 0:
            raise ValueError("bad sector pair for c/c^dag")
        return y

    def ground_state(self, K=80, max_restarts=60, tol=1e-12, seed=1234):
        """(E0, |0>, residual) by restarted Lanczos with full reorthogonalisation."""
        psi = np.empty(self.dim, dtype=np.complex128)
        e0, res = ctypes.c_double(), ctypes.c_double()
        rc = _load().ko_ground_state(self.h, K, max_restarts, tol, seed, ctypes.byref(e0), _ptr(psi),
                                     ctypes.byref(res))
        if rc < 0:
            raise ValueError("empty sector")
        return e0.value, psi, res.value

    def propagate(self, x, tau):
        """exp(-i H tau) x (tau may be negative) by a Chebyshev expansion."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.empty_like(x)
        _load().ko_propagate(self.h, _ptr(x), float(tau), _ptr(y))
        return y


def _groups(orbitals):
    return {s: [k for k, (_, sp) in enumerate(orbitals) if sp == s] for s in (0, 1)}


def green_equilibrium(model, orbitals, dt, n_steps, gs=None, K=80, tol=1e-12):
    """Equilibrium G^>(t_k), G^<(t_k) for t_k = k*dt, k = 0..n_steps.

    Returns (G_gtr, G_les, E0), each G of shape [n_steps+1, n_orb, n_orb]
    (complex) with G[k, a, a'] = G_{a a'}(t_k).  Entries with different spins
    vanish (S_z is conserved).  Time stepping uses exp(-iH dt) repeatedly, each
    step one Chebyshev expansion (Section 3, Eq. (psigreen) with eta = 0).
    """
    sec = Sector(model)
    E0, psi0, _ = sec.ground_state(K=K, tol=tol) if gs is None else gs
    n = len(orbitals)
    t = dt * np.arange(n_steps + 1)
    G_gtr = np.zeros((n_steps + 1, n, n), dtype=np.complex128)
    G_les = np.zeros_like(G_gtr)
    for spin, idx in _groups(orbitals).items():
        if not idx:
            continue
        for dagger, G in ((True, G_gtr), (False, G_les)):
            nb = sec.neighbour(spin, dagger)
            if nb is None:
                continue
            vecs = {a: sec.apply_cop(nb, orbitals[a][0], spin, dagger, psi0) for a in idx}
            for p in idx:
                # particle part: cur = e^{-iHt} c^dag_p |0>, and
                #   G^>_{a p}(t) = -i e^{iE0 t} <c^dag_a 0 | cur>;
                # hole part: cur = e^{+iHt} c_p |0>, and
                #   G^<_{p a}(t) = +i e^{-iE0 t} <c_a 0 | cur>.
                cur = vecs[p].copy()
                for k in range(n_steps + 1):
                    for a in idx:
                        ov = np.vdot(vecs[a], cur)
                        if dagger:
                            G[k, a, p] = -1j * np.exp(1j * E0 * t[k]) * ov
                        else:
                            G[k, p, a] = 1j * np.exp(-1j * E0 * t[k]) * ov
                    if k < n_steps:
                        cur = nb.propagate(cur, dt if dagger else -dt)
    return G_gtr, G_les, E0


def lanczos_run(sector, v0, n):
    """n steps of the Lanczos recursion of Eq. (recursion) from v0 with full
    reorthogonalisation (modified Gram-Schmidt, twice, against every stored
    vector).  Returns (a, b, norm0): the diagonal a_0..a_{m-1}, the couplings
    b_1..b_{m-1} (b[j-1] couples vectors j-1 and j) and ||v0||; m <= n is
    smaller after an invariant subspace is reached."""
    norm0 = float(np.linalg.norm(v0))
    a, b = [], []
    if norm0 == 0.0:
        return np.zeros(0), np.zeros(0), 0.0
    V = [v0 / norm0]
    for j in range(n):
        w = sector.hpsi(V[j])
        if j > 0:
            w = w - b[-1] * V[j - 1]
        aj = float(np.vdot(V[j], w).real)
        w = w - aj * V[j]
        for _ in range(2):
            for v in V:
                w = w - np.vdot(v, w) * v
        a.append(aj)
        if j + 1 == n:
            break
        bj = float(np.linalg.norm(w))
        if bj <= 1e-12 * (abs(aj) + (b[-1] if b else 0.0)):
            break
        b.append(bj)
        V.append(w / bj)
    return np.array(a), np.array(b), norm0


def green_lanczos(model, orbitals, n, omega, eta, gs=None, K=80, tol=1e-12):
    """The Lanczos Green's function of Eq. (gapprox) for diagonal orbitals:
    a second Lanczos run of n steps from c^dag_a|0> (particle part) or c_a|0>
    (hole part), its Ritz pairs (E_m, |m>) from the tridiagonal matrix
    (Eq. (eigen)), and the n-pole sum
        G^>_a(w) = sum_m |<m|c^dag_a 0>|^2 / (w + i eta - E_m + E0),
        G^<_a(w) = sum_m |<m|c_a 0>|^2 / (w + i eta + E_m - E0),
    with <m|c^dag_a 0> = ||c^dag_a 0|| (Q)_{0m}.  Returns (G_gtr, G_les, E0),
    each G of shape [n_orb, len(omega)]."""
    sec = Sector(model)
    E0, psi0, _ = sec.ground_state(K=K, tol=tol) if gs is None else gs
    omega = np.asarray(omega, dtype=np.float64)
    G_gtr = np.zeros((len(orbitals), omega.size), dtype=np.complex128)
    G_les = np.zeros_like(G_gtr)
    for i, (site, spin) in enumerate(orbitals):
        for dagger, G in ((True, G_gtr), (False, G_les)):
            nb = sec.neighbour(spin, dagger)
            if nb is None:
                continue
            v0 = sec.apply_cop(nb, site, spin, dagger, psi0)
            a, b, norm0 = lanczos_run(nb, v0, n)
            if norm0 == 0.0:
                continue
            T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
            Em, Q = np.linalg.eigh(T)
            wgt = (norm0 * Q[0, :]) ** 2
            for m in range(len(Em)):
                if dagger:
                    G[i] += wgt[m] / (omega + 1j * eta - Em[m] + E0)
                else:
                    G[i] += wgt[m] / (omega + 1j * eta + Em[m] - E0)
    return G_gtr, G_les, E0


def green_fourier(G_t, dt, omega, eta):
    """G(omega) from a sampled G(t) (Section 3: Fourier transformation of the
    time-dependent Green's function, made convergent at t_max by the damping
    e^{-eta t} of the broadening).  The time integral over [0, (n_t-1) dt] is
    the trapezoidal rule on t_k = k dt:
        G(omega) = sum_k w_k e^{i (omega + i eta) t_k} G(t_k),
        w_0 = w_{n_t-1} = dt/2, w_k = dt otherwise (no interval: zero).
    G_t: complex [n_series, n_t] or [n_t]; returns [n_series, n_omega] or
    [n_omega]."""
    g = np.asarray(G_t, dtype=np.complex128)
    one = g.ndim == 1
    g = g.reshape(1, -1) if one else g
    omega = np.asarray(omega, dtype=np.float64).ravel()
    n_t = g.shape[1]
    out = np.zeros((g.shape[0], omega.size), dtype=np.complex128)
    if n_t >= 2:
        t = dt * np.arange(n_t)
        w = np.full(n_t, float(dt))
        w[0] = w[-1] = 0.5 * dt
        kernel = np.exp(1j * np.outer(omega + 1j * eta, t))  # [n_omega, n_t]
        out = (g * w) @ kernel.T
    return out[0] if one else out


def keldysh_vectors(ini, fin, orbitals, dt, n_t, gs=None, K=80, tol=1e-12):
    """Steps (i)-(iii) of Section 4: returns (E0, Phi, Psi, Chi).

    Phi[k] = e^{-iH t_k}|0>, Psi[s][k][a] = e^{iH t_k} c_a Phi(t_k) and
    Chi[s][k][a] = e^{iH t_k} c^dag_a Phi(t_k) for the orbitals of spin s.
    Each back-propagation is one Chebyshev expansion over the full time t_k.
    """
    sec_i = Sector(ini)
    E0, psi0, _ = sec_i.ground_state(K=K, tol=tol) if gs is None else gs
    sec_f = Sector(fin)
    t = dt * np.arange(n_t)
    Phi = [psi0.copy()]
    for k in range(1, n_t):
        Phi.append(sec_f.propagate(Phi[-1], dt))
    Psi, Chi = {}, {}
    for spin, idx in _groups(orbitals).items():
        if not idx:
            continue
        for dagger, store in ((False, Psi), (True, Chi)):
            nb = sec_f.neighbour(spin, dagger)
            if nb is None:
                continue
            store[spin] = [[nb.propagate(sec_f.apply_cop(nb, orbitals[a][0], spin, dagger, Phi[k]), -t[k])
                            for a in idx] for k in range(n_t)]
    return E0, Phi, Psi, Chi


def green_keldysh(ini, fin, orbitals, dt, n_t, gs=None, K=80, tol=1e-12):
    """G^<(t_k,t_l), G^>(t_k,t_l) of Section 4, shape [n_t, n_t, n_orb, n_orb].

    G[k, l, a, a'] = G_{a a'}(t_k, t_l); step (iv) is a plain Gram matrix.
    """
    E0, Phi, Psi, Chi = keldysh_vectors(ini, fin, orbitals, dt, n_t, gs=gs, K=K, tol=tol)
    n = len(orbitals)
    G_les = np.zeros((n_t, n_t, n, n), dtype=np.complex128)
    G_gtr = np.zeros_like(G_les)
    for spin, idx in _groups(orbitals).items():
        if spin in Psi:
            for k in range(n_t):
                for l in range(n_t):
                    for ia, a in enumerate(idx):
                        for ib, b in enumerate(idx):
                            G_les[k, l, a, b] = 1j * np.vdot(Psi[spin][l][ib], Psi[spin][k][ia])
        if spin in Chi:
            for k in range(n_t):
                for l in range(n_t):
                    for ia, a in enumerate(idx):
                        for ib, b in enumerate(idx):
                            G_gtr[k, l, a, b] = -1j * np.vdot(Chi[spin][k][ia], Chi[spin][l][ib])
    return G_les, G_gtr, E0


def dense_hamiltonian(sector):
    """The sector Hamiltonian as a dense matrix (small sectors only): every
    term of H*psi written to its own entry, H[s, k] = <s|H|k>."""
    d = sector.dim
    if d > 5000:
        raise ValueError("dense_hamiltonian is for sectors of dimension <= 5000")
    H = np.empty((d, d), dtype=np.complex128)
    _load().ko_dense_h(sector.h, _ptr(H))
    return H


def _imaginary_time_vectors(sector, x, taus, shift):
    """e^{-(H - shift) tau} x for every tau of taus, from the eigen-
    decomposition of the dense sector H: rows of the returned array."""
    w, Q = np.linalg.eigh(dense_hamiltonian(sector))
    px = Q.conj().T @ x
    return np.stack([Q @ (np.exp(-(w - shift) * tau) * px) for tau in taus])


def green_matsubara(model, orbitals, taus, mu, gs=None, K=80, tol=1e-12):
    """The Matsubara function of the initial-state Hamiltonian at zero
    temperature (Section 4, after step (iv): G^M(tau, tau') = G^M(tau - tau'),
    the equilibrium Green's function of H_ini on the imaginary branch), with
    the chemical potential mu in K = H - mu N:
        G^M_{aa'}(+tau) = -<0| c_a e^{-(H - E0 - mu) tau} c^dag_a' |0>,
        G^M_{aa'}(-tau) = +<0| c^dag_a' e^{-(H - E0 + mu) tau} c_a |0>,
    for tau >= 0 (the two one-sided limits at tau = 0).  The imaginary-time
    propagators come from the eigen-decomposition of the dense neighbour-
    sector H (small sectors).  Returns (G_plus, G_minus, E0), each
    [n_tau, n_orb, n_orb] with G_plus[j] = G^M(tau_j), G_minus[j] =
    G^M(-tau_j)."""
    sec = Sector(model)
    E0, psi0, _ = sec.ground_state(K=K, tol=tol) if gs is None else gs
    taus = np.asarray(taus, dtype=np.float64).ravel()
    n = len(orbitals)
    G_plus = np.zeros((taus.size, n, n), dtype=np.complex128)
    G_minus = np.zeros_like(G_plus)
    for spin, idx in _groups(orbitals).items():
        if not idx:
            continue
        for dagger in (True, False):
            nb = sec.neighbour(spin, dagger)
            if nb is None:
                continue
            vecs = {a: sec.apply_cop(nb, orbitals[a][0], spin, dagger, psi0) for a in idx}
            shift = E0 + mu if dagger else E0 - mu
            for p in idx:
                prop = _imaginary_time_vectors(nb, vecs[p], taus, shift)  # [n_tau, d]
                for a in idx:
                    ov = prop @ vecs[a].conj()  # <vecs[a] | prop(tau)>
                    if dagger:
                        G_plus[:, a, p] = -ov
                    else:
                        G_minus[:, p, a] = ov
    return G_plus, G_minus, E0


def green_mixed(ini, fin, orbitals, dt, n_t, taus, mu, gs=None, K=80, tol=1e-12):
    """The mixed real/imaginary-time components of Section 4 (after step
    (iv)) at zero temperature, initial state |0> of H_ini, K = H_ini - mu N on
    the imaginary branch:
        G^right_{aa'}(t_k, tau_j) = +i <xi_a'(tau_j) | Psi_a(t_k)>,
        G^left_{aa'}(tau_j, t_k)  = -i <zeta_a(tau_j) | chi_a'(t_k)>,
    with Psi_a(t) = e^{iHt} c_a Phi(t), chi_a(t) = e^{iHt} c^dag_a Phi(t) of
    steps (ii)-(iii) (H = H_fin) and the imaginary-time vectors
        xi_a(tau) = e^{-(H_ini - E0 + mu) tau} c_a |0>,
        zeta_a(tau) = e^{-(H_ini - E0 - mu) tau} c^dag_a |0>.
    Returns (G_right [n_t, n_tau, n, n], G_left [n_tau, n_t, n, n], E0)."""
    sec_i = Sector(ini)
    E0, psi0, _ = sec_i.ground_state(K=K, tol=tol) if gs is None else gs
    _, _, Psi, Chi = keldysh_vectors(ini, fin, orbitals, dt, n_t, gs=(E0, psi0, 0.0))
    taus = np.asarray(taus, dtype=np.float64).ravel()
    n = len(orbitals)
    G_right = np.zeros((n_t, taus.size, n, n), dtype=np.complex128)
    G_left = np.zeros((taus.size, n_t, n, n), dtype=np.complex128)
    for spin, idx in _groups(orbitals).items():
        for dagger, store in ((False, Psi), (True, Chi)):
            if spin not in store:
                continue
            nb = sec_i.neighbour(spin, dagger)
            shift = E0 + mu if dagger else E0 - mu
            imag = {a: _imaginary_time_vectors(nb, sec_i.apply_cop(nb, orbitals[a][0], spin, dagger, psi0), taus,
                                               shift) for a in idx}
            for k in range(n_t):
                for ia, a in enumerate(idx):
                    for ib, b in enumerate(idx):
                        if not dagger:  # G^right_{ab}(t_k, tau) = i <xi_b(tau) | Psi_a(t_k)>
                            G_right[k, :, a, b] = 1j * (imag[b].conj() @ store[spin][k][ia])
                        else:  # G^left_{ab}(tau, t_k) = -i <zeta_a(tau) | chi_b(t_k)>
                            G_left[:, k, a, b] = -1j * (imag[a].conj() @ store[spin][k][ib])
    return G_right, G_left, E0


def keldysh_entry(ini, fin, orbital_a, orbital_b, dt, k, l, gs=None, K=80, tol=1e-12):
    """One sampled pair (G^<_{ab}(t_k,t_l), G^>_{ab}(t_k,t_l)) at any size.

    Only Phi(t_k), Phi(t_l) and four back-propagated vectors are formed, so a
    single entry of a large Keldysh grid can be checked one by one.
    """
    sec_i = Sector(ini)
    E0, psi0, _ = sec_i.ground_state(K=K, tol=tol) if gs is None else gs
    sec_f = Sector(fin)
    (sa, pa), (sb, pb) = orbital_a, orbital_b
    if pa != pb:
        return 0j, 0j
    tk, tl = dt * k, dt * l
    phi_k = sec_f.propagate(psi0, tk) if k else psi0
    phi_l = sec_f.propagate(psi0, tl) if l else psi0
    out = []
    for dagger in (False, True):
        nb = sec_f.neighbour(pa, dagger)
        if nb is None:
            out.append(0j)
            continue
        va = nb.propagate(sec_f.apply_cop(nb, sa, pa, dagger, phi_k), -tk)
        vb = nb.propagate(sec_f.apply_cop(nb, sb, pb, dagger, phi_l), -tl)
        out.append(1j * np.vdot(vb, va) if not dagger else -1j * np.vdot(va, vb))
    return out[0], out[1]


def _eigh(H):
    """eigh of a Hermitian matrix, in real arithmetic when H is real."""
    if not np.any(H.imag):
        return np.linalg.eigh(H.real)
    return np.linalg.eigh(H)


def _sandwich(Q, Z):
    """conj(Q) Z Q^T (real products when Q is real)."""
    if np.isrealobj(Q):
        return (Q @ Z.real @ Q.T) + 1j * (Q @ Z.imag @ Q.T)
    return Q.conj() @ Z @ Q.T


def _divided_differences(g, dg, E, tol=1e-6):
    """D[m, n] = (g(E_m) - g(E_n)) / (E_m - E_n), the first divided
    difference of a function known on the eigenvalues E (values g, derivatives
    dg); pairs closer than tol take the mean derivative instead."""
    diff = E[:, None] - E[None, :]
    close = np.abs(diff) <= tol
    D = (g[:, None] - g[None, :]) / np.where(close, 1.0, diff)
    return np.where(close, 0.5 * (dg[:, None] + dg[None, :]), D)


def _unit_model(model, kind, i, j=None):
    """The model whose Hamiltonian is dH/dtheta for one parameter theta (H is
    linear in h, eps and U): kind 'eps' (theta = eps[i, j] with i the spin),
    'U' (U_i), 're' / 'im' (the real / imaginary part of h_ij with h_ji tied
    to its conjugate; i == j is the diagonal h_ii)."""
    L = model["L"]
    h = np.zeros((L, L), dtype=np.complex128)
    eps = np.zeros((2, L))
    U = np.zeros(L)
    if kind == "eps":
        eps[i, j] = 1.0
    elif kind == "U":
        U[i] = 1.0
    elif kind == "re":
        h[i, j] += 1.0
        if i != j:
            h[j, i] += 1.0
    else:
        h[i, j] += 1j
        h[j, i] -= 1j
    m = dict(model)
    m["h"], m["eps"], m["U"] = h, eps, U
    return m


def green_equilibrium_grad_dense(model, orbitals, dt, n_steps, dG_gtr=None, dG_les=None):
    """Analytic gradient of a real loss L of the equilibrium Green's function
    (Section 3, Eq. (psigreen) with eta = 0, and the hole part after Eq.
    (gomega)) with respect to the Hamiltonian parameters, from the dense
    eigen-decompositions of the sector and neighbour-sector Hamiltonians
    (small sectors only).  The paper has no gradients; this is the plain
    first-order perturbation theory of the Lehmann form:

      G^>_{aa'}(t) = -i <0| c_a e^{-i(H_+ - E0) t} c^dag_a' |0>,
      G^<_{aa'}(t) = +i <0| c^dag_a' e^{+i(H_- - E0) t} c_a |0>,

    differentiated through three routes --
      * the neighbour Hamiltonians H_+/-: d f(H) = Q (F o Q^dag dH Q) Q^dag
        with F the first divided differences of f on the eigenvalues
        (Daleckii-Krein), f(E) = e^{-/+ i (E - E0) t};
      * E0: dE0 = <0|dH|0> (Hellmann-Feynman), dG^>/dE0 = i t G^>,
        dG^</dE0 = -i t G^<;
      * |0>: d|0> = sum_{n != 0} |n><n|dH|0> / (E0 - E_n).
    The cotangents are dG = dL/dRe G + i dL/dIm G (either may be None = 0),
    so dL = Re sum conj(dG) dG_theta.  Returns (g_eps [2, L], g_hre [L, L],
    g_him [L, L], g_U [L]) in the convention of the library's VJP: g_hre is
    symmetric with the diagonal dL/dh_ii, g_him antisymmetric."""
    L = model["L"]
    n = len(orbitals)
    shape = (n_steps + 1, n, n)
    A = np.zeros(shape, np.complex128) if dG_gtr is None else np.asarray(dG_gtr, np.complex128)
    B = np.zeros(shape, np.complex128) if dG_les is None else np.asarray(dG_les, np.complex128)
    t = dt * np.arange(n_steps + 1)
    sec = Sector(model)
    w0, Q0 = _eigh(dense_hamiltonian(sec))
    if w0.size > 1 and w0[1] - w0[0] < 1e-8 * max(1.0, abs(w0[0])):
        raise ValueError("degenerate ground state: no gradient")
    E0, psi = w0[0], Q0[:, 0]
    dL_dE0 = 0.0
    w_vec = np.zeros(sec.dim, dtype=np.complex128)   # (Omega + Omega^dag)|0>
    Y = []                                            # (sector, Y): dL = Re sum(Y * dH)
    for spin, idx in _groups(orbitals).items():
        if not idx:
            continue
        for dagger in (True, False):
            nb = sec.neighbour(spin, dagger)
            if nb is None:
                continue
            E, Q = _eigh(dense_hamiltonian(nb))
            u = np.stack([sec.apply_cop(nb, orbitals[a][0], spin, dagger, psi) for a in idx])  # [na, dn]
            p = u @ Q.conj()                                                                    # p[a] = Q^dag u_a
            C = np.conj(A if dagger else B)[:, idx][:, :, idx]                                 # [t, a, a']
            sgn = -1.0 if dagger else 1.0                    # e^{sgn i (E - E0) t}
            ph = np.exp(sgn * 1j * np.outer(t, E - E0))      # [t, m]
            pref = -1j if dagger else 1j
            # the Green's function block itself (for the E0 route)
            if dagger:   # G^>_{aa'}(t) = -i sum_m conj(p_am) p_a'm ph_tm
                G = pref * np.einsum("am,bm,tm->tab", p.conj(), p, ph)
            else:        # G^<_{aa'}(t) = +i sum_m conj(p_a'm) p_am ph_tm
                G = pref * np.einsum("bm,am,tm->tab", p.conj(), p, ph)
            dL_dE0 += float(np.sum(C * (-sgn) * 1j * t[:, None, None] * G).real)
            # g_{aa'}(E) = pref sum_t C_t,aa' e^{sgn i (E - E0) t} and its E-derivative
            g = pref * np.einsum("tab,tm->abm", C, ph)
            dg = pref * np.einsum("tab,tm->abm", C * (sgn * 1j * t)[:, None, None], ph)
            Z = np.zeros((nb.dim, nb.dim), dtype=np.complex128)
            na = len(idx)
            for ia in range(na):
                for ib in range(na):
                    D = _divided_differences(g[ia, ib], dg[ia, ib], E)
                    if dagger:   # Z_mn += conj(p_am) p_a'n D
                        Z += np.outer(p[ia].conj(), p[ib]) * D
                    else:        # Z_mn += conj(q_a'm) q_an D
                        Z += np.outer(p[ib].conj(), p[ia]) * D
            Y.append((nb, _sandwich(Q, Z)))
            # (Omega + Omega^dag)|0>, Omega = sum C O with G = <0|O|0>
            for ia, a in enumerate(idx):
                for ib, b in enumerate(idx):
                    if dagger:   # O = -i c_a e^{-i(H+ - E0)t} c^dag_b
                        fwd = Q @ (g[ia, ib] * p[ib])                 # into c_a
                        bwd = Q @ (np.conj(g[ia, ib]) * p[ia])        # into c_b
                        w_vec += nb.apply_cop(sec, orbitals[a][0], spin, False, fwd)
                        w_vec += nb.apply_cop(sec, orbitals[b][0], spin, False, bwd)
                    else:        # O = +i c^dag_b e^{+i(H- - E0)t} c_a
                        fwd = Q @ (g[ia, ib] * p[ia])                 # into c^dag_b
                        bwd = Q @ (np.conj(g[ia, ib]) * p[ib])        # into c^dag_a
                        w_vec += nb.apply_cop(sec, orbitals[b][0], spin, True, fwd)
                        w_vec += nb.apply_cop(sec, orbitals[a][0], spin, True, bwd)
    # the ground-state routes: R = sum_{n != 0} |n><n| / (E0 - E_n)
    inv = np.zeros_like(w0)
    inv[1:] = 1.0 / (E0 - w0[1:])
    Rw = Q0 @ (inv * (Q0.conj().T @ w_vec))
    Y.append((sec, np.outer(psi.conj(), Rw) + dL_dE0 * np.outer(psi.conj(), psi)))

    diags = [(s, np.ascontiguousarray(np.diagonal(Ys).real), s.basis()) for s, Ys in Y]

    def grad(kind, i, j=None):
        tot = 0.0
        if kind in ("eps", "U"):  # diagonal dH: the occupation n_{i sigma} or n_{i up} n_{i dn}
            for s, yd, basis in diags:
                if kind == "eps":
                    occ = (basis >> np.uint64(i * L + j)) & np.uint64(1)
                else:
                    occ = ((basis >> np.uint64(i)) & (basis >> np.uint64(L + i))) & np.uint64(1)
                tot += float(np.dot(yd, occ.astype(np.float64)))
            return tot
        for s, Ys in Y:
            dH = dense_hamiltonian(Sector(_unit_model(model, kind, i, j), s.n_up, s.n_dn))
            tot += float(np.sum(Ys * dH).real)
        return tot

    g_eps = np.array([[grad("eps", sg, i) for i in range(L)] for sg in range(2)])
    g_U = np.array([grad("U", i) for i in range(L)])
    g_hre = np.zeros((L, L))
    g_him = np.zeros((L, L))
    for i in range(L):
        g_hre[i, i] = grad("re", i, i)
        for j in range(i + 1, L):
            g_hre[i, j] = g_hre[j, i] = grad("re", i, j)
            g_him[i, j] = grad("im", i, j)
            g_him[j, i] = -g_him[i, j]
    return g_eps, g_hre, g_him, g_U


def keldysh_entries(ini, fin, samples, dt, gs=None, K=80, tol=1e-12):
    """Several sampled entries of the Keldysh grid at any size: for each
    (k, l, orbital_a, orbital_b) of `samples`, the pair (G^<_{ab}(t_k,t_l),
    G^>_{ab}(t_k,t_l)) of Section 4, steps (i)-(iv), computed exactly as
    keldysh_entry does, with every Phi(t_k) and every back-propagated vector
    formed once and shared between the entries that use it."""
    sec_i = Sector(ini)
    E0, psi0, _ = sec_i.ground_state(K=K, tol=tol) if gs is None else gs
    sec_f = Sector(fin)
    phi, vec, nbs = {}, {}, {}

    def phi_at(k):
        if k not in phi:
            phi[k] = sec_f.propagate(psi0, dt * k) if k else psi0
        return phi[k]

    def back(k, orb, dagger):
        key = (k, orb, dagger)
        if key not in vec:
            site, spin = orb
            if (spin, dagger) not in nbs:
                nbs[(spin, dagger)] = sec_f.neighbour(spin, dagger)
            nb = nbs[(spin, dagger)]
            vec[key] = None if nb is None else nb.propagate(sec_f.apply_cop(nb, site, spin, dagger, phi_at(k)),
                                                            -dt * k)
        return vec[key]

    out = []
    for (k, l, oa, ob) in samples:
        if oa[1] != ob[1]:
            out.append((0j, 0j))
            continue
        pair = []
        for dagger in (False, True):
            va, vb = back(k, tuple(oa), dagger), back(l, tuple(ob), dagger)
            if va is None:
                pair.append(0j)
            else:
                pair.append(1j * np.vdot(vb, va) if not dagger else -1j * np.vdot(va, vb))
        out.append(tuple(pair))
    return out


def green_equilibrium_dense(model, orbitals, dt, n_steps):
    """The equilibrium G^>(t_k), G^<(t_k) of green_equilibrium by the Lehmann
    sum (Section 3, Eq. (psigreen) with eta = 0 and the hole part after Eq.
    (gomega)) from the dense eigen-decompositions of the sector and its
    neighbours (small sectors only):

      G^>_{aa'}(t) = -i sum_m <0|c_a|m><m|c^dag_a'|0> e^{-i(E_m - E0) t},
      G^<_{aa'}(t) = +i sum_m <0|c^dag_a'|m><m|c_a|0> e^{+i(E_m - E0) t},

    |m>, E_m the eigenpairs of the N+1 (N-1) sector.  Returns (G_gtr, G_les,
    E0, gap) with gap = E_1 - E0 of the sector (the degeneracy test)."""
    sec = Sector(model)
    w0, Q0 = _eigh(dense_hamiltonian(sec))
    E0, psi = w0[0], Q0[:, 0]
    gap = w0[1] - w0[0] if w0.size > 1 else np.inf
    n = len(orbitals)
    t = dt * np.arange(n_steps + 1)
    G_gtr = np.zeros((n_steps + 1, n, n), dtype=np.complex128)
    G_les = np.zeros_like(G_gtr)
    for spin, idx in _groups(orbitals).items():
        if not idx:
            continue
        for dagger, G in ((True, G_gtr), (False, G_les)):
            nb = sec.neighbour(spin, dagger)
            if nb is None:
                continue
            E, Q = _eigh(dense_hamiltonian(nb))
            u = np.stack([sec.apply_cop(nb, orbitals[a][0], spin, dagger, psi) for a in idx])
            p = u @ Q.conj()                                   # p[a, m] = <m|u_a>
            if dagger:
                ph = np.exp(-1j * np.outer(t, E - E0))         # [t, m]
                blk = -1j * np.einsum("am,bm,tm->tab", p.conj(), p, ph)
            else:
                ph = np.exp(1j * np.outer(t, E - E0))
                blk = 1j * np.einsum("bm,am,tm->tab", p.conj(), p, ph)
            G[np.ix_(range(n_steps + 1), idx, idx)] = blk
    return G_gtr, G_les, E0, gap


# Fourth-order commutator-free exponential step with two exponentials (the
# "higher-order commutator-free" propagators the outlook of the paper points
# to): with A_1, A_2 the Hamiltonian at the Gauss nodes t + c_{1,2} h,
# c_{1,2} = 1/2 -/+ sqrt(3)/6,
#   U(t + h, t) = exp(-i h (a1 A_1 + a2 A_2)) exp(-i h (a2 A_1 + a1 A_2)),
# a1 = (3 - 2 sqrt(3))/12, a2 = (3 + 2 sqrt(3))/12, the right factor first.
CF4_A1 = (3.0 - 2.0 * np.sqrt(3.0)) / 12.0
CF4_A2 = (3.0 + 2.0 * np.sqrt(3.0)) / 12.0
CF4_C = (0.5 - np.sqrt(3.0) / 6.0, 0.5 + np.sqrt(3.0) / 6.0)


def cf4_exponents(dparams):
    """For each step the parameter offsets of the two exponentials' (halved)
    Hamiltonians: a2 A_1 + a1 A_2 = H(fin + 2(a2 d_1 + a1 d_2)) / 2 (applied
    first) and a1 A_1 + a2 A_2 = H(fin + 2(a1 d_1 + a2 d_2)) / 2, H being
    linear in its parameters and a1 + a2 = 1/2.  dparams: [n_steps, 2, 3L]
    (offsets of eps (spin-major, 2L) then U (L) at the two Gauss nodes)."""
    d = np.asarray(dparams, dtype=np.float64)
    first = 2.0 * (CF4_A2 * d[:, 0] + CF4_A1 * d[:, 1])
    second = 2.0 * (CF4_A1 * d[:, 0] + CF4_A2 * d[:, 1])
    return first, second


def _shifted(model, dp):
    L = model["L"]
    m = dict(model)
    m["eps"] = np.asarray(model["eps"], dtype=np.float64) + np.asarray(dp[:2 * L]).reshape(2, L)
    m["U"] = np.asarray(model["U"], dtype=np.float64) + np.asarray(dp[2 * L:3 * L])
    return m


def green_keldysh_td(ini, fin, orbitals, dt, n_t, dparams, n_sub=1, gs=None, K=80, tol=1e-12):
    """The Keldysh G^<, G^> of Section 4 (steps (i)-(iv), shaped like
    green_keldysh) for a time-dependent Hamiltonian after the quench,
    H(t) = H_fin + sum_{i sigma} de_{i sigma}(t) n_{i sigma} + sum_i dU_i(t)
    n_{i up} n_{i dn}, each of the (n_t - 1) n_sub steps of h = dt / n_sub
    propagated by the fourth-order commutator-free step above with every
    exponential a Chebyshev expansion; dparams [(n_t-1) n_sub, 2, 3L] holds
    the offsets at the two Gauss nodes of each step.  Phi(t_k) = U(t_k, 0)|0>,
    Psi_a(t_k) = U(t_k, 0)^dag c_a Phi(t_k), chi_a likewise with c^dag."""
    sec_i = Sector(ini)
    E0, psi0, _ = sec_i.ground_state(K=K, tol=tol) if gs is None else gs
    n_steps = (n_t - 1) * n_sub
    h = dt / n_sub
    first, second = cf4_exponents(np.asarray(dparams).reshape(n_steps, 2, -1)) if n_steps else ([], [])
    cache = {}

    def sector(dp, nu, nd):
        key = (tuple(np.round(dp, 17)), nu, nd)
        if key not in cache:
            cache[key] = Sector(_shifted(fin, dp), nu, nd)
        return cache[key]

    def step(x, s, nu, nd, backward):
        if not backward:  # U_s = e^{-i h/2 H2} e^{-i h/2 H1}
            x = sector(first[s], nu, nd).propagate(x, 0.5 * h)
            return sector(second[s], nu, nd).propagate(x, 0.5 * h)
        # U_s^dag = e^{+i h/2 H1} e^{+i h/2 H2}
        x = sector(second[s], nu, nd).propagate(x, -0.5 * h)
        return sector(first[s], nu, nd).propagate(x, -0.5 * h)

    nu0, nd0 = fin["n_up"], fin["n_dn"]
    Phi = [psi0.copy()]
    x = psi0.copy()
    for s in range(n_steps):
        x = step(x, s, nu0, nd0, False)
        if (s + 1) % n_sub == 0:
            Phi.append(x.copy())
    sec_f = Sector(fin)
    n = len(orbitals)
    G_les = np.zeros((n_t, n_t, n, n), dtype=np.complex128)
    G_gtr = np.zeros_like(G_les)
    for spin, idx in _groups(orbitals).items():
        if not idx:
            continue
        for dagger, G in ((False, G_les), (True, G_gtr)):
            nb = sec_f.neighbour(spin, dagger)
            if nb is None:
                continue
            vecs = []
            for k in range(n_t):
                row = []
                for a in idx:
                    v = sec_f.apply_cop(nb, orbitals[a][0], spin, dagger, Phi[k])
                    for s in range(k * n_sub - 1, -1, -1):
                        v = step(v, s, nb.n_up, nb.n_dn, True)
                    row.append(v)
                vecs.append(row)
            for k in range(n_t):
                for l in range(n_t):
                    for ia, a in enumerate(idx):
                        for ib, b in enumerate(idx):
                            if not dagger:  # G^<_{ab}(t_k,t_l) = i <Psi_b(t_l)|Psi_a(t_k)>
                                G[k, l, a, b] = 1j * np.vdot(vecs[l][ib], vecs[k][ia])
                            else:  # G^>_{ab}(t_k,t_l) = -i <chi_a(t_k)|chi_b(t_l)>
                                G[k, l, a, b] = -1j * np.vdot(vecs[k][ia], vecs[l][ib])
    return G_les, G_gtr, E0


def green_four_time(ini, fin, ops, dt, n_t, gs=None, K=80, tol=1e-12):
    """Four-time correlation function of Section 6 (the outlook's higher-order
    Green's functions) after the quench of Section 4:
        G[k1, k2, k3, k4] = <0| A1(t1) A2(t2) A3(t3) A4(t4) |0>,  t_k = k dt,
    A(t) = e^{iHt} A e^{-iHt} with H = H_fin, |0> the ground state of H_ini,
    ops = four (site, spin, dagger) triples (dagger 1: c^dag, 0: c).  With
    Phi(t) = e^{-iHt}|0>, the right vectors R(t3, t4) = e^{iH t3} A3
    e^{-iH(t3 - t4)} A4 Phi(t4) and the left vectors L(t1, t2) = e^{iH t2}
    A2^dag e^{-iH(t2 - t1)} A1^dag Phi(t1) live in one sector and
    G = <L(t1, t2) | R(t3, t4)>; every exponential is one Chebyshev expansion.
    Returns complex [n_t, n_t, n_t, n_t] (zero when the operators do not
    conserve the particle numbers)."""
    sec_i = Sector(ini)
    E0, psi0, _ = sec_i.ground_state(K=K, tol=tol) if gs is None else gs
    sec_f = Sector(fin)
    Phi = [psi0.copy()]
    for k in range(1, n_t):
        Phi.append(sec_f.propagate(Phi[-1], dt))
    G = np.zeros((n_t,) * 4, dtype=np.complex128)

    def chain(first, second):
        # sectors after `first` then `second` are applied to Phi's sector
        s1 = sec_f.neighbour(first[1], bool(first[2]))
        s2 = None if s1 is None else s1.neighbour(second[1], bool(second[2]))
        return s1, s2

    def pair_vectors(first, second):
        # V[ta][tb] = e^{iH ta} B e^{-iH(ta - tb)} A Phi(tb), A = first, B = second
        s1, s2 = chain(first, second)
        if s2 is None:
            return None, None
        V = [[None] * n_t for _ in range(n_t)]
        for tb in range(n_t):
            v = sec_f.apply_cop(s1, first[0], first[1], bool(first[2]), Phi[tb])
            for ta in range(n_t):
                u = s1.propagate(v, (ta - tb) * dt)
                w = s1.apply_cop(s2, second[0], second[1], bool(second[2]), u)
                V[ta][tb] = s2.propagate(w, -ta * dt)
        return (s2.n_up, s2.n_dn), V

    a1, a2, a3, a4 = [tuple(int(v) for v in o) for o in ops]
    key_r, R = pair_vectors(a4, a3)
    key_l, Lv = pair_vectors((a1[0], a1[1], 1 - a1[2]), (a2[0], a2[1], 1 - a2[2]))
    if R is None or Lv is None or key_r != key_l:
        return G
    for k1 in range(n_t):
        for k2 in range(n_t):
            for k3 in range(n_t):
                for k4 in range(n_t):
                    G[k1, k2, k3, k4] = np.vdot(Lv[k2][k1], R[k3][k4])
    return G


# ------------------------------------------------------------------ NE-CPT
# Section 5: the nonequilibrium cluster-perturbation theory of the paper's
# application, a cluster of L_c sites (impurity at site 0) coupled by the
# hopping V between its last site and the first site of a non-interacting
# bath chain.  Every function lives on the L-shaped contour 0 -> t_max -> 0 ->
# -i beta, discretised by the trapezoidal rule: forward points t_j = j dt
# (weight dt), backward points (weight -dt), imaginary points -i tau_k,
# tau_k = k dtau (weight -i dtau), half weights at the ends of each branch.

def contour(dt, n_t, beta, n_tau):
    """Contour points as (kind, index, s, z, w): kind 0 forward, 1 backward,
    2 imaginary; s the position along the contour (a later point has a
    larger s; the branch ends t_max and 0 appear twice, the later copy on the
    later branch); z the complex time; w the quadrature weight."""
    dtau = beta / n_tau
    pts = []
    for j in range(n_t):
        w = dt * (0.5 if j in (0, n_t - 1) else 1.0) if n_t > 1 else 0.0
        pts.append((0, j, len(pts), complex(j * dt), w))
    for j in range(n_t - 1, -1, -1):
        w = -dt * (0.5 if j in (0, n_t - 1) else 1.0) if n_t > 1 else 0.0
        pts.append((1, j, len(pts), complex(j * dt), w))
    for k in range(n_tau + 1):
        w = -1j * dtau * (0.5 if k in (0, n_tau) else 1.0)
        pts.append((2, k, len(pts), complex(0.0, -k * dtau), w))
    return pts


def _ordered(s1, s2, later, earlier):
    """The contour-ordered value from its two orderings (the mean on the
    diagonal, where the two one-sided limits differ by the jump)."""
    if s1 > s2:
        return later
    if s1 < s2:
        return earlier
    return 0.5 * (later + earlier)


def cluster_contour_gf(ini, fin, spin, dt, n_t, beta, n_tau, mu=0.0):
    """The cluster Green's function G'_{ij}(z, z') = -i <T_C c_i(z) c^dag_j(z')>
    of one spin on the contour of length beta, at a temperature 1/beta low
    enough that only the ground state |0> of H_ini (and, through the trace,
    the lowest states of its neighbour sectors) contributes.  From the
    zero-temperature components of Section 4:
      real-real:  G^> (z later), G^< (z' later);
      G(t, -i tau)  = G^right(t, tau) + conj(G^left_{ji}(beta - tau, t)),
      G(-i tau, t)  = G^left(tau, t) + conj(G^right_{ji}(t, beta - tau)),
      G(-i tau, -i tau') = i G^M_beta(tau - tau'), with
      G^M_beta(tau) = G^M(tau) - G^M(tau - beta) for tau > 0 and
      G^M_beta(-tau) = G^M(-tau) - G^M(beta - tau),
    the second terms being the antiperiodic tails that the trace at inverse
    temperature beta adds near the end of the imaginary branch (terms of
    relative size e^{-beta gap} are dropped).  The mean of the two orderings
    on the diagonal z = z'.  Returns [L_c, L_c, n_pts, n_pts]."""
    L = fin["L"]
    orbs = [(i, spin) for i in range(L)]
    pts = contour(dt, n_t, beta, n_tau)
    dtau = beta / n_tau
    taus = dtau * np.arange(n_tau + 1)
    sec = Sector(ini)
    gs = sec.ground_state()
    Gl, Gg, _ = green_keldysh(ini, fin, orbs, dt, n_t, gs=gs)
    Gr, Glf, _ = green_mixed(ini, fin, orbs, dt, n_t, taus, mu, gs=gs)
    Gp, Gm, _ = green_matsubara(ini, orbs, taus, mu, gs=gs)
    n = len(pts)
    G = np.zeros((L, L, n, n), dtype=np.complex128)
    NT = n_tau

    def GMb_pos(k):  # G^M_beta(tau_k)
        return Gp[k] - Gm[NT - k]

    def GMb_neg(k):  # G^M_beta(-tau_k)
        return Gm[k] - Gp[NT - k]

    for p, (k1, i1, s1, _, _) in enumerate(pts):
        for q, (k2, i2, s2, _, _) in enumerate(pts):
            if k1 < 2 and k2 < 2:
                val = _ordered(s1, s2, Gg[i1, i2], Gl[i1, i2])
            elif k1 < 2:  # real earlier than imaginary
                val = Gr[i1, i2] + np.conj(Glf[NT - i2, i1]).T
            elif k2 < 2:  # imaginary later than real
                val = Glf[i1, i2] + np.conj(Gr[i2, NT - i1]).T
            else:
                if i1 > i2:
                    val = 1j * GMb_pos(i1 - i2)
                elif i1 < i2:
                    val = 1j * GMb_neg(i2 - i1)
                else:
                    val = 1j * 0.5 * (GMb_pos(0) + GMb_neg(0))
            G[:, :, p, q] = val
    return G


def bath_surface_gf(L_b, T_b, dt, n_t, beta, n_tau):
    """g_00(z, z') of the first site of a chain of L_b sites with hopping -T_b
    (on-site energy and chemical potential 0), Section 5 Eqs. (gb1), (gb2):
    -i [e^{-i T (z - z')} (1 + e^{-beta T})^{-1}]_00 for z later and
    +i [e^{-i T (z - z')} (e^{beta T} + 1)^{-1}]_00 for z' later, from the
    eigen-decomposition of the hopping matrix T."""
    h = -T_b * (np.eye(L_b, k=1) + np.eye(L_b, k=-1))
    eps, phi = np.linalg.eigh(h)
    w0 = phi[0] ** 2
    pts = contour(dt, n_t, beta, n_tau)
    z = np.array([p[3] for p in pts])
    s = np.array([p[2] for p in pts])
    a = np.exp(-1j * np.outer(z, eps))   # e^{-i eps z}
    b = np.exp(1j * np.outer(z, eps))    # e^{+i eps z'}
    f = 1.0 / (np.exp(beta * eps) + 1.0)
    later = -1j * (a * (w0 * (1.0 - f))) @ b.T
    earlier = 1j * (a * (w0 * f)) @ b.T
    S1, S2 = np.meshgrid(s, s, indexing="ij")
    return np.where(S1 > S2, later, np.where(S1 < S2, earlier, 0.5 * (later + earlier)))


def necpt_occupations(ini, fin, L_b, T_b, V, dt, n_t, beta, n_tau, mu=0.0):
    """Section 5, Eq. (cpteq): G = (G'^{-1} - V)^{-1} on the contour for the
    cluster coupled at its last site to the bath by V.  The bath integrated
    out, the cluster block obeys G = G' + G' * Delta * G, Delta = V^2 g_00 on
    the last site, * the contour integral (trapezoidal weights W):
        G_{Lj} = (1 - G'_{LL} W Delta W)^{-1} G'_{Lj},
        G_{ij} = G'_{ij} + G'_{iL} W Delta W G_{Lj}.
    Returns n[spin, k, i] = n_{i spin}(t_k) = -i G^<_{ii}(t_k, t_k) (the forward
    point t_k against the backward point t_k) for the cluster sites."""
    L = fin["L"]
    pts = contour(dt, n_t, beta, n_tau)
    W = np.diag([p[4] for p in pts])
    Delta = V * V * bath_surface_gf(L_b, T_b, dt, n_t, beta, n_tau)
    M = W @ Delta @ W
    npt = len(pts)
    fwd = [p for p, q in enumerate(pts) if q[0] == 0]            # t_0 .. t_max
    bwd = [p for p, q in enumerate(pts) if q[0] == 1][::-1]      # t_0 .. t_max
    out = np.zeros((2, n_t, L))
    for spin in (0, 1):
        Gc = cluster_contour_gf(ini, fin, spin, dt, n_t, beta, n_tau, mu)
        Lst = L - 1
        X = np.linalg.solve(np.eye(npt) - Gc[Lst, Lst] @ M, np.eye(npt))
        for i in range(L):
            GLi = X @ Gc[Lst, i]
            Gii = Gc[i, i] + Gc[i, Lst] @ M @ GLi
            for k in range(n_t):
                out[spin, k, i] = (-1j * Gii[fwd[k], bwd[k]]).real
    return out
