"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module only *defines model Hamiltonians and random inputs*; it holds none
of the method's arithmetic (no H*psi, no Lanczos, no propagation, no Green's
function).  Both the CPU oracle and the CUDA path receive what is built here.

Model convention (Section 2 and Section 4 of the paper):

    H = sum_{sigma} sum_{i != j} h_ij c^dag_{i sigma} c_{j sigma}
        + sum_{i sigma} eps_{i sigma} n_{i sigma}
        + sum_i U_i n_{i up} n_{i dn}

The paper writes the hopping as -T sum c^dag c (Hubbard ring, Section 3;
SIAM chain, Section 4), so a hopping amplitude T enters as h_ij = -T.  The
local field of Eq. (hfi), H_field = -h (n_1up - n_1dn), enters as
eps_{1 up} -= h, eps_{1 dn} += h.

Site index i = 0..L-1, spin sigma = 0 (up) / 1 (down).  A model is a plain
dict with numpy arrays:  L, n_up, n_dn, h (L x L complex Hermitian),
eps (2 x L real: eps[sigma, i]), U (L real).
"""
from __future__ import annotations

import math

import numpy as np


def make_model(L, n_up, n_dn, h, eps=None, U=None):
    h = np.asarray(h, dtype=np.complex128).reshape(L, L)
    eps = np.zeros((2, L)) if eps is None else np.asarray(eps, dtype=np.float64).reshape(2, L)
    U = np.zeros(L) if U is None else np.broadcast_to(np.asarray(U, dtype=np.float64), (L,)).copy()
    return {"L": int(L), "n_up": int(n_up), "n_dn": int(n_dn), "h": h, "eps": eps, "U": U}


def with_sector(model, n_up, n_dn):
    m = dict(model)
    m["n_up"], m["n_dn"] = int(n_up), int(n_dn)
    return m


def sector_dim(L, n_up, n_dn):
    if n_up < 0 or n_dn < 0 or n_up > L or n_dn > L:
        return 0
    return math.comb(L, n_up) * math.comb(L, n_dn)


# ---------------------------------------------------------------- geometries
def ring_hopping(L, T=1.0, pbc=True):
    """Nearest-neighbour ring (Section 3, Fig. 1 model): h_{i,i+1} = -T."""
    h = np.zeros((L, L))
    for i in range(L - 1 if not pbc else L):
        j = (i + 1) % L
        if i == j:
            continue
        h[i, j] += -T
        h[j, i] += -T
    return h


def chain_hopping(L, T=1.0):
    """Open chain, sites 0..L-1, impurity at site 0 (Section 4, SIAM chain)."""
    return ring_hopping(L, T, pbc=False)


def star_hopping(V):
    """Impurity 0 coupled to bath sites 1..nb with amplitude V_k (star SIAM)."""
    V = np.asarray(V, dtype=np.float64)
    L = len(V) + 1
    h = np.zeros((L, L))
    h[0, 1:] = V
    h[1:, 0] = V
    return h


# -------------------------------------------------------------------- models
def hubbard_ring(L, U, n_up, n_dn, T=1.0, pbc=True):
    return make_model(L, n_up, n_dn, ring_hopping(L, T, pbc), None, np.full(L, float(U)))


def siam_chain(L, U, n_up, n_dn, T=1.0, field=0.0, eps_imp=None):
    """SIAM on a chain with the impurity at site 0 and optional field (Eq. hfi)."""
    eps_imp = -U / 2.0 if eps_imp is None else eps_imp
    eps = np.zeros((2, L))
    eps[0, 0] = eps_imp - field
    eps[1, 0] = eps_imp + field
    Uv = np.zeros(L)
    Uv[0] = U
    return make_model(L, n_up, n_dn, chain_hopping(L, T), eps, Uv)


def siam_star(eps_d, U, eps_k, V_k, n_up, n_dn, field=0.0):
    eps_k = np.asarray(eps_k, dtype=np.float64)
    L = len(eps_k) + 1
    eps = np.zeros((2, L))
    eps[:, 1:] = eps_k
    eps[0, 0] = eps_d - field
    eps[1, 0] = eps_d + field
    Uv = np.zeros(L)
    Uv[0] = U
    return make_model(L, n_up, n_dn, star_hopping(V_k), eps, Uv)


def random_model(L, n_up, n_dn, seed, complex_hopping=True, density=1.0):
    """Random Hermitian hopping, random eps and U (test inputs only)."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(-1, 1, (L, L))
    if complex_hopping:
        h = h + 1j * rng.uniform(-1, 1, (L, L))
    if density < 1.0:
        mask = rng.uniform(0, 1, (L, L)) < density
        h = h * mask
    h = 0.5 * (h + h.conj().T)
    np.fill_diagonal(h, 0.0)
    eps = rng.uniform(-1, 1, (2, L))
    U = rng.uniform(0, 4, L)
    return make_model(L, n_up, n_dn, h, eps, U)


# ------------------------------------------------------- benchmark workloads
def config_c1():
    """Equilibrium star SIAM: 1 impurity + 5 bath sites, (3,3), d = 400.

    U = 4, eps_d = -U/2, bath energies {-2,-1,0,1,2}, V_k = 0.5; Krylov M = 40;
    G_imp(t) on t in [0, 20] at dt = 0.05 (401 points).
    """
    U = 4.0
    m = siam_star(-U / 2, U, [-2.0, -1.0, 0.0, 1.0, 2.0], [0.5] * 5, 3, 3)
    return {"model": m, "M": 40, "dt": 0.05, "n_steps": 400, "orbitals": [(0, 0)]}


def config_c2():
    """Hubbard ring L = 12, T = 1, PBC, half filling (6,6), d = 853,776.

    Ground state at U = 8, sudden quench to U = 4; Keldysh G_ij(t,t') for all
    i, j (spin up) on a 100 x 100 grid with dt = 0.05 and Krylov M = 20.
    """
    L = 12
    return {
        "ini": hubbard_ring(L, 8.0, 6, 6),
        "fin": hubbard_ring(L, 4.0, 6, 6),
        "M": 20, "dt": 0.05, "n_t": 100,
        "orbitals": [(i, 0) for i in range(L)],
    }


def config_c3():
    """Local magnetic excitation on a 16-site chain (1 correlated + 15 bath).

    U = 8 at site 0, eps_imp = -U/2, T = 1, field h = 2 in H_ini switched off
    for t > 0; sector (7,7), d = 130,873,600; impurity G(t,t') on a 50 x 50
    grid, t_k = 0.2 k, internal Krylov step 0.05 with M = 20.
    """
    L = 16
    return {
        "ini": siam_chain(L, 8.0, 7, 7, field=2.0),
        "fin": siam_chain(L, 8.0, 7, 7, field=0.0),
        "M": 20, "dt": 0.2, "dt_internal": 0.05, "n_t": 50,
        "orbitals": [(0, 0), (0, 1)],
    }


def config_c4(n_inst=256, seed=20240501):
    """256 star-SIAM instances of random size and filling (batched solves)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        L = int(rng.integers(6, 13))
        nu = int(rng.integers(1, L))
        nd = int(rng.integers(1, L))
        U = float(rng.uniform(1, 8))
        ek = rng.uniform(-3, 3, L - 1)
        vk = rng.uniform(0.2, 1.0, L - 1)
        out.append(siam_star(-U / 2, U, ek, vk, nu, nd))
    return {"models": out, "M": 20, "dt": 0.05, "n_steps": 400, "orbitals": [(0, 0)]}


def c5_parameters(seed):
    """Star SIAM L = 10 parameter draw: 9 eps_k, 9 V_k and U (adjoint config)."""
    rng = np.random.default_rng(seed)
    U = float(rng.uniform(1, 8))
    ek = rng.uniform(-3, 3, 9)
    vk = rng.uniform(0.2, 1.0, 9)
    return ek, vk, U


def config_c5(eps_d=-2.0):
    """Adjoint workload: star L = 10, (5,5), d = 63,504, 401 times, dt = 0.05.

    eps_d is a fixed constant (not differentiated); the target G is generated
    from the seed-7 parameters, the optimisation starts from seed 8.
    """
    tgt = c5_parameters(7)
    start = c5_parameters(8)
    return {
        "target": siam_star(eps_d, tgt[2], tgt[0], tgt[1], 5, 5),
        "start": siam_star(eps_d, start[2], start[0], start[1], 5, 5),
        "eps_d": eps_d, "M": 20, "dt": 0.05, "n_steps": 400,
        "checkpoint": 20, "orbitals": [(0, 0)],
    }


def random_state(d, seed):
    """Seeded normalised complex vector of length d (interleaved-ready)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    return v / np.linalg.norm(v)


def periodic_drive(L, amp_eps=0.7, omega=1.3, amp_U=0.8, omega_U=2.1, sites=None):
    """A smooth drive of the on-site terms after the quench: returns f(t), the
    offsets [eps_up (L), eps_dn (L), U (L)] at time t.  Every driven site's
    energy oscillates with a site- and spin-dependent phase; U of site 0
    oscillates too (a periodically modulated impurity).  sites: the driven
    sites (default all)."""
    sites = range(L) if sites is None else list(sites)

    def f(t):
        p = np.zeros(3 * L)
        for s in range(2):
            for i in sites:
                p[s * L + i] = amp_eps * math.sin(omega * t + 0.5 * i + 1.1 * s)
        p[2 * L] = amp_U * math.cos(omega_U * t)
        return p
    return f


def drive_samples(f, dt, n_t, n_sub, nodes):
    """The drive sampled where the driven Keldysh calls take it: for internal
    step s (h = dt / n_sub, t_s = s h) and node c of `nodes` (fractions of
    the step), f(t_s + c h); shape [(n_t - 1) n_sub, len(nodes), 3L]."""
    h = dt / n_sub
    return np.array([[f(s * h + c * h) for c in nodes] for s in range((n_t - 1) * n_sub)])
