"""Pins for the CPU oracle: checks against things other than the oracle itself.

* brute force: a dense Fock-space Hamiltonian built from Jordan-Wigner
  matrices with numpy Kronecker products (an independent construction of the
  second-quantised operators) on L <= 5;
* library routines: numpy eigh and scipy expm on those dense matrices;
* closed forms: U = 0 free fermions (single-particle h), the Hubbard atom;
* invariants: sum rule, hermiticity, particle-hole symmetry, particle number,
  the equal-time values the paper states for its Fig. 2 and Fig. 4 models.

Each plausible mistake (a dropped term, a wrong sign or index, a transposed
operand, a conjugate missing) fails at least one of these.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ dense JW tools
def jw_annihilators(n_modes):
    """Dense c_m on the 2^n Fock space, basis index = sum_m n_m 2^m."""
    dim = 1 << n_modes
    occ = ((np.arange(dim)[:, None] >> np.arange(n_modes)[None, :]) & 1)
    out = []
    for m in range(n_modes):
        c = np.zeros((dim, dim))
        for k in range(dim):
            if occ[k, m]:
                sgn = (-1) ** int(occ[k, :m].sum())
                c[k ^ (1 << m), k] = sgn
        out.append(c)
    return out


def jw_parts(L):
    c = jw_annihilators(2 * L)
    return c


def dense_fock_h(model, c):
    L = model["L"]
    dim = c[0].shape[0]
    H = np.zeros((dim, dim), dtype=np.complex128)
    h, eps, U = model["h"], model["eps"], model["U"]
    for s in range(2):
        for i in range(L):
            ci = c[s * L + i]
            H += (eps[s, i] + h[i, i].real) * (ci.T @ ci)
            for j in range(L):
                if i != j and h[i, j] != 0:
                    H += h[i, j] * (ci.T @ c[s * L + j])
    for i in range(L):
        H += U[i] * (c[i].T @ c[i]) @ (c[L + i].T @ c[L + i])
    return H


def sector_index(L, nu, nd):
    dim = 1 << (2 * L)
    k = np.arange(dim)
    up = np.array([bin(x & ((1 << L) - 1)).count("1") for x in k])
    dn = np.array([bin(x >> L).count("1") for x in k])
    return np.nonzero((up == nu) & (dn == nd))[0]  # ascending = sorted states


def rel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


# --------------------------------------------------------------- basis pins
@pytest.mark.parametrize("L,nu,nd", [(4, 2, 2), (5, 2, 3), (6, 1, 5), (7, 3, 3)])
def test_basis_order_and_size(L, nu, nd):
    s = oracle.Sector(W.hubbard_ring(L, 1.0, nu, nd))
    b = s.basis()
    assert s.dim == math.comb(L, nu) * math.comb(L, nd)
    assert np.all(np.diff(b.astype(np.float64)) > 0)
    ups = sorted(x for x in range(1 << L) if bin(x).count("1") == nu)
    dns = sorted(x for x in range(1 << L) if bin(x).count("1") == nd)
    Du = len(ups)
    for idx in range(0, s.dim, max(1, s.dim // 50)):
        assert int(b[idx]) == ups[idx % Du] | (dns[idx // Du] << L)


# ---------------------------------------------------------- H*psi and c/c^dag
@pytest.mark.parametrize("L", [2, 3, 4, 5])
def test_hpsi_vs_jordan_wigner(L):
    c = jw_parts(L)
    rng = np.random.default_rng(L)
    for seed in range(3):
        nu, nd = int(rng.integers(0, L + 1)), int(rng.integers(0, L + 1))
        m = W.random_model(L, nu, nd, seed=100 * L + seed, complex_hopping=True)
        H = dense_fock_h(m, c)
        idx = sector_index(L, nu, nd)
        Hs = H[np.ix_(idx, idx)]
        assert np.allclose(Hs, Hs.conj().T)
        s = oracle.Sector(m)
        x = W.random_state(s.dim, seed)
        assert rel(s.hpsi(x), Hs @ x) < 1e-13


@pytest.mark.parametrize("L", [3, 4])
def test_cop_vs_jordan_wigner(L):
    c = jw_parts(L)
    m = W.random_model(L, 1, 2, seed=7)
    for spin in (0, 1):
        for site in range(L):
            for dagger in (False, True):
                src = oracle.Sector(W.with_sector(m, 1, 2))
                dst = src.neighbour(spin, dagger)
                if dst is None:
                    continue
                op = c[spin * L + site]
                op = op.T if dagger else op
                i_src = sector_index(L, 1, 2)
                i_dst = sector_index(L, dst.n_up, dst.n_dn)
                x = W.random_state(src.dim, site + 10 * spin)
                ref = op[np.ix_(i_dst, i_src)] @ x
                assert np.max(np.abs(src.apply_cop(dst, site, spin, dagger, x) - ref)) < 1e-15


def test_hpsi_hermitian_larger():
    m = W.random_model(8, 3, 4, seed=3)
    s = oracle.Sector(m)
    x, y = W.random_state(s.dim, 1), W.random_state(s.dim, 2)
    assert abs(np.vdot(x, s.hpsi(y)) - np.vdot(s.hpsi(x), y)) < 1e-12


# ------------------------------------------------------------- ground state
@pytest.mark.parametrize("L,nu,nd,seed", [(4, 2, 2, 1), (5, 2, 3, 2), (5, 3, 3, 3)])
def test_ground_state_vs_eigh(L, nu, nd, seed):
    c = jw_parts(L)
    m = W.random_model(L, nu, nd, seed=seed, complex_hopping=True)
    idx = sector_index(L, nu, nd)
    Hs = dense_fock_h(m, c)[np.ix_(idx, idx)]
    w, v = np.linalg.eigh(Hs)
    E0, psi, res = oracle.Sector(m).ground_state()
    assert abs(E0 - w[0]) <= 1e-13 * max(1, abs(w[0]))
    assert abs(abs(np.vdot(v[:, 0], psi)) - 1) < 1e-12
    assert res < 1e-12 * max(1, abs(E0))


def free_fermion_e0(h, eps_s, n):
    w = np.linalg.eigvalsh(h + np.diag(eps_s))
    return w[:n].sum(), w


def test_ground_state_U0_closed_form():
    # open chain L = 10 at half filling: single-particle levels -2cos(k pi/11)
    # are nondegenerate, so the Slater determinant ground state is unique.
    L = 10
    m = W.make_model(L, 5, 5, W.chain_hopping(L), np.vstack([np.linspace(-0.3, 0.2, L)] * 2), np.zeros(L))
    E_up, _ = free_fermion_e0(m["h"], m["eps"][0], 5)
    E_dn, _ = free_fermion_e0(m["h"], m["eps"][1], 5)
    E0, _, _ = oracle.Sector(m).ground_state()
    assert abs(E0 - (E_up + E_dn)) < 1e-12 * abs(E_up + E_dn)


def test_hubbard_atom_energies():
    U, e = 3.0, -1.2
    for nu, nd, ref in [(0, 0, 0.0), (1, 0, e), (0, 1, e), (1, 1, 2 * e + U)]:
        m = W.make_model(1, nu, nd, np.zeros((1, 1)), np.array([[e], [e]]), np.array([U]))
        E0, _, _ = oracle.Sector(m).ground_state()
        assert abs(E0 - ref) < 1e-14


# --------------------------------------------------------------- propagation
@pytest.mark.parametrize("tau", [0.05, 0.7, -2.3])
def test_propagate_vs_expm(tau):
    L = 4
    c = jw_parts(L)
    m = W.random_model(L, 2, 1, seed=11, complex_hopping=True)
    idx = sector_index(L, 2, 1)
    Hs = dense_fock_h(m, c)[np.ix_(idx, idx)]
    s = oracle.Sector(m)
    x = W.random_state(s.dim, 5)
    ref = sla.expm(-1j * tau * Hs) @ x
    assert np.max(np.abs(s.propagate(x, tau) - ref)) < 1e-13


def test_propagate_norm_and_reversal():
    s = oracle.Sector(W.hubbard_ring(8, 4.0, 4, 3))
    x = W.random_state(s.dim, 9)
    y = s.propagate(x, 3.0)
    assert abs(np.linalg.norm(y) - 1) < 1e-13
    assert np.max(np.abs(s.propagate(y, -3.0) - x)) < 1e-13
    # stepping agrees with one long expansion (group property)
    z = x
    for _ in range(6):
        z = s.propagate(z, 0.5)
    assert np.max(np.abs(z - y)) < 1e-12


# ------------------------------------------------------ equilibrium G pins
def dense_sector(m, c, nu, nd):
    idx = sector_index(m["L"], nu, nd)
    return idx, dense_fock_h(W.with_sector(m, nu, nd), c)[np.ix_(idx, idx)]


def test_green_equilibrium_vs_dense_lehmann():
    L = 4
    c = jw_parts(L)
    m = W.random_model(L, 2, 2, seed=21, complex_hopping=True)
    orbs = [(0, 0), (2, 0), (1, 1), (3, 1)]
    dt, n = 0.1, 12
    Gg, Gl, E0 = oracle.green_equilibrium(m, orbs, dt, n)
    Hfull = dense_fock_h(m, c)
    i0 = sector_index(L, 2, 2)
    w, v = np.linalg.eigh(Hfull[np.ix_(i0, i0)])
    assert abs(E0 - w[0]) < 1e-12
    g = np.zeros(Hfull.shape[0], dtype=np.complex128)
    g[i0] = v[:, 0]
    t = dt * np.arange(n + 1)
    for k in range(n + 1):
        U_t = sla.expm(-1j * t[k] * Hfull)
        for a, (ia, sa) in enumerate(orbs):
            for b, (ib, sb) in enumerate(orbs):
                ca, cb = c[sa * L + ia], c[sb * L + ib]
                ref_g = -1j * np.exp(1j * w[0] * t[k]) * (g.conj() @ ca @ U_t @ cb.T @ g)
                ref_l = 1j * np.exp(-1j * w[0] * t[k]) * (g.conj() @ cb.T @ U_t.conj().T @ ca @ g)
                assert abs(Gg[k, a, b] - ref_g) < 1e-12
                assert abs(Gl[k, a, b] - ref_l) < 1e-12


def test_green_equilibrium_U0_closed_form():
    # complex Hermitian hopping, so a transposed or unconjugated density
    # matrix rho[k, l] = <c^dag_l c_k> = (V V^dag)[k, l] would fail here.
    L = 8
    m = W.random_model(L, 4, 3, seed=5, complex_hopping=True)
    m["U"][:] = 0.0
    eps = m["eps"]
    orbs = [(i, 0) for i in range(0, L, 2)] + [(1, 1), (4, 1)]
    dt, n = 0.2, 10
    Gg, Gl, _ = oracle.green_equilibrium(m, orbs, dt, n)
    for spin, N in ((0, 4), (1, 3)):
        hs = m["h"] + np.diag(eps[spin])
        w, v = np.linalg.eigh(hs)
        assert w[N] - w[N - 1] > 1e-3  # closed shell
        rho = v[:, :N] @ v[:, :N].conj().T
        idx = [k for k, o in enumerate(orbs) if o[1] == spin]
        for k in range(n + 1):
            U_t = sla.expm(-1j * hs * dt * k)
            ref_g = -1j * U_t @ (np.eye(L) - rho)
            ref_l = 1j * U_t @ rho
            for a in idx:
                for b in idx:
                    i, j = orbs[a][0], orbs[b][0]
                    assert abs(Gg[k, a, b] - ref_g[i, j]) < 1e-12
                    assert abs(Gl[k, a, b] - ref_l[i, j]) < 1e-12
    # opposite spins never mix
    assert np.all(Gg[:, :4, 4:] == 0) and np.all(Gl[:, 4:, :4] == 0)


def test_hubbard_atom_two_poles():
    # half-filled atom, eps = -U/2: spin-averaged G^R(t) = -i cos(U t / 2).
    U = 2.6
    dt, n = 0.25, 16
    t = dt * np.arange(n + 1)
    GR = 0
    for nu, nd in ((1, 0), (0, 1)):
        m = W.make_model(1, nu, nd, np.zeros((1, 1)), np.full((2, 1), -U / 2), np.array([U]))
        Gg, Gl, _ = oracle.green_equilibrium(m, [(0, 0), (0, 1)], dt, n)
        GR = GR + 0.5 * (Gg - Gl)
    avg = 0.5 * (GR[:, 0, 0] + GR[:, 1, 1])
    assert np.max(np.abs(avg - (-1j * np.cos(U * t / 2)))) < 1e-13


def test_equilibrium_sum_rule_and_ph_symmetry():
    cfg = W.config_c1()
    Gg, Gl, _ = oracle.green_equilibrium(cfg["model"], [(0, 0), (1, 0), (3, 0)], 0.1, 30)
    assert np.max(np.abs(1j * (Gg[0] - Gl[0]) - np.eye(3))) < 1e-12
    # particle-hole symmetric star SIAM: G^R_imp(t) is purely imaginary
    assert np.max(np.abs((Gg - Gl)[:, 0, 0].real)) < 1e-11
    # ring without the -U/2 shift: e^{iUt/2} G^R_ii(t) is purely imaginary
    U = 3.0
    m = W.hubbard_ring(6, U, 3, 3)
    Gg, Gl, _ = oracle.green_equilibrium(m, [(0, 0)], 0.1, 25)
    t = 0.1 * np.arange(26)
    assert np.max(np.abs((np.exp(1j * U * t / 2) * (Gg - Gl)[:, 0, 0]).real)) < 1e-11


# ------------------------------------------------------------ Keldysh pins
def test_keldysh_U0_quench_closed_form():
    L = 6
    ini = W.random_model(L, 3, 2, seed=8, complex_hopping=True)
    fin = W.random_model(L, 3, 2, seed=9, complex_hopping=True)
    ini["U"][:] = 0.0
    fin["U"][:] = 0.0
    eps_i, eps_f = ini["eps"], fin["eps"]
    orbs = [(0, 0), (2, 0), (5, 0), (1, 1), (3, 1)]
    dt, nt = 0.3, 7
    Gl, Gg, _ = oracle.green_keldysh(ini, fin, orbs, dt, nt)
    for spin, N in ((0, 3), (1, 2)):
        w, v = np.linalg.eigh(ini["h"] + np.diag(eps_i[spin]))
        assert w[N] - w[N - 1] > 1e-3
        rho = v[:, :N] @ v[:, :N].conj().T   # rho[k, l] = <c^dag_l c_k>
        hf = fin["h"] + np.diag(eps_f[spin])
        idx = [k for k, o in enumerate(orbs) if o[1] == spin]
        for k in range(nt):
            Uk = sla.expm(-1j * hf * dt * k)
            for l in range(nt):
                Ul = sla.expm(-1j * hf * dt * l)
                ref_l = 1j * Uk @ rho @ Ul.conj().T
                ref_g = -1j * Uk @ (np.eye(L) - rho) @ Ul.conj().T
                for a in idx:
                    for b in idx:
                        i, j = orbs[a][0], orbs[b][0]
                        assert abs(Gl[k, l, a, b] - ref_l[i, j]) < 1e-12
                        assert abs(Gg[k, l, a, b] - ref_g[i, j]) < 1e-12


def test_keldysh_vs_dense_interacting():
    L = 3
    c = jw_parts(L)
    ini = W.siam_chain(L, 2.0, 2, 1, field=0.4)
    fin = W.siam_chain(L, 2.0, 2, 1, field=0.0)
    orbs = [(0, 0), (1, 0), (2, 1)]
    dt, nt = 0.4, 5
    Gl, Gg, E0 = oracle.green_keldysh(ini, fin, orbs, dt, nt)
    Hi, Hf = dense_fock_h(ini, c), dense_fock_h(fin, c)
    i0 = sector_index(L, 2, 1)
    w, v = np.linalg.eigh(Hi[np.ix_(i0, i0)])
    g = np.zeros(Hi.shape[0], dtype=np.complex128)
    g[i0] = v[:, 0]
    Us = [sla.expm(-1j * Hf * dt * k) for k in range(nt)]

    def heis(op, k):  # c(t_k) = U^dag op U
        return Us[k].conj().T @ op @ Us[k]

    for k in range(nt):
        for l in range(nt):
            for a, (ia, sa) in enumerate(orbs):
                for b, (ib, sb) in enumerate(orbs):
                    ca, cb = c[sa * L + ia], c[sb * L + ib]
                    ref_l = 1j * (g.conj() @ heis(cb.T, l) @ heis(ca, k) @ g)
                    ref_g = -1j * (g.conj() @ heis(ca, k) @ heis(cb.T, l) @ g)
                    assert abs(Gl[k, l, a, b] - ref_l) < 1e-12
                    assert abs(Gg[k, l, a, b] - ref_g) < 1e-12


def test_keldysh_invariants_and_no_quench():
    m_i = W.siam_chain(6, 2.0, 3, 3, field=0.3)
    m_f = W.siam_chain(6, 2.0, 3, 3, field=0.0)
    orbs = [(i, 0) for i in range(6)] + [(i, 1) for i in range(6)]
    dt, nt = 0.25, 6
    Gl, Gg, _ = oracle.green_keldysh(m_i, m_f, orbs, dt, nt)
    n = len(orbs)
    for k in range(nt):
        # sum rule i (G^> - G^<)(t,t) = delta (Section 4, discussion of Fig. 2)
        assert np.max(np.abs(1j * (Gg[k, k] - Gl[k, k]) - np.eye(n))) < 1e-12
        # particle number: sum_i n_i,sigma(t) = N_sigma (n = -i G^<_ii(t,t))
        occ = (-1j * np.diag(Gl[k, k])).real
        assert abs(occ[:6].sum() - 3) < 1e-12 and abs(occ[6:].sum() - 3) < 1e-12
    # hermiticity G^<_{ab}(t,t')^* = -G^<_{ba}(t',t), same for G^>
    assert np.max(np.abs(Gl.conj() + Gl.transpose(1, 0, 3, 2))) < 1e-12
    assert np.max(np.abs(Gg.conj() + Gg.transpose(1, 0, 3, 2))) < 1e-12
    # no quench: G^<(t,t') equals the equilibrium hole part at t - t'
    Gl0, _, _ = oracle.green_keldysh(m_f, m_f, [(0, 0), (2, 0)], dt, nt)
    _, Gle, _ = oracle.green_equilibrium(m_f, [(0, 0), (2, 0)], dt, nt - 1)
    for k in range(nt):
        for l in range(k + 1):
            assert np.max(np.abs(Gl0[k, l] - Gle[k - l])) < 1e-12


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_golden_fig2_equal_time_values():
    g = _read_golden("fig2_siam_chain_t0.txt")
    L, U = int(g["L"]), g["U"]
    ini = W.siam_chain(L, U, int(g["n_up"]), int(g["n_dn"]), T=g["T"], field=g["field"])
    fin = W.siam_chain(L, U, int(g["n_up"]), int(g["n_dn"]), T=g["T"], field=0.0)
    les, gtr = oracle.keldysh_entry(ini, fin, (0, 0), (0, 0), 0.1, 0, 0)
    assert abs(les.imag - gtr.imag - g["im_les_minus_im_gtr"]) < 1e-12
    assert abs(les.real - g["re_les"]) < 1e-12 and abs(gtr.real - g["re_gtr"]) < 1e-12


def test_golden_fig4_total_polarisation():
    g = _read_golden("fig4_polarisation.txt")
    L, U = int(g["L"]), g["U"]
    ini = W.siam_chain(L, U, int(g["n_up"]), int(g["n_dn"]), T=g["T"], field=g["field"])
    fin = W.siam_chain(L, U, int(g["n_up"]), int(g["n_dn"]), T=g["T"], field=0.0)
    orbs = [(i, 0) for i in range(L)] + [(i, 1) for i in range(L)]
    Gl, _, _ = oracle.green_keldysh(ini, fin, orbs, 1.0, 3)
    for k in range(3):
        n = (-1j * np.diag(Gl[k, k])).real
        m = n[:L] - n[L:]
        assert abs(m.sum() - g["sum_m"]) < 1e-11
        assert abs(m[0]) > 1e-3  # the impurity is polarised at t = 0


# ------------------------------------------- Lanczos G(omega), Eq. (gapprox)
def _dense_resolvent_parts(m, L, orbs, omega, eta):
    c = jw_parts(L)
    H = dense_fock_h(m, c)
    i0 = sector_index(L, m["n_up"], m["n_dn"])
    w, v = np.linalg.eigh(H[np.ix_(i0, i0)])
    g = np.zeros(H.shape[0], dtype=np.complex128)
    g[i0] = v[:, 0]
    E0 = w[0]
    eye = np.eye(H.shape[0])
    out_g = np.zeros((len(orbs), omega.size), dtype=np.complex128)
    out_l = np.zeros_like(out_g)
    for a, (site, spin) in enumerate(orbs):
        ca = c[spin * L + site]
        pg, pl = ca.T @ g, ca @ g
        for k, om in enumerate(omega):
            out_g[a, k] = pg.conj() @ np.linalg.solve((om + 1j * eta + E0) * eye - H, pg)
            out_l[a, k] = pl.conj() @ np.linalg.solve((om + 1j * eta - E0) * eye + H, pl)
    return out_g, out_l, E0, H, g, c


def test_green_lanczos_full_krylov_is_exact():
    """With n at least the sector dimension the Lanczos resolvent is the exact
    one (Eq. (gomega)): compare with the dense resolvent on the Fock space."""
    L = 4
    m = W.random_model(L, 2, 1, seed=41, complex_hopping=True)
    orbs = [(0, 0), (3, 0), (2, 1)]
    omega = np.linspace(-5.0, 5.0, 23)
    Gg, Gl, E0 = oracle.green_lanczos(m, orbs, 40, omega, 0.15)
    rg, rl, e0, *_ = _dense_resolvent_parts(m, L, orbs, omega, 0.15)
    assert abs(E0 - e0) < 1e-12
    assert np.max(np.abs(Gg - rg)) < 1e-11 and np.max(np.abs(Gl - rl)) < 1e-11


def test_green_lanczos_moments_and_sum_rule():
    """With n < d the n-pole function reproduces the first 2n moments
    <0|c (H - E0)^r c^dag|0> of the high-frequency expansion (Eq. (ghigh) and
    the remark after it), and the weights of both parts sum to 1."""
    L = 4
    m = W.random_model(L, 2, 2, seed=43, complex_hopping=True)
    site, spin = 1, 0
    n = 4
    sec = oracle.Sector(m)
    E0, psi0, _ = sec.ground_state(K=80, tol=1e-13)
    *_, H, g, c = _dense_resolvent_parts(m, L, [(site, spin)], np.zeros(1), 0.1)
    ca = c[spin * L + site]
    wsum = 0.0
    for dagger in (True, False):
        nb = sec.neighbour(spin, dagger)
        v0 = sec.apply_cop(nb, site, spin, dagger, psi0)
        a, b, norm0 = oracle.lanczos_run(nb, v0, n)
        Em, Q = np.linalg.eigh(np.diag(a) + np.diag(b, 1) + np.diag(b, -1))
        wgt = (norm0 * Q[0, :]) ** 2
        wsum += wgt.sum()
        shift = -E0 if dagger else E0  # particle: H - E0; hole: -(H - E0) in the denominator
        p = (ca.T if dagger else ca) @ g
        Hs = H - E0 * np.eye(H.shape[0]) if dagger else E0 * np.eye(H.shape[0]) - H
        x = p.copy()
        for r in range(2 * n):
            exact = float((p.conj() @ x).real)
            lan = float(np.sum(wgt * ((Em + shift) if dagger else (shift - Em)) ** r))
            assert abs(lan - exact) <= 1e-9 * max(1.0, abs(exact)), (dagger, r, lan, exact)
            x = Hs @ x
    assert abs(wsum - 1.0) < 1e-12


# ---------------------------------- G(omega) from G(t), the damped transform
def _trapezoid_exp(lam, dt, n_t):
    """sum_k w_k e^{i lam t_k}, t_k = k dt, trapezoidal weights, summed in
    closed form as a geometric series in z = e^{i lam dt}."""
    if n_t < 2:
        return np.zeros_like(lam, dtype=np.complex128)
    z = np.exp(1j * lam * dt)
    return dt * ((1 - z ** n_t) / (1 - z) - 0.5 * (1 + z ** (n_t - 1)))


def test_fourier_geometric_series():
    """A sum of exponentials transforms into the closed-form geometric sums:
    pins the weights (end points halved), the sign of omega and of eta, and
    the time index of every sample."""
    rng = np.random.default_rng(61)
    E = np.array([-2.3, 0.4, 5.1])
    A = rng.normal(size=(2, 3)) + 1j * rng.normal(size=(2, 3))
    omega = np.linspace(-6.05, 6.05, 37)  # no omega equals a pole E
    for dt, n_t, eta in ((0.05, 1000, 0.0), (0.1, 7, 0.3), (0.2, 2, 0.1), (0.1, 1, 0.2)):
        t = dt * np.arange(n_t)
        G = A @ np.exp(-1j * np.outer(E, t))  # two series
        F = oracle.green_fourier(G, dt, omega, eta)
        ref = sum(A[:, m, None] * _trapezoid_exp(omega - E[m] + 1j * eta, dt, n_t)[None, :] for m in range(3))
        assert F.shape == (2, omega.size)
        assert np.max(np.abs(F - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref))), (dt, n_t, eta)
        assert np.max(np.abs(oracle.green_fourier(G[1], dt, omega, eta) - F[1])) <= 1e-12 * max(1.0, np.max(np.abs(F)))


def test_fourier_of_equilibrium_G_is_the_lehmann_sum():
    """The transform of the oracle's G^>(t) and of -G^<(t) equals the same
    trapezoidal sums taken over the Lehmann poles and weights of a dense eigh
    of the Fock-space H, and approaches the resolvent of Eq. (gomega) (the
    particle and hole parts) as dt -> 0 with e^{-eta t_max} negligible."""
    L = 4
    m = W.random_model(L, 2, 1, seed=47, complex_hopping=True)
    orbs = [(1, 0), (2, 1)]
    dt, n, eta = 0.01, 6000, 0.5  # t_max = 60, e^{-30}
    omega = np.linspace(-5.0, 5.0, 41)
    Gg, Gl, E0 = oracle.green_equilibrium(m, orbs, dt, n)
    rg, rl, e0, H, g, c = _dense_resolvent_parts(m, L, orbs, omega, eta)
    assert abs(E0 - e0) < 1e-12
    Ew, Vw = np.linalg.eigh(H)
    for a, (site, spin) in enumerate(orbs):
        ca = c[spin * L + site]
        Fg = oracle.green_fourier(Gg[:, a, a], dt, omega, eta)
        Fl = oracle.green_fourier(-Gl[:, a, a], dt, omega, eta)
        wg = np.abs(Vw.conj().T @ (ca.T @ g)) ** 2  # |<m|c^dag_a 0>|^2
        wl = np.abs(Vw.conj().T @ (ca @ g)) ** 2    # |<m|c_a 0>|^2
        lg = -1j * sum(wg[k] * _trapezoid_exp(omega - (Ew[k] - E0) + 1j * eta, dt, n + 1)
                       for k in range(Ew.size) if wg[k] > 1e-15)
        ll = -1j * sum(wl[k] * _trapezoid_exp(omega + (Ew[k] - E0) + 1j * eta, dt, n + 1)
                       for k in range(Ew.size) if wl[k] > 1e-15)
        assert np.max(np.abs(Fg - lg)) < 1e-9 and np.max(np.abs(Fl - ll)) < 1e-9
        # the quadrature error of the trapezoidal rule is (|lambda| dt)^2 / 12
        # relative, |lambda| <= 12 here
        scale = max(np.max(np.abs(rg[a])), np.max(np.abs(rl[a])))
        assert np.max(np.abs(Fg - rg[a])) < 2e-3 * scale
        assert np.max(np.abs(Fl - rl[a])) < 2e-3 * scale
        # causality: -Im of both parts is positive (the trapezoidal sum of a
        # damped exponential has a positive real part)
        assert np.min(-Fg.imag) > 0 and np.min(-Fl.imag) > 0


# ------------------------ Matsubara and mixed components (zero temperature)
def _n_total(c):
    return sum(ck.T @ ck for ck in c)


def test_matsubara_vs_jordan_wigner():
    """G^M(+tau) = -<0|c_a e^{-tau (K - K0)} c^dag_b|0> and G^M(-tau) =
    <0|c^dag_b e^{-tau (K - K0)} c_a|0> with K = H - mu N, computed with scipy
    expm on the full Fock space built from Jordan-Wigner matrices."""
    L = 4
    m = W.random_model(L, 2, 1, seed=51, complex_hopping=True)
    orbs = [(0, 0), (2, 0), (1, 1), (3, 1)]
    taus = np.array([0.0, 0.3, 1.1, 2.5])
    mu = 0.2
    Gp, Gm, E0 = oracle.green_matsubara(m, orbs, taus, mu)
    c = jw_parts(L)
    H = dense_fock_h(m, c)
    i0 = sector_index(L, 2, 1)
    w, v = np.linalg.eigh(H[np.ix_(i0, i0)])
    assert abs(E0 - w[0]) < 1e-12
    g = np.zeros(H.shape[0], dtype=np.complex128)
    g[i0] = v[:, 0]
    Kd = H - mu * _n_total(c) - (E0 - 3 * mu) * np.eye(H.shape[0])  # K - K0
    for j, tau in enumerate(taus):
        P = sla.expm(-tau * Kd)
        for a, (ia, sa) in enumerate(orbs):
            for b, (ib, sb) in enumerate(orbs):
                ca, cb = c[sa * L + ia], c[sb * L + ib]
                assert abs(Gp[j, a, b] - (-(g.conj() @ ca @ P @ cb.T @ g))) < 1e-12
                assert abs(Gm[j, a, b] - (g.conj() @ cb.T @ P @ ca @ g)) < 1e-12
    # the jump at tau = 0: G^M(0+) - G^M(0-) = -<{c_a, c^dag_b}> = -delta_ab
    assert np.max(np.abs(Gp[0] - Gm[0] + np.eye(4))) < 1e-12


def test_matsubara_and_mixed_U0_closed_form():
    """Free fermions (complex hopping, a quench of hopping and on-site
    energies): G^M(+tau) = -[e^{-(h-mu)tau}(1-rho)], G^M(-tau) =
    [e^{(h-mu)tau} rho], G^right(t,tau) = i[e^{-i h_f t} rho e^{(h_i-mu)tau}],
    G^left(tau,t) = -i[e^{-(h_i-mu)tau}(1-rho) e^{i h_f t}], rho[k,l] =
    <c^dag_l c_k> of the initial ground state."""
    L = 6
    ini = W.random_model(L, 3, 2, seed=53, complex_hopping=True)
    fin = W.random_model(L, 3, 2, seed=54, complex_hopping=True)
    ini["U"][:] = 0.0
    fin["U"][:] = 0.0
    orbs = [(0, 0), (3, 0), (5, 0), (1, 1), (4, 1)]
    taus = np.array([0.0, 0.4, 1.7])
    mu, dt, nt = 0.1, 0.25, 4
    Gp, Gm, _ = oracle.green_matsubara(ini, orbs, taus, mu)
    Gr, Gf, _ = oracle.green_mixed(ini, fin, orbs, dt, nt, taus, mu)
    for spin, N in ((0, 3), (1, 2)):
        hi = ini["h"] + np.diag(ini["eps"][spin])
        hf = fin["h"] + np.diag(fin["eps"][spin])
        w, v = np.linalg.eigh(hi)
        assert w[N] - w[N - 1] > 1e-3  # closed shell
        rho = v[:, :N] @ v[:, :N].conj().T
        one = np.eye(L)
        idx = [k for k, o in enumerate(orbs) if o[1] == spin]
        for j, tau in enumerate(taus):
            Em = sla.expm(-(hi - mu * one) * tau)
            Ep = sla.expm((hi - mu * one) * tau)
            ref_p, ref_m = -Em @ (one - rho), Ep @ rho
            for k in range(nt):
                Uf = sla.expm(-1j * hf * dt * k)
                ref_r = 1j * Uf @ rho @ Ep
                ref_f = -1j * Em @ (one - rho) @ Uf.conj().T
                for a in idx:
                    for b in idx:
                        i, jj = orbs[a][0], orbs[b][0]
                        assert abs(Gr[k, j, a, b] - ref_r[i, jj]) < 1e-12
                        assert abs(Gf[j, k, a, b] - ref_f[i, jj]) < 1e-12
            for a in idx:
                for b in idx:
                    i, jj = orbs[a][0], orbs[b][0]
                    assert abs(Gp[j, a, b] - ref_p[i, jj]) < 1e-12
                    assert abs(Gm[j, a, b] - ref_m[i, jj]) < 1e-12
    # opposite spins never mix
    assert np.all(Gr[:, :, :3, 3:] == 0) and np.all(Gf[:, :, 3:, :3] == 0)


def test_mixed_interacting_quench_vs_jordan_wigner():
    """Interacting quench on L = 3: G^right_{ab}(t,tau) = i<0|c^dag_b(tau)
    c_a(t)|0> and G^left_{ab}(tau,t) = -i<0|c_a(tau) c^dag_b(t)|0> with
    imaginary-time operators of K_ini = H_ini - mu N and real-time ones of
    H_fin, from expm on the Jordan-Wigner Fock space; and the boundary
    relations G^left(tau, 0) = i G^M(tau), G^right(0, tau) = i G^M(-tau)."""
    L = 3
    ini = W.random_model(L, 2, 1, seed=57, complex_hopping=True)
    fin = W.random_model(L, 2, 1, seed=57, complex_hopping=True)
    fin["U"] = 0.5 * ini["U"] + 1.0
    fin["eps"] = ini["eps"] - 0.3
    orbs = [(0, 0), (2, 0), (1, 1)]
    taus = np.array([0.0, 0.5, 1.3])
    mu, dt, nt = -0.15, 0.3, 5
    Gr, Gf, E0 = oracle.green_mixed(ini, fin, orbs, dt, nt, taus, mu)
    Gp, Gm, _ = oracle.green_matsubara(ini, orbs, taus, mu)
    c = jw_parts(L)
    Hi, Hf = dense_fock_h(ini, c), dense_fock_h(fin, c)
    i0 = sector_index(L, 2, 1)
    w, v = np.linalg.eigh(Hi[np.ix_(i0, i0)])
    assert abs(E0 - w[0]) < 1e-12
    g = np.zeros(Hi.shape[0], dtype=np.complex128)
    g[i0] = v[:, 0]
    Kd = Hi - mu * _n_total(c) - (E0 - 3 * mu) * np.eye(Hi.shape[0])
    for j, tau in enumerate(taus):
        P = sla.expm(-tau * Kd)
        for k in range(nt):
            U = sla.expm(-1j * Hf * dt * k)
            for a, (ia, sa) in enumerate(orbs):
                for b, (ib, sb) in enumerate(orbs):
                    ca, cb = c[sa * L + ia], c[sb * L + ib]
                    ref_r = 1j * (g.conj() @ cb.T @ P @ U.conj().T @ ca @ U @ g)
                    ref_f = -1j * (g.conj() @ ca @ P @ U.conj().T @ cb.T @ U @ g)
                    assert abs(Gr[k, j, a, b] - ref_r) < 1e-11
                    assert abs(Gf[j, k, a, b] - ref_f) < 1e-11
    assert np.max(np.abs(Gf[:, 0] - 1j * Gp)) < 1e-12
    assert np.max(np.abs(Gr[0] - 1j * Gm)) < 1e-12


def test_matsubara_hubbard_atom():
    """Half-filled atom, eps = -U/2, mu = 0: adding or removing an electron
    costs U/2, so the spin-averaged G^M(+tau) = -e^{-U tau/2}/2 and
    G^M(-tau) = e^{-U tau/2}/2."""
    U = 2.6
    taus = np.linspace(0.0, 3.0, 7)
    Gp = Gm = 0
    for nu, nd in ((1, 0), (0, 1)):
        m = W.make_model(1, nu, nd, np.zeros((1, 1)), np.full((2, 1), -U / 2), np.array([U]))
        p, q, _ = oracle.green_matsubara(m, [(0, 0), (0, 1)], taus, 0.0)
        Gp, Gm = Gp + 0.25 * (p[:, 0, 0] + p[:, 1, 1]), Gm + 0.25 * (q[:, 0, 0] + q[:, 1, 1])
    assert np.max(np.abs(Gp + 0.5 * np.exp(-U * taus / 2))) < 1e-14
    assert np.max(np.abs(Gm - 0.5 * np.exp(-U * taus / 2))) < 1e-14


def test_keldysh_entry_matches_the_gram_route():
    """The single-entry route used for sampled full-size parity equals the
    full Gram-matrix route (itself pinned to Jordan-Wigner expm and the
    free-fermion closed forms) for off-diagonal times, both spins and a
    complex-hopping quench -- a swapped time or orbital index fails."""
    ini = W.random_model(4, 2, 1, seed=71, complex_hopping=True)
    fin = W.random_model(4, 2, 1, seed=72, complex_hopping=True)
    orbs = [(0, 0), (2, 0), (1, 1), (3, 1)]
    dt, nt = 0.2, 5
    Gl, Gg, _ = oracle.green_keldysh(ini, fin, orbs, dt, nt)
    for (k, l) in ((0, 3), (4, 1), (2, 2)):
        for a, b in ((0, 1), (1, 0), (2, 3), (0, 2)):
            les, gtr = oracle.keldysh_entry(ini, fin, orbs[a], orbs[b], dt, k, l)
            assert abs(les - Gl[k, l, a, b]) < 1e-12 and abs(gtr - Gg[k, l, a, b]) < 1e-12, (k, l, a, b)


# ------------------------------------------- dense analytic gradient pins
def _dense_expm_green(model, c, orbs, dt, n):
    """G^>(t_k), G^<(t_k) from the Jordan-Wigner Fock matrices: ground state
    by eigh of the sector block, propagators by scipy expm of the whole Fock
    H (powers of one step)."""
    L = model["L"]
    H = dense_fock_h(model, c)
    i0 = sector_index(L, model["n_up"], model["n_dn"])
    w, v = np.linalg.eigh(H[np.ix_(i0, i0)])
    g = np.zeros(H.shape[0], dtype=np.complex128)
    g[i0] = v[:, 0]
    step = sla.expm(-1j * dt * H)
    U_t = np.eye(H.shape[0], dtype=np.complex128)
    no = len(orbs)
    Gg = np.zeros((n + 1, no, no), dtype=np.complex128)
    Gl = np.zeros_like(Gg)
    ops = [c[s * L + i] for (i, s) in orbs]
    for k in range(n + 1):
        t = k * dt
        for a in range(no):
            for b in range(no):
                Gg[k, a, b] = -1j * np.exp(1j * w[0] * t) * (g.conj() @ ops[a] @ U_t @ ops[b].T @ g)
                Gl[k, a, b] = 1j * np.exp(-1j * w[0] * t) * (g.conj() @ ops[b].T @ U_t.conj().T @ ops[a] @ g)
        U_t = step @ U_t
    return Gg, Gl


@pytest.mark.parametrize("seed,nu,nd", [(41, 2, 2), (42, 1, 2)])
def test_dense_gradient_vs_expm_central_differences(seed, nu, nd):
    """The analytic gradient (perturbation theory of the Lehmann form) against
    central differences (step 1e-5) of the Jordan-Wigner expm forward, for
    every parameter: eps, U, the diagonal and the real and imaginary parts of
    every hopping pair, with random complex cotangents on both parts and
    orbitals of both spins.  A dropped route (E0, |0>, the neighbour
    Hamiltonians), a sign or a conjugate fails it."""
    L = 4
    c = jw_parts(L)
    m = W.random_model(L, nu, nd, seed=seed, complex_hopping=True)
    orbs = [(0, 0), (2, 0), (1, 1)]
    dt, n = 0.15, 10
    rng = np.random.default_rng(seed)
    shape = (n + 1, len(orbs), len(orbs))
    A = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    B = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    g_eps, g_hre, g_him, g_U = oracle.green_equilibrium_grad_dense(m, orbs, dt, n, A, B)

    def loss(mm):
        Gg, Gl = _dense_expm_green(mm, c, orbs, dt, n)
        return float(np.sum((np.conj(A) * Gg).real) + np.sum((np.conj(B) * Gl).real))

    def fd(kind, i, j):
        out = []
        for dlt in (1e-5, -1e-5):
            mm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
            if kind == "eps":
                mm["eps"][i, j] += dlt
            elif kind == "U":
                mm["U"][i] += dlt
            elif kind == "re":
                mm["h"][i, j] += dlt
                if i != j:
                    mm["h"][j, i] += dlt
            else:
                mm["h"][i, j] += 1j * dlt
                mm["h"][j, i] -= 1j * dlt
            out.append(loss(mm))
        return (out[0] - out[1]) / 2e-5

    checks = [(g_eps[s, i], fd("eps", s, i)) for s in range(2) for i in range(L)]
    checks += [(g_U[i], fd("U", i, None)) for i in range(L)]
    checks += [(g_hre[i, j], fd("re", i, j)) for i in range(L) for j in range(i, L)]
    checks += [(g_him[i, j], fd("im", i, j)) for i in range(L) for j in range(i + 1, L)]
    scale = max(1.0, max(abs(r) for _, r in checks))
    for k, (g, r) in enumerate(checks):
        assert abs(g - r) < 1e-7 * scale, (k, g, r)
    # the tied conventions: symmetric real part, antisymmetric imaginary part
    assert np.array_equal(g_hre, g_hre.T) and np.array_equal(g_him, -g_him.T)
    # the diagonal of h acts like eps on both spins
    assert np.max(np.abs(np.diag(g_hre) - g_eps.sum(0))) < 1e-9 * scale


def test_dense_gradient_U0_translation_and_zero_cotangent():
    """Zero cotangents give a zero gradient; on the translation-invariant U = 0
    ring with the loss of a site-diagonal function summed over all sites, every
    site's eps gradient is the same (symmetry of the loss)."""
    L = 6
    m = W.hubbard_ring(L, 0.0, 2, 2, pbc=False)
    m["h"] = W.ring_hopping(L, 1.0, pbc=True).astype(np.complex128)
    m["h"][0, 1] = m["h"][1, 0] = -1.0 + 0.0j
    # antiperiodic twist keeps the 6-ring closed-shell at (2,2)
    m["h"][0, L - 1] = m["h"][L - 1, 0] = 1.0
    orbs = [(i, 0) for i in range(L)]
    dt, n = 0.1, 8
    g0 = oracle.green_equilibrium_grad_dense(m, orbs, dt, n)
    assert all(np.max(np.abs(x)) == 0.0 for x in g0)
    A = np.zeros((n + 1, L, L), dtype=np.complex128)
    for i in range(L):
        A[:, i, i] = 1.0 + 0.5j
    g_eps, _, _, _ = oracle.green_equilibrium_grad_dense(m, orbs, dt, n, A, A)
    assert np.max(np.abs(g_eps[0] - g_eps[0, 0])) < 1e-9 * max(1.0, abs(g_eps[0, 0]))


def test_keldysh_entries_share_work_and_match_single_entries():
    """The batched sampling route gives the single-entry route's numbers (which
    are pinned to the Gram route above) for a mix of times, orbitals and
    spins, including a pair of opposite spins (zero)."""
    ini = W.random_model(4, 2, 1, seed=73, complex_hopping=True)
    fin = W.random_model(4, 2, 1, seed=74, complex_hopping=True)
    dt = 0.25
    samples = [(3, 0, (0, 0), (2, 0)), (1, 4, (2, 0), (0, 0)), (4, 4, (1, 1), (3, 1)), (2, 2, (0, 0), (1, 1)),
               (0, 3, (3, 1), (3, 1))]
    got = oracle.keldysh_entries(ini, fin, samples, dt)
    for (k, l, a, b), (les, gtr) in zip(samples, got):
        rl, rg = oracle.keldysh_entry(ini, fin, a, b, dt, k, l)
        assert abs(les - rl) < 1e-13 and abs(gtr - rg) < 1e-13, (k, l, a, b)
    assert got[3] == (0j, 0j)


@pytest.mark.parametrize("seed,L,nu,nd", [(81, 5, 2, 3), (82, 6, 3, 1), (83, 4, 4, 2)])
def test_dense_lehmann_route_equals_chebyshev_route(seed, L, nu, nd):
    """The dense Lehmann route (used for many small instances at once) equals
    the Chebyshev route (pinned above to Jordan-Wigner expm, closed forms and
    the Hubbard atom) for complex hopping, both spins, a full band (no
    particle part) and off-diagonal orbital pairs."""
    m = W.random_model(L, nu, nd, seed=seed, complex_hopping=True)
    orbs = [(0, 0), (L - 1, 0), (1, 1), (2, 1)]
    dt, n = 0.1, 30
    Gg, Gl, E0, gap = oracle.green_equilibrium_dense(m, orbs, dt, n)
    rg, rl, e_or = oracle.green_equilibrium(m, orbs, dt, n, K=max(80, 200), tol=1e-14)
    assert gap > 1e-6 and abs(E0 - e_or) < 1e-12 * max(1.0, abs(e_or))
    assert np.max(np.abs(Gg - rg)) < 1e-11 and np.max(np.abs(Gl - rl)) < 1e-11
    if nu == L:
        assert np.all(Gg[:, :2, :2] == 0)


# ------------------------------------------- time-dependent H(t) (Section 6)
def _td_field(t, L):
    """A smooth drive: every on-site energy and the impurity U oscillate."""
    p = np.zeros(3 * L)
    for s in range(2):
        for i in range(L):
            p[s * L + i] = 0.7 * np.sin(1.3 * t + 0.5 * i + 1.1 * s)
    p[2 * L] = 0.8 * np.cos(2.1 * t)
    return p


def _td_dparams(field, dt, n_t, n_sub, L):
    h = dt / n_sub
    return np.array([[field(s * h + c * h, L) for c in oracle.CF4_C]
                     for s in range((n_t - 1) * n_sub)])


def _td_dense_reference(ini, fin, orbs, dt, nt, field, L, nu, nd):
    """G^<, G^> from a dense Jordan-Wigner H(t) on the whole Fock space, the
    propagator U(t, 0) integrated by scipy's DOP853 to 1e-13."""
    import scipy.integrate as sint
    c = jw_parts(L)
    Hf = dense_fock_h(fin, c)
    num = [c[q].T @ c[q] for q in range(2 * L)]
    ops = num + [num[i] @ num[L + i] for i in range(L)]
    dim = Hf.shape[0]

    def rhs(t, y):
        p = field(t, L)
        H = Hf + sum(p[q] * ops[q] for q in range(3 * L))
        return (-1j * (H @ y.reshape(dim, dim))).ravel()
    sol = sint.solve_ivp(rhs, (0.0, dt * (nt - 1)), np.eye(dim, dtype=np.complex128).ravel(),
                         method="DOP853", rtol=1e-13, atol=1e-14, t_eval=dt * np.arange(nt))
    assert sol.status == 0
    Us = [sol.y[:, k].reshape(dim, dim) for k in range(nt)]
    Hi = dense_fock_h(ini, c)
    i0 = sector_index(L, nu, nd)
    w, v = np.linalg.eigh(Hi[np.ix_(i0, i0)])
    g = np.zeros(dim, dtype=np.complex128)
    g[i0] = v[:, 0]
    n = len(orbs)
    Rl = np.zeros((nt, nt, n, n), dtype=np.complex128)
    Rg = np.zeros_like(Rl)
    heis = [[Us[k].conj().T @ c[s * L + i] @ Us[k] for (i, s) in orbs] for k in range(nt)]
    for k in range(nt):
        for l in range(nt):
            for a in range(n):
                for b in range(n):
                    ca, cbd = heis[k][a], heis[l][b].conj().T
                    Rl[k, l, a, b] = 1j * (g.conj() @ cbd @ ca @ g)
                    Rg[k, l, a, b] = -1j * (g.conj() @ ca @ cbd @ g)
    return Rl, Rg


def test_cf4_fourth_order_vs_dense_ode():
    """The commutator-free step converges to the exact driven G with order
    four (error ratio ~16 per halving of h); the exponentials in the other
    order (a planted swap) fall to order two and fail this."""
    L, nu, nd = 3, 2, 1
    ini = W.siam_chain(L, 2.0, nu, nd, field=0.4)
    fin = W.siam_chain(L, 2.0, nu, nd, field=0.0)
    orbs = [(0, 0), (1, 0), (2, 1)]
    dt, nt = 0.4, 5
    Rl, Rg = _td_dense_reference(ini, fin, orbs, dt, nt, _td_field, L, nu, nd)
    errs = []
    for n_sub in (2, 4, 8):
        Gl, Gg, _ = oracle.green_keldysh_td(ini, fin, orbs, dt, nt,
                                            _td_dparams(_td_field, dt, nt, n_sub, L), n_sub=n_sub)
        errs.append(max(np.max(np.abs(Gl - Rl)), np.max(np.abs(Gg - Rg))))
    assert errs[-1] < 5e-8, errs
    for e0, e1 in zip(errs, errs[1:]):
        assert 13.0 < e0 / e1 < 20.0, errs


def test_cf4_constant_offsets_equal_the_shifted_quench():
    """Offsets constant in time make every step exact: the driven G equals the
    quench G of Section 4 with the offsets added to H_fin; a zero drive gives
    the plain quench.  The sum rule holds at every time either way."""
    L = 4
    ini = W.siam_chain(L, 3.0, 2, 2, field=0.5)
    fin = W.siam_chain(L, 3.0, 2, 2, field=0.0)
    orbs = [(0, 0), (0, 1), (1, 1)]
    dt, nt, n_sub = 0.3, 4, 3
    p0 = _td_field(0.37, L)
    dp = np.tile(p0, ((nt - 1) * n_sub, 2, 1))
    Gl, Gg, _ = oracle.green_keldysh_td(ini, fin, orbs, dt, nt, dp, n_sub=n_sub)
    Gl2, Gg2, _ = oracle.green_keldysh(ini, oracle._shifted(fin, p0), orbs, dt, nt)
    assert rel(Gl, Gl2) < 1e-12 and rel(Gg, Gg2) < 1e-12
    Gl0, Gg0, _ = oracle.green_keldysh_td(ini, fin, orbs, dt, nt, 0 * dp, n_sub=n_sub)
    Gl3, Gg3, _ = oracle.green_keldysh(ini, fin, orbs, dt, nt)
    assert rel(Gl0, Gl3) < 1e-12 and rel(Gg0, Gg3) < 1e-12
    dp = _td_dparams(_td_field, dt, nt, n_sub, L)
    Gl, Gg, _ = oracle.green_keldysh_td(ini, fin, orbs, dt, nt, dp, n_sub=n_sub)
    for k in range(nt):
        assert np.max(np.abs(1j * (np.diagonal(Gg[k, k]) - np.diagonal(Gl[k, k])) - 1.0)) < 1e-12
    for G in (Gl, Gg):
        assert np.max(np.abs(np.conj(G) + G.transpose(1, 0, 3, 2))) < 1e-12


def test_cf4_nodes_and_weights():
    """The two exponentials' weights sum to the step (a1 + a2 = 1/2 each) and
    the nodes are the two-point Gauss-Legendre nodes on [0, 1]."""
    assert abs(2 * (oracle.CF4_A1 + oracle.CF4_A2) - 1.0) < 1e-15
    x, _ = np.polynomial.legendre.leggauss(2)
    assert np.allclose(sorted(oracle.CF4_C), (x + 1) / 2, atol=1e-15)
    first, second = oracle.cf4_exponents(np.array([[[1.0], [0.0]]]))
    assert abs(first[0, 0] - 2 * oracle.CF4_A2) < 1e-15 and abs(second[0, 0] - 2 * oracle.CF4_A1) < 1e-15


# ------------------------------------- four-time correlations (Section 6)
FOUR_OPS = [[(0, 0, 0), (2, 1, 0), (1, 1, 1), (0, 0, 1)],   # c c c^dag c^dag, both spins
            [(1, 0, 1), (1, 0, 0), (0, 1, 1), (2, 1, 0)],   # c^dag c c^dag c
            [(0, 0, 1), (1, 0, 0), (2, 0, 1), (0, 0, 0)]]   # one spin: c^dag c c^dag c


@pytest.mark.parametrize("ops", FOUR_OPS)
def test_four_time_vs_dense_jordan_wigner(ops):
    """<0|A1(t1) A2(t2) A3(t3) A4(t4)|0> after a field quench on L = 3 (U = 2)
    against Heisenberg operators U^dag A U built from Jordan-Wigner matrices
    and scipy expm on the 64-state Fock space, all 4^4 time combinations."""
    L = 3
    c = jw_parts(L)
    ini = W.siam_chain(L, 2.0, 2, 1, field=0.4)
    fin = W.siam_chain(L, 2.0, 2, 1, field=0.0)
    dt, nt = 0.3, 4
    G = oracle.green_four_time(ini, fin, ops, dt, nt)
    Hi, Hf = dense_fock_h(ini, c), dense_fock_h(fin, c)
    i0 = sector_index(L, 2, 1)
    w, v = np.linalg.eigh(Hi[np.ix_(i0, i0)])
    g = np.zeros(Hi.shape[0], dtype=np.complex128)
    g[i0] = v[:, 0]
    Us = [sla.expm(-1j * Hf * dt * k) for k in range(nt)]
    mats = [c[s * L + i].T if dag else c[s * L + i] for (i, s, dag) in ops]
    heis = [[Us[k].conj().T @ m @ Us[k] for k in range(nt)] for m in mats]
    for k in np.ndindex(nt, nt, nt, nt):
        ref = g.conj() @ heis[0][k[0]] @ heis[1][k[1]] @ heis[2][k[2]] @ heis[3][k[3]] @ g
        assert abs(G[k] - ref) < 1e-12, (k, G[k], ref)
    assert np.max(np.abs(G)) > 1e-2


def test_four_time_free_fermions_wick():
    """U = 0 quench of random complex hoppings (L = 5, (3, 2)): the four-time
    function factorises by Wick's theorem into two-time functions
    <c_x(t) c^dag_y(t')> = [u(t) (1 - rho) u(t')^dag]_xy of the single-particle
    propagator u(t) = e^{-i h_f t} and the initial one-body density rho:
    <c_a c_b c^dag_c c^dag_d> = <c_a c^dag_d><c_b c^dag_c> - <c_a c^dag_c><c_b c^dag_d>."""
    L = 5
    ini = W.random_model(L, 3, 2, seed=21, complex_hopping=True)
    fin = W.random_model(L, 3, 2, seed=22, complex_hopping=True)
    ini["U"][:] = 0.0
    fin["U"][:] = 0.0
    dt, nt = 0.25, 4
    P = {}
    for spin, N in ((0, 3), (1, 2)):
        w, v = np.linalg.eigh(ini["h"] + np.diag(ini["eps"][spin]))
        assert w[N] - w[N - 1] > 1e-3
        rho = v[:, :N] @ v[:, :N].conj().T
        hf = fin["h"] + np.diag(fin["eps"][spin])
        u = [sla.expm(-1j * hf * dt * k) for k in range(nt)]
        P[spin] = [[u[k] @ (np.eye(L) - rho) @ u[l].conj().T for l in range(nt)] for k in range(nt)]

    def two(x, y, k, l):  # <c_x(t_k) c^dag_y(t_l)>
        return P[x[1]][k][l][x[0], y[0]] if x[1] == y[1] else 0.0

    for ops in ([(0, 0, 0), (3, 1, 0), (1, 1, 1), (4, 0, 1)], [(0, 0, 0), (2, 0, 0), (4, 0, 1), (1, 0, 1)]):
        G = oracle.green_four_time(ini, fin, ops, dt, nt)
        a, b, cc, d = ops
        for k in np.ndindex(nt, nt, nt, nt):
            ref = (two(a, d, k[0], k[3]) * two(b, cc, k[1], k[2]) - two(a, cc, k[0], k[2]) * two(b, d, k[1], k[3]))
            assert abs(G[k] - ref) < 1e-12, (ops, k)


def test_four_time_particle_number_selection():
    """Operators that change the particle numbers give zero; a product with
    A1 A2 = c_a c_a vanishes identically (Pauli)."""
    L = 3
    ini = W.siam_chain(L, 2.0, 2, 1, field=0.4)
    fin = W.siam_chain(L, 2.0, 2, 1, field=0.0)
    G = oracle.green_four_time(ini, fin, [(0, 0, 0), (1, 0, 0), (2, 0, 0), (0, 0, 1)], 0.3, 3)
    assert np.all(G == 0)
    G = oracle.green_four_time(ini, fin, [(1, 0, 0), (1, 0, 0), (0, 0, 1), (2, 0, 1)], 0.3, 3)
    for k in range(3):
        assert np.max(np.abs(G[k, k])) < 1e-14


# ------------------------------------------------------- NE-CPT (Section 5)
def _free_chain_occupations(L_c, L_b, V, h, beta, dt, n_t):
    """Exact occupations of the non-interacting cluster + bath chain after the
    field quench: n_i(t) = [e^{-i h_f t} f(h_ini) e^{i h_f t}]_ii with the
    Fermi function at inverse temperature beta (single-particle matrices)."""
    N = L_c + L_b
    hop = -(np.eye(N, k=1) + np.eye(N, k=-1))
    hop[L_c - 1, L_c] = hop[L_c, L_c - 1] = -V
    out = np.zeros((2, n_t, L_c))
    for spin, sg in ((0, -1.0), (1, 1.0)):
        hi = hop.copy()
        hi[0, 0] += sg * h
        e, v = np.linalg.eigh(hi)
        rho = (v / (np.exp(beta * e) + 1.0)) @ v.T
        for k in range(n_t):
            U = sla.expm(-1j * hop * dt * k)
            out[spin, k] = np.real(np.diag(U @ rho @ U.conj().T))[:L_c]
    return out


def test_necpt_decoupled_is_the_isolated_cluster():
    """V = 0: the contour equation returns the cluster's own occupations
    n_i(t) = -i G^<_ii(t, t) of the four-step method."""
    L = 4
    ini = W.siam_chain(L, 1.0, 2, 2, field=0.2)
    fin = W.siam_chain(L, 1.0, 2, 2, field=0.0)
    n = oracle.necpt_occupations(ini, fin, 100, 1.0, 0.0, 0.1, 6, 15.0, 150)
    Gl, _, _ = oracle.green_keldysh(ini, fin, [(i, s) for s in (0, 1) for i in range(L)], 0.1, 6)
    for k in range(6):
        occ = (-1j * np.diagonal(Gl[k, k])).real
        assert np.max(np.abs(n[0, k] - occ[:L])) < 1e-12 and np.max(np.abs(n[1, k] - occ[L:])) < 1e-12


def test_necpt_free_fermions_converge_to_the_exact_chain():
    """U = 0: cluster perturbation theory is exact for non-interacting
    electrons, so the occupations of the L_c = 4 cluster inside the 204-site
    chain must approach the exact single-particle result at inverse
    temperature beta = 15 as the contour steps shrink (second order of the
    trapezoidal rule: 5.1e-3, 1.3e-3, 3.7e-4 at dt = dtau = 0.2, 0.1, 0.05),
    down to the e^{-beta gap} of the zero-temperature cluster.  A wrong sign
    of the bath coupling, a dropped antiperiodic tail or a transposed mixed
    component leaves errors of order 1e-2 that do not shrink."""
    L, L_b, beta, h = 4, 200, 15.0, 0.2
    ini = W.siam_chain(L, 0.0, 2, 2, field=h)
    fin = W.siam_chain(L, 0.0, 2, 2, field=0.0)
    errs = []
    for dt in (0.2, 0.1, 0.05):
        n_t = int(round(0.6 / dt)) + 1
        n = oracle.necpt_occupations(ini, fin, L_b, 1.0, 1.0, dt, n_t, beta, int(round(beta / dt)))
        errs.append(np.max(np.abs(n - _free_chain_occupations(L, L_b, 1.0, h, beta, dt, n_t))))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 2.5, errs
    assert errs[2] < 6e-4, errs


def test_necpt_particle_hole_symmetry():
    """The half-filled, particle-hole symmetric chain with the impurity field
    keeps n_iup(t) + n_idn(t) = 1 at every site and time; the discretised
    equation approaches it at second order."""
    L = 4
    ini = W.siam_chain(L, 1.0, 2, 2, field=0.2)
    fin = W.siam_chain(L, 1.0, 2, 2, field=0.0)
    dev = []
    for dt in (0.2, 0.1):
        n_t = int(round(0.4 / dt)) + 1
        n = oracle.necpt_occupations(ini, fin, 100, 1.0, 1.0, dt, n_t, 15.0, int(round(15.0 / dt)))
        dev.append(np.max(np.abs(n[0] + n[1] - 1.0)))
    assert dev[1] < 3e-3 and dev[0] / dev[1] > 3.0, dev


def test_four_time_equilibrium_depends_on_differences_only():
    """Without a quench (H_ini = H_fin) the four-time function depends only on
    the time differences: shifting all four times by one grid step leaves it
    unchanged (the ground state is stationary)."""
    m = W.random_model(4, 2, 1, seed=5, complex_hopping=True)
    ops = [(1, 0, 0), (2, 1, 1), (0, 1, 0), (3, 0, 1)]
    G = oracle.green_four_time(m, m, ops, 0.2, 4)
    assert np.max(np.abs(G)) > 1e-3
    for k in np.ndindex(3, 3, 3, 3):
        assert abs(G[k] - G[tuple(x + 1 for x in k)]) < 1e-12
