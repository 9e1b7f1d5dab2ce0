"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: integer/index work (strings, c/c^dag maps) bit-exact; H*psi to
1e-12 relative (one FP64 summation order against another); propagated
vectors 1e-11 absolute (unit vectors, tens of Krylov steps); ground-state
energy 1e-12 relative and Green's functions 1e-10 absolute (the stated
parity bar of this path).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1109_1205_gb300 as kg  # noqa: E402

G_TOL = 1e-10
E_TOL = 1e-12


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def stream():
    return torch.cuda.current_stream()


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


# --------------------------------------------------------------- ranking
@pytest.mark.parametrize("L,nu,nd", [(1, 0, 1), (6, 3, 2), (12, 6, 6), (16, 7, 8), (20, 3, 17)])
def test_strings_are_rank_ordered(L, nu, nd):
    s = kg.Sector(W.hubbard_ring(L, 1.0, nu, nd))
    up, dn = s.strings()
    for arr, n in ((up, nu), (dn, nd)):
        assert len(arr) == math.comb(L, n)
        if L <= 16:
            ref = np.array(sorted(x for x in range(1 << L) if bin(x).count("1") == n), dtype=np.uint32)
            assert np.array_equal(arr, ref)
        else:
            assert np.all(np.diff(arr.astype(np.int64)) > 0)
            assert all(bin(int(x)).count("1") == n for x in arr[:: max(1, len(arr) // 997)])
    assert s.dim == math.comb(L, nu) * math.comb(L, nd)


# ------------------------------------------------------------------ H*psi
HPSI_MODELS = [
    ("complex", W.random_model(6, 3, 2, seed=1, complex_hopping=True)),
    ("real-nonuniform", W.random_model(8, 4, 3, seed=2, complex_hopping=False, density=0.6)),
    ("ring-uniform", W.hubbard_ring(10, 4.0, 5, 4)),
    ("c1-star", W.config_c1()["model"]),
    ("chain-field", W.siam_chain(9, 3.0, 4, 5, field=0.7)),
    ("c2-ring-full", W.config_c2()["fin"]),
]


@pytest.mark.parametrize("name,model", HPSI_MODELS, ids=[m[0] for m in HPSI_MODELS])
def test_hpsi_parity(name, model):
    s = kg.Sector(model)
    o = oracle.Sector(model)
    assert s.dim == o.dim
    x = W.random_state(s.dim, 7)
    xd = dev(x)
    yd = torch.empty_like(xd)
    s.hpsi(xd, yd, stream())
    y = host(yd)
    ref = o.hpsi(x)
    assert relerr(y, ref) < 1e-12, name


def test_hpsi_linearity_and_hermiticity():
    m = W.random_model(7, 3, 3, seed=4, complex_hopping=True)
    s = kg.Sector(m)
    x, z = W.random_state(s.dim, 1), W.random_state(s.dim, 2)
    yx, yz = torch.empty(s.dim, dtype=torch.complex128, device="cuda"), torch.empty(s.dim, dtype=torch.complex128,
                                                                                 device="cuda")
    s.hpsi(dev(x), yx, stream())
    s.hpsi(dev(z), yz, stream())
    hx, hz = host(yx), host(yz)
    assert abs(np.vdot(z, hx) - np.vdot(hz, x)) < 1e-12


# ------------------------------------------------------------ c / c^dag
def test_cop_bit_exact():
    m = W.random_model(6, 3, 2, seed=9, complex_hopping=True)
    s = kg.Sector(m)
    o = oracle.Sector(m)
    x = W.random_state(s.dim, 3)
    xd = dev(x)
    for spin in (0, 1):
        for dagger in (False, True):
            on = o.neighbour(spin, dagger)
            dn = s.neighbour_dim(spin, dagger)
            assert dn == on.dim
            for site in range(6):
                yd = torch.empty(dn, dtype=torch.complex128, device="cuda")
                s.apply_cop(site, spin, dagger, xd, yd, stream())
                assert np.array_equal(host(yd), o.apply_cop(on, site, spin, dagger, x)), (site, spin, dagger)


def test_cop_missing_neighbour_is_einval():
    s = kg.Sector(W.hubbard_ring(4, 1.0, 4, 0))
    with pytest.raises(kg.KGError) as e:
        s.neighbour_dim(0, True)  # N_up = L: no room for c^dag_up
    assert e.value.code == kg.KG_EINVAL
    with pytest.raises(kg.KGError):
        s.neighbour_dim(1, False)  # N_dn = 0: nothing to annihilate


# ------------------------------------------------------- overlaps
@pytest.mark.parametrize("n_x,n_y,d", [(1, 1, 1), (3, 5, 1000), (12, 12, 731808), (32, 40, 4097), (17, 1, 300001)])
def test_overlaps_parity(n_x, n_y, d):
    rng = np.random.default_rng(n_x * 1000 + n_y)
    X = rng.standard_normal((n_x, d)) + 1j * rng.standard_normal((n_x, d))
    Y = rng.standard_normal((n_y, d)) + 1j * rng.standard_normal((n_y, d))
    G = torch.empty((n_y, n_x), dtype=torch.complex128, device="cuda")
    Xd, Yd = dev(X), dev(Y)
    kg.kg_overlaps(Xd, n_x, Yd, n_y, d, G, stream())
    ref = np.conj(X) @ Y.T  # ref[a, b] = <x_a | y_b>
    got = host(G)
    assert np.max(np.abs(got - ref.T)) < 1e-12 * max(1.0, np.sqrt(d))
    # deterministic: a second call gives the same bits
    G2 = torch.empty_like(G)
    kg.kg_overlaps(Xd, n_x, Yd, n_y, d, G2, stream())
    assert np.array_equal(host(G2), got)


def test_overlaps_rejects_bad_sizes():
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    for n_x, n_y, d in ((0, 1, 8), (33, 1, 8), (1, 0, 8), (1, 1, 0)):
        with pytest.raises(kg.KGError) as e:
            kg.kg_overlaps(x, n_x, x, n_y, d, x, stream())
        assert e.value.code == kg.KG_EINVAL


# ---------------------------------------------------------- ground state
GS_MODELS = [
    ("c1", W.config_c1()["model"]),
    ("complex-L7", W.random_model(7, 3, 4, seed=5, complex_hopping=True)),
    ("ring-L10", W.hubbard_ring(10, 4.0, 5, 5)),
    ("chain-field", W.siam_chain(8, 1.0, 4, 4, field=0.2)),
    ("tiny-d1", W.make_model(2, 2, 0, W.chain_hopping(2), None, [1.0, 2.0])),
    ("d-below-M", W.random_model(4, 1, 2, seed=3)),
]


@pytest.mark.parametrize("name,model", GS_MODELS, ids=[m[0] for m in GS_MODELS])
def test_ground_state_parity(name, model):
    s = kg.Sector(model)
    E0, res, _ = s.ground_state()
    e_or, psi_or, _ = oracle.Sector(model).ground_state()
    assert abs(E0 - e_or) <= E_TOL * max(1.0, abs(e_or)), (E0, e_or)
    assert res <= 1e-12 * max(1.0, abs(E0))
    psi = s.ground_state_vector()
    assert abs(np.linalg.norm(psi) - 1) < 1e-13
    assert abs(abs(np.vdot(psi_or, psi)) - 1) < 1e-10


# ------------------------------------------------------------ propagation
@pytest.mark.parametrize("reorth", [0, 1, 2])
@pytest.mark.parametrize("dt,n", [(0.05, 20), (-0.05, 12), (0.1, 5)])
def test_propagate_parity(reorth, dt, n):
    m = W.random_model(7, 3, 3, seed=11, complex_hopping=True)
    s = kg.Sector(m)
    o = oracle.Sector(m)
    x = W.random_state(s.dim, 5)
    xd = dev(x)
    s.propagate(xd, dt, n, kg.kg_opts_default(reorth=reorth))
    y = host(xd)
    ref = o.propagate(x, dt * n)
    assert np.max(np.abs(y - ref)) < 1e-11
    assert abs(np.linalg.norm(y) - 1) < 1e-12


@pytest.mark.parametrize("schedule", list(range(8)))
def test_hop_sum_schedules(schedule):
    """Exact integer hop sums (schedule bit 0 clear) and FP64 hop sums (bit 0
    set), with the step exponential by Taylor series (bit 1 clear) or by the
    eigen-decomposition of T (bit 1 set), with exact integer Gram-Schmidt
    dots (bit 2 clear) or FP64 ones (bit 2 set), on uniform-hopping models,
    through propagation and the ground state."""
    for model in (W.hubbard_ring(10, 4.0, 5, 4), W.siam_chain(9, 3.0, 4, 5, field=0.7)):
        s = kg.Sector(model)
        o = oracle.Sector(model)
        x = W.random_state(s.dim, 12)
        xd = dev(x)
        opts = kg.kg_opts_default(schedule=schedule)
        s.propagate(xd, -0.05, 10, opts)
        assert np.max(np.abs(host(xd) - o.propagate(x, -0.5))) < 1e-11
        E0, _, _ = s.ground_state(opts)
        e_or, _, _ = o.ground_state()
        assert abs(E0 - e_or) <= E_TOL * max(1.0, abs(e_or))


@pytest.mark.parametrize("reorth", [1, 2])
def test_exact_dots_equal_fp64_dots(reorth):
    """The exact integer Gram-Schmidt dots and the FP64 ones give the same
    propagation to rounding, for complex hopping and a vector whose components
    span 30 decades (the fixed-point images keep 52 bits of each vector's
    largest component), and both match the oracle."""
    m = W.random_model(8, 4, 3, seed=29, complex_hopping=True)
    s = kg.Sector(m)
    rng = np.random.default_rng(31)
    x = W.random_state(s.dim, 14) * 10.0 ** rng.uniform(-30, 0, s.dim)
    x /= np.linalg.norm(x)
    out = []
    for schedule in (0, 4):
        xd = dev(x)
        s.propagate(xd, 0.05, 12, kg.kg_opts_default(schedule=schedule, reorth=reorth))
        out.append(host(xd))
    assert np.max(np.abs(out[0] - out[1])) < 1e-13
    ref = oracle.Sector(m).propagate(x, 0.6)
    assert np.max(np.abs(out[0] - ref)) < 1e-11


def test_integer_hop_sums_wide_dynamic_range():
    """A vector whose components span many decades (and exact zeros) through
    the exact-sum H*psi: the result must match the oracle component-wise to
    the precision of the largest component."""
    m = W.hubbard_ring(8, 2.0, 4, 3)
    s = kg.Sector(m)
    o = oracle.Sector(m)
    rng = np.random.default_rng(3)
    x = W.random_state(s.dim, 13) * 10.0 ** rng.uniform(-30, 0, s.dim)
    x[::7] = 0.0
    xd = dev(x)
    yd = torch.empty_like(xd)
    s.hpsi(xd, yd, stream())
    y = host(yd)
    ref = o.hpsi(x)
    assert np.max(np.abs(y - ref)) < 1e-15 * np.max(np.abs(x)) * 20


def test_propagate_large_sector_and_graphs():
    m = W.hubbard_ring(10, 4.0, 5, 4)
    s = kg.Sector(m)
    o = oracle.Sector(m)
    x = W.random_state(s.dim, 6)
    for graphs in (0, 1):
        xd = dev(x)
        s.propagate(xd, 0.05, 8, kg.kg_opts_default(use_graphs=graphs))
        assert np.max(np.abs(host(xd) - o.propagate(x, 0.4))) < 1e-11


@pytest.mark.parametrize("M", [12, 40])
def test_step_exponential_taylor_vs_eigen(M):
    """The two forms of e^{-iT tau} e_1 (scaled Taylor series; implicit-QR
    eigen-decomposition) agree to rounding, with M on both sides of 32 (one
    or two components per lane) and a step large enough for sub-steps."""
    m = W.random_model(7, 3, 3, seed=17, complex_hopping=True)
    s = kg.Sector(m)
    x = W.random_state(s.dim, 8)
    out = []
    for schedule in (0, 2):
        xd = dev(x)
        s.propagate(xd, 0.3, 4, kg.kg_opts_default(M=M, schedule=schedule))
        out.append(host(xd))
    # same Krylov spaces, so the two agree to rounding whatever M is
    assert np.max(np.abs(out[0] - out[1])) < 1e-12
    if M == 40:  # and with enough Krylov vectors, with the oracle
        ref = oracle.Sector(m).propagate(x, 1.2)
        assert np.max(np.abs(out[0] - ref)) < 1e-11


@pytest.mark.parametrize("model", [W.hubbard_ring(14, 4.0, 7, 6), W.siam_chain(14, 3.0, 6, 7, field=0.5)],
                         ids=["ring14_7_6", "chain14_6_7"])
def test_hpsi_and_propagation_beyond_l2(model):
    """Sectors whose vectors exceed the 129 MB L2 (d = 10,306,296, 165 MB;
    D_up = 3432 or 3003, D_dn odd in one): the standalone kg_hpsi matches the
    oracle's H*psi to 1e-12 relative and three propagation steps match the
    oracle's Chebyshev propagation to 1e-11."""
    s = kg.Sector(model)
    o = oracle.Sector(model)
    assert s.dim == 10_306_296 and 16 * s.dim > (129 << 20)
    x = W.random_state(s.dim, 31)
    y = torch.empty(s.dim, dtype=torch.complex128, device="cuda")
    s.hpsi(dev(x), y, stream())
    assert relerr(host(y), o.hpsi(x)) < 1e-12
    xd = dev(x)
    s.propagate(xd, 0.05, 3)
    assert np.max(np.abs(host(xd) - o.propagate(x, 0.15))) < 1e-11


def test_bad_schedule_rejected():
    s = kg.Sector(W.random_model(4, 2, 2, seed=1))
    with pytest.raises(kg.KGError):
        s.green_equilibrium([(0, 0)], 0.1, 2, kg.kg_opts_default(schedule=8))


# ------------------------------------------------------- equilibrium G
def test_green_equilibrium_c1_full():
    cfg = W.config_c1()
    s = kg.Sector(cfg["model"])
    opts = kg.kg_opts_default(M=cfg["M"], M_gs=cfg["M"])
    Gg, Gl = s.green_equilibrium(cfg["orbitals"], cfg["dt"], cfg["n_steps"], opts)
    rg, rl, _ = oracle.green_equilibrium(cfg["model"], cfg["orbitals"], cfg["dt"], cfg["n_steps"])
    assert np.max(np.abs(Gg - rg)) < G_TOL
    assert np.max(np.abs(Gl - rl)) < G_TOL
    # sum rule at t = 0
    assert abs(1j * (Gg[0, 0, 0] - Gl[0, 0, 0]) - 1) < 1e-12


@pytest.mark.parametrize("reorth", [0, 1, 2])
def test_green_equilibrium_both_spins(reorth):
    m = W.random_model(6, 3, 2, seed=21, complex_hopping=True)
    orbs = [(0, 0), (2, 0), (5, 0), (1, 1), (4, 1)]
    s = kg.Sector(m)
    Gg, Gl = s.green_equilibrium(orbs, 0.1, 30, kg.kg_opts_default(reorth=reorth))
    rg, rl, _ = oracle.green_equilibrium(m, orbs, 0.1, 30)
    assert np.max(np.abs(Gg - rg)) < G_TOL
    assert np.max(np.abs(Gl - rl)) < G_TOL


def test_green_equilibrium_edge_sectors():
    # full up band: no particle part for spin up; empty down band: no hole part
    m = W.make_model(3, 3, 0, W.chain_hopping(3), None, [2.0, 1.0, 0.5])
    s = kg.Sector(m)
    orbs = [(0, 0), (1, 1)]
    Gg, Gl = s.green_equilibrium(orbs, 0.2, 6)
    rg, rl, _ = oracle.green_equilibrium(m, orbs, 0.2, 6)
    assert np.max(np.abs(Gg - rg)) < G_TOL and np.max(np.abs(Gl - rl)) < G_TOL
    assert np.all(Gg[:, 0, 0] == 0) and np.all(Gl[:, 1, 1] == 0)


def test_hubbard_atom_on_gpu():
    U = 2.6
    for nu, nd in ((1, 0), (0, 1), (1, 1)):
        m = W.make_model(1, nu, nd, np.zeros((1, 1)), np.full((2, 1), -U / 2), np.array([U]))
        Gg, Gl = kg.Sector(m).green_equilibrium([(0, 0), (0, 1)], 0.25, 8)
        rg, rl, _ = oracle.green_equilibrium(m, [(0, 0), (0, 1)], 0.25, 8)
        assert np.max(np.abs(Gg - rg)) < 1e-13 and np.max(np.abs(Gl - rl)) < 1e-13


# ------------------------------------------------ batched instances
def batch_models():
    """Star SIAM instances of different sizes and fillings (c4-like) plus edge
    cases: a full up band (no particle part) and a one-site sector."""
    rng = np.random.default_rng(77)
    out = []
    for L in (6, 7, 8, 9, 5, 10):
        nu, nd = int(rng.integers(1, L)), int(rng.integers(1, L))
        U = float(rng.uniform(1, 8))
        out.append(W.siam_star(-U / 2, U, rng.uniform(-3, 3, L - 1), rng.uniform(0.2, 1.0, L - 1), nu, nd))
    out.append(W.siam_star(-1.0, 2.0, [0.5, -0.5], [0.4, 0.6], 3, 1))     # N_up = L
    out.append(W.make_model(1, 1, 0, np.zeros((1, 1)), [[-0.3], [0.2]], [1.5]))  # d = 1
    return out


def test_batched_equilibrium_parity():
    models = batch_models()
    secs = [kg.Sector(m) for m in models]
    orbs = [(0, 0), (0, 1)]
    dt, n = 0.05, 60
    Gg, Gl, status = kg.kg_green_equilibrium_batched([s.handle for s in secs], orbs, dt, n)
    assert np.all(status == 0), status
    for i, m in enumerate(models):
        rg, rl, _ = oracle.green_equilibrium(m, orbs, dt, n)
        assert np.max(np.abs(Gg[i] - rg)) < G_TOL, i
        assert np.max(np.abs(Gl[i] - rl)) < G_TOL, i
        # the plain per-instance path gives the same numbers
        pg, pl = kg.Sector(m).green_equilibrium(orbs, dt, n)
        assert np.max(np.abs(Gg[i] - pg)) < 1e-12 and np.max(np.abs(Gl[i] - pl)) < 1e-12, i
    assert np.all(Gg[6, :, 0, 0] == 0)  # full up band: no particle part


def _c4_dims(m):
    L, nu, nd = m["L"], m["n_up"], m["n_dn"]
    dims = [math.comb(L, nu) * math.comb(L, nd)]
    if nu < L:
        dims.append(math.comb(L, nu + 1) * math.comb(L, nd))
    if nu > 0:
        dims.append(math.comb(L, nu - 1) * math.comb(L, nd))
    return dims


def test_batched_c4_full_size():
    """The whole batched workload: 256 star instances (L 6..12, random
    fillings, d from 36 to 853,776) for all 400 steps (dt = 0.05, M = 20) in
    one batched call.  The 148 instances whose sector and neighbours have at
    most 5,000 states are compared with the oracle's dense Lehmann route (on
    the host cores while the GPU works); the larger ones with the
    per-instance GPU path (the 12 largest and every 8th of the rest).  An
    instance the batch reports degenerate must be degenerate for the oracle."""
    from concurrent.futures import ThreadPoolExecutor
    cfg = W.config_c4()
    models, orbs, dt, n = cfg["models"], cfg["orbitals"], cfg["dt"], cfg["n_steps"]
    small = [i for i, m in enumerate(models) if max(_c4_dims(m)) <= 5000]
    assert len(small) == 148

    def oracle_side():
        return {i: oracle.green_equilibrium_dense(models[i], orbs, dt, n) for i in small}

    with ThreadPoolExecutor(1) as ex:
        fut = ex.submit(oracle_side)
        secs = [kg.Sector(m) for m in models]
        opts = kg.kg_opts_default(M=cfg["M"])
        Gg, Gl, status = kg.kg_green_equilibrium_batched([s.handle for s in secs], orbs, dt, n, opts)
        assert set(np.unique(status)) <= {kg.KG_OK, kg.KG_EDEGEN}, np.unique(status)
        large = sorted((i for i in range(len(models)) if i not in small), key=lambda i: -_c4_dims(models[i])[0])
        plain = large[:12] + large[12::8]
        for i in plain:
            if status[i] != kg.KG_OK:
                continue
            pg, pl = kg.Sector(models[i]).green_equilibrium(orbs, dt, n, opts)
            assert np.max(np.abs(Gg[i] - pg)) < 1e-12 and np.max(np.abs(Gl[i] - pl)) < 1e-12, i
        ref = fut.result()
    checked = 0
    for i in small:
        rg, rl, E0, gap = ref[i]
        if status[i] == kg.KG_EDEGEN:
            assert gap < 1e-6 * max(1.0, abs(E0)), (i, gap)
            continue
        if gap < 1e-8 * max(1.0, abs(E0)):
            continue  # degenerate for the oracle: G is not unique
        assert np.max(np.abs(Gg[i] - rg)) < G_TOL and np.max(np.abs(Gl[i] - rl)) < G_TOL, i
        checked += 1
    assert checked >= 140


# ------------------------------------------------------------- Keldysh G
def keldysh_case():
    ini = W.siam_chain(6, 2.0, 3, 3, field=0.3)
    fin = W.siam_chain(6, 2.0, 3, 3, field=0.0)
    orbs = [(i, 0) for i in range(6)] + [(i, 1) for i in range(6)]
    return ini, fin, orbs


def test_keldysh_parity_and_staged_api():
    ini, fin, orbs = keldysh_case()
    dt, nt = 0.1, 10
    si, sf = kg.Sector(ini), kg.Sector(fin)
    Gl, Gg = kg.kg_green_keldysh(si.handle, sf.handle, orbs, dt, nt)
    rl, rg, _ = oracle.green_keldysh(ini, fin, orbs, dt, nt)
    assert np.max(np.abs(Gl - rl)) < G_TOL
    assert np.max(np.abs(Gg - rg)) < G_TOL
    # staged: rows (in any order), then the Gram, equal the one-shot call
    K = kg.Keldysh(si, sf, orbs, dt, nt)
    for k in reversed(range(nt)):
        dl, dg = K.row(k)
        assert np.max(np.abs(dl - rl[k, k])) < G_TOL and np.max(np.abs(dg - rg[k, k])) < G_TOL
    Sl, Sg = K.gram()
    assert np.max(np.abs(Sl - Gl)) < 1e-12 and np.max(np.abs(Sg - Gg)) < 1e-12
    K.close()


def test_keldysh_gram_needs_all_rows():
    ini, fin, orbs = keldysh_case()
    si, sf = kg.Sector(ini), kg.Sector(fin)
    K = kg.Keldysh(si, sf, orbs[:2], 0.1, 4)
    K.row(0)
    with pytest.raises(kg.KGError) as e:
        K.gram()
    assert e.value.code == kg.KG_EINVAL
    K.close()


def test_keldysh_internal_substeps_and_phi_roundtrip():
    ini, fin, orbs = keldysh_case()
    orbs = [(0, 0), (3, 0), (0, 1)]
    si, sf = kg.Sector(ini), kg.Sector(fin)
    opts = kg.kg_opts_default(dt_internal=0.1)
    Gl, Gg = kg.kg_green_keldysh(si.handle, sf.handle, orbs, 0.3, 5, opts)
    rl, rg, _ = oracle.green_keldysh(ini, fin, orbs, 0.3, 5)
    assert np.max(np.abs(Gl - rl)) < G_TOL and np.max(np.abs(Gg - rg)) < G_TOL
    K = kg.Keldysh(si, sf, orbs, 0.3, 5, opts)
    phi = K.get_phi(4)
    K.set_phi(4, phi)
    dl, dg = K.row(4)
    assert np.max(np.abs(dl - rl[4, 4])) < G_TOL and np.max(np.abs(dg - rg[4, 4])) < G_TOL
    K.close()


@pytest.mark.parametrize("budget_mb,expect", [(0, (0, 1, 1)), (300, (0, 1, 1)), (120, (0, 1, 0)),
                                               (60, (None, 0, 0))])
def test_keldysh_memory_plans(budget_mb, expect):
    """The Keldysh memory plan under device budgets from ample to tight
    (chain of 10 sites, (5,5), d = 63,504; four blocks of two columns, 8
    times): everything resident; columns kept with workspaces re-made per
    row; columns kept without the Gram-Schmidt planes; Phi(t_k) in host
    memory with rows that keep no columns.  Every plan gives the oracle's
    grid through kg_green_keldysh, and its rows (and Gram, when the columns
    are kept) through the staged API."""
    ini = W.siam_chain(10, 2.0, 5, 5, field=0.4)
    fin = W.siam_chain(10, 2.0, 5, 5, field=0.0)
    orbs = [(0, 0), (1, 0), (0, 1), (1, 1)]
    dt, nt = 0.1, 8
    rl, rg, _ = oracle.green_keldysh(ini, fin, orbs, dt, nt)
    si, sf = kg.Sector(ini), kg.Sector(fin)
    opts = kg.kg_opts_default(mem_budget_mb=budget_mb)
    K = kg.Keldysh(si, sf, orbs, dt, nt, opts)
    plan = K.plan()
    got = (plan["phi_on_host"], plan["stores_kept"], plan["planes"])
    if expect[0] is None:
        assert got[0] in (1, 2) and got[1:] == expect[1:], plan
    else:
        assert got == expect, plan
    for k in range(nt):
        dl, dg = K.row(k)
        assert np.max(np.abs(dl - rl[k, k])) < G_TOL and np.max(np.abs(dg - rg[k, k])) < G_TOL, k
    if plan["stores_kept"]:
        Sl, Sg = K.gram()
        assert np.max(np.abs(Sl - rl)) < G_TOL and np.max(np.abs(Sg - rg)) < G_TOL
    else:
        with pytest.raises(kg.KGError) as e:
            K.gram()
        assert e.value.code == kg.KG_EINVAL
    # Phi round trip through the plan's storage
    phi = K.get_phi(5)
    K.set_phi(5, phi)
    assert np.array_equal(K.get_phi(5), phi)
    K.close()
    Gl, Gg = kg.kg_green_keldysh(si.handle, sf.handle, orbs, dt, nt, opts)
    assert np.max(np.abs(Gl - rl)) < G_TOL and np.max(np.abs(Gg - rg)) < G_TOL


def test_keldysh_mismatched_sectors():
    a = kg.Sector(W.hubbard_ring(4, 1.0, 2, 2))
    b = kg.Sector(W.hubbard_ring(4, 1.0, 2, 1))
    with pytest.raises(kg.KGError) as e:
        kg.kg_green_keldysh(a.handle, b.handle, [(0, 0)], 0.1, 3)
    assert e.value.code == kg.KG_EINVAL


# ------------------------------------------------ full-size c2, whole grid
C2_SAMPLES = ([(k, k, 0, b) for k in (0, 3, 40, 99) for b in (0, 5)]
              + [(99, 0, 0, 0), (99, 0, 0, 5), (60, 20, 0, 0), (60, 20, 0, 5), (20, 60, 5, 0)])


@pytest.fixture(scope="module")
def c2_grid():
    """The Hubbard-ring quench at its full size (d = 853,776; columns in the
    N-1 / N+1 sectors, d = 731,808), in the launch configuration of the
    benchmark: every row of step (iii) through the staged API (the call the
    benchmark times), then the step-(iv) Gram of 1,200 vectors per part.  The
    oracle's ground state and sampled entries are computed on the host cores
    meanwhile (the library calls release the interpreter)."""
    from concurrent.futures import ThreadPoolExecutor
    cfg = W.config_c2()
    orbs = cfg["orbitals"]

    def oracle_side():
        e_or, psi_or, _ = oracle.Sector(cfg["ini"]).ground_state()
        samples = [(k, l, orbs[a], orbs[b]) for (k, l, a, b) in C2_SAMPLES]
        return e_or, oracle.keldysh_entries(cfg["ini"], cfg["fin"], samples, cfg["dt"], gs=(e_or, psi_or, 0.0))

    with ThreadPoolExecutor(1) as ex:
        fut = ex.submit(oracle_side)
        si, sf = kg.Sector(cfg["ini"]), kg.Sector(cfg["fin"])
        opts = kg.kg_opts_default(M=cfg["M"])
        E0, _, _ = si.ground_state(opts)
        K = kg.Keldysh(si, sf, orbs, cfg["dt"], cfg["n_t"], opts)
        diag = [K.row(k) for k in range(cfg["n_t"])]
        Gl, Gg = K.gram()
        K.close()
        e_or, entries = fut.result()
    return {"E0": E0, "e_or": e_or, "diag": diag, "Gl": Gl, "Gg": Gg, "entries": entries}


def test_c2_ground_state_full_size(c2_grid):
    assert abs(c2_grid["E0"] - c2_grid["e_or"]) <= E_TOL * abs(c2_grid["e_or"])


def test_c2_rows_at_depth_vs_oracle(c2_grid):
    """Time-diagonal blocks returned by the rows themselves (99 backward
    G-steps per column at k = 99, the benchmarked row) against the oracle."""
    for (k, l, a, b), (les, gtr) in zip(C2_SAMPLES, c2_grid["entries"]):
        if k != l:
            continue
        dl, dg = c2_grid["diag"][k]
        assert abs(dl[a, b] - les) < G_TOL and abs(dg[a, b] - gtr) < G_TOL, (k, a, b)


def test_c2_gram_off_diagonal_vs_oracle(c2_grid):
    """Entries of the full-size step-(iv) Gram off the time diagonal."""
    Gl, Gg = c2_grid["Gl"], c2_grid["Gg"]
    for (k, l, a, b), (les, gtr) in zip(C2_SAMPLES, c2_grid["entries"]):
        assert abs(Gl[k, l, a, b] - les) < G_TOL and abs(Gg[k, l, a, b] - gtr) < G_TOL, (k, l, a, b)
    # the Gram's diagonal blocks are the rows' own blocks
    for k in range(Gl.shape[0]):
        dl, dg = c2_grid["diag"][k]
        assert np.max(np.abs(Gl[k, k] - dl)) < 1e-12 and np.max(np.abs(Gg[k, k] - dg)) < 1e-12, k


def test_c2_whole_grid_invariants(c2_grid):
    """Properties of every entry of the 100 x 100 x 12 x 12 grid: hermiticity
    G(t,t')_{ab}^* = -G(t',t)_{ba}, the sum rule i(G^> - G^<)(t,t) = 1 (and 0
    off the orbital diagonal), half filling n_i(t) = 1/2 from particle-hole
    symmetry, and the ring's translation invariance G_{ab} = G_{a+1,b+1}."""
    Gl, Gg = c2_grid["Gl"], c2_grid["Gg"]
    n = Gl.shape[2]
    for G in (Gl, Gg):
        assert np.max(np.abs(np.conj(G) + G.transpose(1, 0, 3, 2))) < 1e-12
        rolled = np.roll(np.roll(G, 1, axis=2), 1, axis=3)
        assert np.max(np.abs(rolled - G)) < G_TOL
    t = np.arange(Gl.shape[0])
    eq_l, eq_g = Gl[t, t], Gg[t, t]
    assert np.max(np.abs(1j * (eq_g - eq_l) - np.eye(n)[None])) < G_TOL
    occ = (-1j * np.diagonal(eq_l, axis1=1, axis2=2)).real
    assert np.max(np.abs(occ - 0.5)) < G_TOL


# ------------------------------------- Lanczos G(omega), Eq. (gapprox)
@pytest.mark.parametrize("name", ["star_c1", "chain_int", "complex"])
def test_green_lanczos_parity(name):
    """Continued fractions of the GPU Lanczos coefficients against the oracle's
    Ritz-pair sum (Eq. (gapprox)) from its own Lanczos runs.  Past the first
    converged Ritz values the individual coefficients of two correct Lanczos
    runs part at rounding level times a large condition number, and so does
    an unconverged n-pole function; the comparison is therefore made where
    the result is defined to rounding: Krylov spaces that exhaust the sector
    (the resolvent is then exact)."""
    if name == "star_c1":
        m, orbs, n = W.config_c1()["model"], [(0, 0), (2, 1)], 40   # the Krylov space closes at ~13
    elif name == "chain_int":
        # uniform hopping: exact integer hop sums; sectors of 100 and 50 states
        m, orbs, n = W.siam_chain(5, 3.0, 2, 3, field=0.7), [(0, 0), (3, 1)], 120
    else:
        m, orbs, n = W.random_model(5, 2, 2, seed=23, complex_hopping=True), [(1, 0), (4, 1)], 120
    omega = np.linspace(-8.0, 8.0, 41)
    s = kg.Sector(m)
    Gg, Gl, coef = s.green_lanczos(orbs, n, omega, 0.1)
    rg, rl, _ = oracle.green_lanczos(m, orbs, n, omega, 0.1)
    assert np.max(np.abs(Gg - rg)) < G_TOL and np.max(np.abs(Gl - rl)) < G_TOL
    # spectral sum rule: b_0^2 of both parts add up to <{c, c^dag}> = 1
    assert np.max(np.abs(coef[:, 0, n] ** 2 + coef[:, 1, n] ** 2 - 1.0)) < 1e-12


def test_green_lanczos_first_coefficients_full_size_chain():
    """On a large sector (d = 15,876) the first Lanczos coefficients, before
    any Ritz value converges, agree with the oracle's to rounding."""
    m = W.siam_chain(9, 3.0, 4, 5, field=0.7)
    s = kg.Sector(m)
    _, _, coef = s.green_lanczos([(0, 0)], 8, np.zeros(1), 0.1)
    sec = oracle.Sector(m)
    _, psi0, _ = sec.ground_state(K=80, tol=1e-13)
    nb = sec.neighbour(0, True)
    a, b, n0 = oracle.lanczos_run(nb, sec.apply_cop(nb, 0, 0, True, psi0), 8)
    assert np.max(np.abs(coef[0, 0, :8] - a)) < 1e-9
    assert abs(coef[0, 0, 8] - n0) < 1e-12 and np.max(np.abs(coef[0, 0, 9:16] - b)) < 1e-9


def test_green_lanczos_edges():
    # full up band: no particle part for spin up; n = 1 is a single pole
    m = W.make_model(3, 3, 1, W.chain_hopping(3), None, [2.0, 1.0, 0.5])
    s = kg.Sector(m)
    omega = np.linspace(-3, 3, 7)
    Gg, Gl, coef = s.green_lanczos([(0, 0), (1, 1)], 1, omega, 0.2)
    rg, rl, _ = oracle.green_lanczos(m, [(0, 0), (1, 1)], 1, omega, 0.2)
    assert np.all(Gg[0] == 0) and np.max(np.abs(Gl - rl)) < G_TOL and np.max(np.abs(Gg - rg)) < G_TOL
    with pytest.raises(kg.KGError):
        s.green_lanczos([(0, 0)], 256, omega, 0.1)


# --------------------------- fine output grid, Eq. (udelta) at several times
def test_fine_grid_one_is_the_plain_path():
    m = W.random_model(6, 3, 2, seed=21, complex_hopping=True)
    orbs = [(0, 0), (2, 0), (1, 1)]
    s = kg.Sector(m)
    Gg, Gl = s.green_equilibrium(orbs, 0.1, 20)
    Fg, Fl = s.green_equilibrium_fine(orbs, 0.1, 20, 1)
    assert np.max(np.abs(Fg - Gg)) < 1e-12 and np.max(np.abs(Fl - Gl)) < 1e-12


@pytest.mark.parametrize("fine,n", [(4, 40), (5, 37)])
def test_fine_grid_vs_oracle(fine, n):
    """Several output times per Krylov space (step fine*dt, M = 40), including
    a last space that serves fewer times; against the oracle's G(t)."""
    cfg = W.config_c1()
    s = kg.Sector(cfg["model"])
    orbs = [(0, 0), (1, 1)]
    opts = kg.kg_opts_default(M=40)
    Gg, Gl = s.green_equilibrium_fine(orbs, 0.05, n, fine, opts)
    rg, rl, _ = oracle.green_equilibrium(cfg["model"], orbs, 0.05, n)
    assert np.max(np.abs(Gg - rg)) < G_TOL and np.max(np.abs(Gl - rl)) < G_TOL
    with pytest.raises(kg.KGError):
        s.green_equilibrium_fine(orbs, 0.05, n, 33, opts)
