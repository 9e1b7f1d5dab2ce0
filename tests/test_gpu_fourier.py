"""GPU parity of the damped Fourier transform G(t) -> G(omega) (Section 3,
the time-dependent Lanczos route to the spectral function) against the
oracle's transform, on random series and on the equilibrium G(t) of the
star SIAM.

Tolerance: the transform is linear, so a difference of the inputs or of the
rounding order bounds the difference of the outputs by sum_k w_k e^{-eta t_k}
|dG(t_k)|; the tests use 1e-12 times sum_k w_k |G(t_k)| for identical inputs
and the G(t) parity bar (1e-10) times sum_k w_k e^{-eta t_k} for the chain.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1109_1205_gb300 as kg  # noqa: E402


def weight_scale(G, dt):
    w = np.full(G.shape[-1], dt)
    w[0] = w[-1] = 0.5 * dt
    return np.abs(G) @ w


def random_series(rng, n_series, n_t, dt):
    """Damped sums of a few exponentials plus noise: G(t)-like series."""
    t = dt * np.arange(n_t)
    E = rng.uniform(-8.0, 8.0, size=(n_series, 6))
    A = rng.normal(size=(n_series, 6)) + 1j * rng.normal(size=(n_series, 6))
    G = np.einsum("sm,smk->sk", A, np.exp(-1j * E[:, :, None] * t[None, None, :]))
    return G + 0.1 * (rng.normal(size=G.shape) + 1j * rng.normal(size=G.shape))


@pytest.mark.parametrize("eta", [0.0, 0.15])
def test_fourier_parity_random(eta):
    # 1500 samples: two full tiles of 512 and a ragged one (476 = 3 chunks of
    # 128 + 92); 300 frequencies: two blocks of 128 and a ragged 44; the
    # series split over several blocks, summed by the second kernel.
    rng = np.random.default_rng(71)
    dt = 0.05
    G = random_series(rng, 3, 1500, dt)
    omega = np.linspace(-12.0, 12.0, 300)
    F = kg.kg_green_fourier(G, dt, omega, eta)
    R = oracle.green_fourier(G, dt, omega, eta)
    tol = 1e-12 * weight_scale(G, dt)
    assert np.all(np.max(np.abs(F - R), axis=1) <= tol)


def test_fourier_parity_long_series_fine_grid():
    # the sampling of the paper's Fig. 1 calculation: dt' = 0.01 up to
    # t_max = 1000 (100,001 samples), eta = 0.01; 129 frequencies
    rng = np.random.default_rng(72)
    dt, n_t, eta = 0.01, 100001, 0.01
    G = random_series(rng, 1, n_t, dt)
    omega = np.linspace(-10.0, 10.0, 129)
    F = kg.kg_green_fourier(G, dt, omega, eta)
    R = oracle.green_fourier(G, dt, omega, eta)
    assert np.max(np.abs(F - R)) <= 1e-12 * weight_scale(G, dt)[0]


def test_fourier_small_cases():
    rng = np.random.default_rng(73)
    omega = np.array([-1.5, 0.0, 0.25, 3.0])
    for n_t in (2, 3, 127, 128, 129, 511, 512, 513):
        G = random_series(rng, 2, n_t, 0.1)
        for eta in (0.0, 0.4):
            F = kg.kg_green_fourier(G, 0.1, omega, eta)
            R = oracle.green_fourier(G, 0.1, omega, eta)
            assert np.all(np.max(np.abs(F - R), axis=1) <= 1e-12 * weight_scale(G, 0.1)), (n_t, eta)
    # two samples: (dt/2) (g_0 + e^{i (omega + i eta) dt} g_1)
    g = np.array([1.0 + 0.5j, -0.25 + 2.0j])
    F = kg.kg_green_fourier(g, 0.2, omega, 0.3)
    ref = 0.1 * (g[0] + np.exp(1j * (omega + 0.3j) * 0.2) * g[1])
    assert np.max(np.abs(F - ref)) < 1e-15
    # a single sample (an empty interval) and no frequencies: no launch
    assert np.all(kg.kg_green_fourier(np.ones((3, 1)), 0.1, omega, 0.1) == 0)
    assert kg.kg_green_fourier(np.ones((3, 10)), 0.1, [], 0.1).shape == (3, 0)


def test_fourier_of_equilibrium_G_matches_oracle_chain():
    """G(t) of the star SIAM (c1 model, d = 400) from the GPU path, transformed
    on the GPU, against the oracle's G(t) transformed by the oracle; the
    spectral function is non-negative (the transform of a positive Lehmann
    sum under the trapezoidal rule)."""
    cfg = W.config_c1()
    s = kg.Sector(cfg["model"])
    dt, n_steps, eta = 0.05, 800, 0.5  # t_max = 40, e^{-20}
    omega = np.linspace(-6.0, 6.0, 241)
    Fg, Fl = s.spectrum_td([(0, 0), (2, 1)], dt, n_steps, omega, eta)
    Gg, Gl, _ = oracle.green_equilibrium(cfg["model"], [(0, 0), (2, 1)], dt, n_steps)
    bound = 1e-10 * np.sum(0.05 * np.exp(-eta * dt * np.arange(n_steps + 1)))
    for a in range(2):
        Rg = oracle.green_fourier(Gg[:, a, a], dt, omega, eta)
        Rl = oracle.green_fourier(-Gl[:, a, a], dt, omega, eta)
        assert np.max(np.abs(Fg[a] - Rg)) < 2 * bound and np.max(np.abs(Fl[a] - Rl)) < 2 * bound
        A = -(Fg[a] + Fl[a]).imag / np.pi
        assert np.min(A) > -1e-7  # e^{-eta t_max} truncation only
    s.close()


# ------------------------- time-dependent Lanczos with restarts (Fig. 1)
@pytest.mark.parametrize("f,q", [(1, 50), (5, 10)])
def test_restarted_exhausted_space_is_exact(f, q):
    """A Krylov space as large as the sector makes every interval exact: the
    restarted G(t) equals the oracle's for one space or several."""
    m = W.random_model(5, 2, 2, seed=37, complex_hopping=True)
    orbs = [(0, 0), (3, 0), (1, 1)]
    s = kg.Sector(m)
    Gg, Gl = s.green_restarted(orbs, 120, f, q, 0.1)
    rg, rl, _ = oracle.green_equilibrium(m, orbs, 0.1, f * q)
    assert np.max(np.abs(Gg - rg)) < 1e-10 and np.max(np.abs(Gl - rl)) < 1e-10


def test_restarted_short_intervals_vs_oracle():
    """Intervals short enough for n = 30 (Delta t = 0.5 on the L = 8 ring,
    output every 0.05): the restarted G(t) equals the oracle's to 1e-10."""
    m = W.hubbard_ring(8, 4.0, 4, 4)
    orbs = [(0, 0), (3, 0)]
    s = kg.Sector(m)
    Gg, Gl = s.green_restarted(orbs, 30, 8, 10, 0.05)
    rg, rl, _ = oracle.green_equilibrium(m, orbs, 0.05, 80)
    assert np.max(np.abs(Gg - rg)) < 1e-10 and np.max(np.abs(Gl - rl)) < 1e-10


def test_restarted_single_space_is_the_lanczos_pole_sum():
    """f = 1 (Eq. (res)): one Krylov space of n = 40 for the whole interval is
    the n-pole conventional Lanczos function in time, built from the same
    Lanczos coefficients that kg_green_lanczos returns."""
    m = W.hubbard_ring(10, 8.0, 5, 5)
    s = kg.Sector(m)
    n, dt, q = 40, 0.05, 400
    Gg, Gl = s.green_restarted([(0, 0)], n, 1, q, dt)
    _, _, coef = s.green_lanczos([(0, 0)], n, np.zeros(1), 0.1)
    E0, _, _ = s.ground_state()
    t = dt * np.arange(q + 1)
    for kind, G, sgn in ((0, Gg, 1.0), (1, Gl, -1.0)):
        a, b = coef[0, kind, :n], coef[0, kind, n:]
        mm = int(np.count_nonzero(a)) if np.any(a) else 0
        T = np.diag(a[:mm]) + np.diag(b[1:mm], 1) + np.diag(b[1:mm], -1)
        th, Z = np.linalg.eigh(T)
        w = (b[0] * Z[0]) ** 2
        # G^>(t) = -i sum w e^{-i(th - E0) t}; G^<(t) = +i sum w e^{+i(th - E0) t}
        ref = (-1j if sgn > 0 else 1j) * np.exp(-1j * sgn * np.outer(t, th - E0)) @ w
        assert np.max(np.abs(G[:, 0, 0] - ref)) < 1e-10


def test_fig1_restart_comparison():
    """Section 3, Fig. 1 on its own model (L = 10 ring, U = 8, half filling,
    n = 100, t_max = 1000, dt' = 0.01, eta = 0.01): the converged spectrum
    (f = 1000) and the conventional-Lanczos one (f = 1) are non-negative, the
    f = 100 spectrum has negative weight, and both approximations deviate
    from the converged one by a comparable amount."""
    import bench
    r = bench.fig1_restarts()
    f1, f100, f1000 = r["f=1"], r["f=100"], r["f=1000"]
    assert f1000["min_A"] > -1e-4 and f1["min_A"] > -1e-4
    assert f100["min_A"] < -1e-2 and f100["negative_weight"] > 1e-3
    assert 0.01 < f1["l1_to_f1000"] < 1.0 and 0.01 < f100["l1_to_f1000"] < 1.0
