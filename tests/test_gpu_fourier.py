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
