"""GPU parity of the zero-temperature Matsubara function (Section 4, after
step (iv)) from the conventional Lanczos runs against the oracle's dense
imaginary-time propagators.  Tolerance 1e-11 relative to max(1, |G|) where
the Krylov space exhausts the sector, 1e-10 where it does not (the
imaginary-time exponential of a 150-step Krylov space of the 300-dimensional
star-SIAM sectors is exact to rounding for tau <= 10)."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1109_1205_gb300 as kg  # noqa: E402


def diag(G):
    return np.stack([G[:, a, a] for a in range(G.shape[1])])


def test_matsubara_exhausted_krylov_space():
    m = W.random_model(5, 2, 2, seed=61, complex_hopping=True)
    orbs = [(0, 0), (3, 0), (2, 1)]
    taus = np.array([0.0, 0.2, 1.0, 3.0, 7.0])
    mu = 0.15
    s = kg.Sector(m)
    Gp, Gm = s.green_matsubara(orbs, 120, mu, taus)
    Rp, Rm, _ = oracle.green_matsubara(m, orbs, taus, mu)
    Rp, Rm = diag(Rp), diag(Rm)
    assert np.max(np.abs(Rp.imag)) < 1e-13 and np.max(np.abs(Rm.imag)) < 1e-13
    scale = np.maximum(1.0, np.maximum(np.abs(Rp.real), np.abs(Rm.real)))
    assert np.max(np.abs(Gp - Rp.real) / scale) < 1e-11 and np.max(np.abs(Gm - Rm.real) / scale) < 1e-11
    # the jump at tau = 0: G^M(0+) - G^M(0-) = -1
    assert np.max(np.abs(Gp[:, 0] - Gm[:, 0] + 1.0)) < 1e-12
    s.close()


def test_matsubara_star_siam():
    cfg = W.config_c1()
    orbs = [(0, 0), (2, 1)]
    taus = np.linspace(0.0, 10.0, 21)
    s = kg.Sector(cfg["model"])
    Gp, Gm = s.green_matsubara(orbs, 150, 0.0, taus)
    Rp, Rm, _ = oracle.green_matsubara(cfg["model"], orbs, taus, 0.0)
    assert np.max(np.abs(Gp - diag(Rp).real)) < 1e-10 and np.max(np.abs(Gm - diag(Rm).real)) < 1e-10
    # particle-hole symmetric impurity: G^M_00(-tau) = -G^M_00(+tau); decaying with tau
    assert np.max(np.abs(Gm[0] + Gp[0])) < 1e-10
    assert np.all(np.diff(-Gp[0]) < 0)
    s.close()


def test_matsubara_edges():
    # full up band: no particle part for spin up
    m = W.make_model(3, 3, 1, W.chain_hopping(3), None, [2.0, 1.0, 0.5])
    s = kg.Sector(m)
    taus = np.array([0.0, 0.5])
    Gp, Gm = s.green_matsubara([(0, 0), (1, 1)], 10, 0.3, taus)
    Rp, Rm, _ = oracle.green_matsubara(m, [(0, 0), (1, 1)], taus, 0.3)
    assert np.all(Gp[0] == 0)
    assert np.max(np.abs(Gp - diag(Rp).real)) < 1e-11 and np.max(np.abs(Gm - diag(Rm).real)) < 1e-11
    assert s.green_matsubara([(0, 0)], 10, 0.0, []) [0].shape == (1, 0)
    for bad in (dict(n=256, tau=taus), dict(n=10, tau=[-0.1]), dict(n=10, tau=[float("nan")])):
        with pytest.raises(kg.KGError):
            s.green_matsubara([(0, 0)], bad["n"], 0.0, bad["tau"])
    with pytest.raises(kg.KGError):
        s.green_matsubara([(0, 0)], 10, float("inf"), taus)
    s.close()


@pytest.mark.parametrize("case", ["random", "star"])
def test_matsubara_steps_full_matrix(case):
    """Every orbital pair of each spin on tau_k = k dtau by imaginary-time
    Krylov steps (M = 20 per step), against the oracle's dense propagators;
    the diagonal also against the Lanczos route."""
    if case == "random":
        m = W.random_model(5, 2, 2, seed=61, complex_hopping=True)
        orbs, mu, dtau, n = [(0, 0), (3, 0), (1, 1), (4, 1)], 0.15, 0.1, 30
    else:
        m = W.config_c1()["model"]
        orbs, mu, dtau, n = [(0, 0), (1, 0), (2, 1)], 0.0, 0.25, 40
    s = kg.Sector(m)
    Gp, Gm = s.green_matsubara_steps(orbs, mu, dtau, n)
    taus = dtau * np.arange(n + 1)
    Rp, Rm, _ = oracle.green_matsubara(m, orbs, taus, mu)
    scale = max(1.0, np.max(np.abs(Rp)), np.max(np.abs(Rm)))
    assert np.max(np.abs(Gp - Rp)) < 1e-10 * scale and np.max(np.abs(Gm - Rm)) < 1e-10 * scale
    # tau = 0: G^M(0+) - G^M(0-) = -delta within each spin
    same = np.array([[o1[1] == o2[1] for o2 in orbs] for o1 in orbs])
    assert np.max(np.abs((Gp[0] - Gm[0])[same] + np.eye(len(orbs))[same])) < 1e-12
    Lp, Lm = s.green_matsubara(orbs, 120, mu, taus)
    assert np.max(np.abs(diag(Gp).real - Lp)) < 1e-10 * scale and np.max(np.abs(diag(Gm).real - Lm)) < 1e-10 * scale
    with pytest.raises(kg.KGError):
        s.green_matsubara_steps(orbs, mu, -0.1, 2)
    s.close()


MIXED_CASES = {
    # an interacting quench with complex hopping, orbitals of both spins
    "interacting": (lambda: (W.random_model(4, 2, 1, seed=91, complex_hopping=True),
                             W.random_model(4, 2, 1, seed=92, complex_hopping=True)),
                    [(0, 0), (2, 0), (1, 1), (3, 1)], 0.1),
    # the field quench of a 6-site SIAM chain (the paper's Section 4 setting)
    "chain-field": (lambda: (W.siam_chain(6, 2.0, 3, 3, field=0.3), W.siam_chain(6, 2.0, 3, 3, field=0.0)),
                    [(0, 0), (1, 0), (0, 1)], 0.0),
}


@pytest.mark.parametrize("name", list(MIXED_CASES))
def test_mixed_components_vs_oracle(name):
    """G^right(t_k, tau_j) and G^left(tau_j, t_k) (Section 4, after step (iv))
    from the stored imaginary-time vectors and Keldysh columns, against the
    oracle's dense imaginary-time propagators and Chebyshev columns."""
    make, orbs, mu = MIXED_CASES[name]
    ini, fin = make()
    dt, nt, dtau, ntau = 0.2, 5, 0.25, 8
    si, sf = kg.Sector(ini), kg.Sector(fin)
    Gr, Gl = kg.kg_green_mixed(si.handle, sf.handle, orbs, dt, nt, mu, dtau, ntau, kg.kg_opts_default(M=20))
    rr, rl, _ = oracle.green_mixed(ini, fin, orbs, dt, nt, dtau * np.arange(ntau + 1), mu)
    assert Gr.shape == rr.shape and Gl.shape == rl.shape
    assert np.max(np.abs(Gr - rr)) < 1e-10 and np.max(np.abs(Gl - rl)) < 1e-10
    # boundary: at t = 0 the real-time columns are c|0>, c^dag|0>, so
    # G^left(tau, 0) = i G^M(tau) and G^right(0, tau) = i G^M(-tau)
    Gp, Gm = si.green_matsubara_steps(orbs, mu, dtau, ntau, kg.kg_opts_default(M=20))
    assert np.max(np.abs(Gl[:, 0] - 1j * Gp)) < 1e-10
    assert np.max(np.abs(Gr[0] - 1j * Gm)) < 1e-10


def test_matsubara_steps_reject_a_too_large_step():
    """A step far beyond what its Krylov dimension resolves (M = 4, dtau = 2
    on a star whose spectrum spans ~10) is refused by the step's error
    estimate instead of returning an inaccurate G^M."""
    cfg = W.config_c1()
    s = kg.Sector(cfg["model"])
    with pytest.raises(kg.KGError) as e:
        s.green_matsubara_steps([(0, 0)], 0.0, 2.0, 3, kg.kg_opts_default(M=4))
    assert e.value.code == kg.KG_ENOCONV and "too large" in kg.kg_last_error()
    Gp, Gm = s.green_matsubara_steps([(0, 0)], 0.0, 0.25, 3, kg.kg_opts_default(M=20))
    Rp, Rm, _ = oracle.green_matsubara(cfg["model"], [(0, 0)], 0.25 * np.arange(4), 0.0)
    assert np.max(np.abs(Gp - Rp)) < 1e-10 and np.max(np.abs(Gm - Rm)) < 1e-10
