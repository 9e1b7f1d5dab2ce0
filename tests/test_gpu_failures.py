"""Failure detection through status codes, with every fault made on the host.

Each case plants its failure in what the host passes in -- a NaN in an input
vector, a ground-state search given too few restarts, a Hamiltonian whose two
lowest levels are split by far less than the degeneracy threshold -- and
checks the status the library returns.  Nothing here faults, traps or stalls
the GPU: a non-finite norm sets a column's status on the device and empties
its Krylov space, so the remaining kernels of the step skip that column, and
the host reads the status back.  After each failure the same handle (or the
process's CUDA context) still computes correct results.
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nan_in_input_vector_is_enumeric(bad):
    m = W.random_model(7, 3, 3, seed=11, complex_hopping=True)
    s = kg.Sector(m)
    x = W.random_state(s.dim, 5)
    x[17] = complex(bad, 0.0)
    xd = dev(x)
    with pytest.raises(kg.KGError) as e:
        s.propagate(xd, 0.05, 3)
    assert e.value.code == kg.KG_ENUMERIC
    # the handle and the context are still good: a clean vector propagates
    x[17] = 0.1
    x /= np.linalg.norm(x)
    xd = dev(x)
    s.propagate(xd, 0.05, 3)
    torch.cuda.synchronize()
    ref = oracle.Sector(m).propagate(x, 0.15)
    assert np.max(np.abs(xd.cpu().numpy() - ref)) < 1e-11


def test_nan_in_keldysh_phi_is_enumeric():
    ini = W.siam_chain(6, 2.0, 3, 3, field=0.3)
    fin = W.siam_chain(6, 2.0, 3, 3, field=0.0)
    si, sf = kg.Sector(ini), kg.Sector(fin)
    K = kg.Keldysh(si, sf, [(0, 0), (1, 1)], 0.1, 4)
    phi = K.get_phi(3)
    good = phi.copy()
    phi[5] = complex(np.nan, np.nan)
    K.set_phi(3, phi)
    with pytest.raises(kg.KGError) as e:
        K.row(3)
    assert e.value.code == kg.KG_ENUMERIC
    K.set_phi(3, good)
    dl, dg = K.row(3)
    rl, rg = oracle.keldysh_entry(ini, fin, (0, 0), (0, 0), 0.1, 3, 3)
    assert abs(dl[0, 0] - rl) < 1e-10 and abs(dg[0, 0] - rg) < 1e-10
    K.close()


def test_too_few_restarts_is_enoconv():
    m = W.config_c1()["model"]
    s = kg.Sector(m)
    with pytest.raises(kg.KGError) as e:
        s.ground_state(kg.kg_opts_default(M_gs=6, max_restarts=1))
    assert e.value.code == kg.KG_ENOCONV
    # the Green's function refuses to run on an unconverged ground state ...
    with pytest.raises(kg.KGError) as e2:
        s.green_equilibrium([(0, 0)], 0.05, 2, kg.kg_opts_default(M_gs=6, max_restarts=1))
    assert e2.value.code == kg.KG_ENOCONV
    # ... and converges with enough restarts
    E0, res, _ = s.ground_state(kg.kg_opts_default(M_gs=40))
    e_or, _, _ = oracle.Sector(m).ground_state()
    assert abs(E0 - e_or) < 1e-12 * abs(e_or)


def test_split_degenerate_ground_state_is_edegen():
    """Two dimers (0,1) and (2,3) joined by a hopping of 1e-10, one up
    electron: the two lowest levels are -1 -/+ 5e-11 (a Ritz gap far below
    the 1e-8 threshold), so the ground state is degenerate for the method."""
    h = np.zeros((4, 4))
    h[0, 1] = h[1, 0] = -1.0
    h[2, 3] = h[3, 2] = -1.0
    h[1, 2] = h[2, 1] = -1e-10
    m = W.make_model(4, 1, 0, h)
    w = np.linalg.eigvalsh(oracle.dense_hamiltonian(oracle.Sector(m)))
    assert 0 < w[1] - w[0] < 1e-9
    s = kg.Sector(m)
    with pytest.raises(kg.KGError) as e:
        s.ground_state()
    assert e.value.code == kg.KG_EDEGEN
    # the batched solver reports it per instance and leaves that G zero
    good = kg.Sector(W.siam_star(-1.0, 2.0, [0.5, -0.5], [0.4, 0.6], 1, 2))
    bad = kg.Sector(m)
    Gg, Gl, status = kg.kg_green_equilibrium_batched([good.handle, bad.handle], [(0, 0)], 0.05, 4)
    assert status[0] == kg.KG_OK and status[1] == kg.KG_EDEGEN
    assert np.all(Gg[1] == 0) and np.all(Gl[1] == 0)
    rg, rl, _ = oracle.green_equilibrium(W.siam_star(-1.0, 2.0, [0.5, -0.5], [0.4, 0.6], 1, 2), [(0, 0)], 0.05, 4)
    assert np.max(np.abs(Gg[0] - rg)) < 1e-10 and np.max(np.abs(Gl[0] - rl)) < 1e-10
