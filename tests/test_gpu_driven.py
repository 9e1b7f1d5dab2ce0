"""GPU parity of the driven Keldysh Green's function (a Hamiltonian with a
general time dependence after the quench, propagated by the fourth-order
commutator-free exponential steps the outlook of Section 6 proposes).

* The CUDA path against the oracle's CF4 route (each exponential a Chebyshev
  expansion) on the same drive samples: 1e-10, both Keldysh components, with
  internal sub-steps, in the one-shot call and the staged API.
* Constant offsets: the driven call equals the quench of Section 4 with the
  offsets added to H_fin (one Krylov step of h versus two of h/2).
* The Keldysh memory plan with the drive: Phi in host memory, rows keeping
  no columns, still the oracle's values.
* Bad drives are KG_EINVAL.
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

G_TOL = 1e-10


def driven_case(L=6, nu=3, nd=3):
    ini = W.siam_chain(L, 2.0, nu, nd, field=0.3)
    fin = W.siam_chain(L, 2.0, nu, nd, field=0.0)
    return ini, fin


def test_driven_keldysh_parity_one_shot_and_staged():
    ini, fin = driven_case()
    orbs = [(0, 0), (2, 0), (0, 1), (5, 1)]
    dt, nt, n_sub = 0.2, 6, 4
    dp = W.drive_samples(W.periodic_drive(6), dt, nt, n_sub, oracle.CF4_C)
    rl, rg, _ = oracle.green_keldysh_td(ini, fin, orbs, dt, nt, dp, n_sub=n_sub)
    si, sf = kg.Sector(ini), kg.Sector(fin)
    opts = kg.kg_opts_default(dt_internal=dt / n_sub)
    Gl, Gg = kg.kg_green_keldysh_td(si.handle, sf.handle, orbs, dt, nt, dp, opts)
    assert np.max(np.abs(Gl - rl)) < G_TOL and np.max(np.abs(Gg - rg)) < G_TOL
    # the drive matters: the undriven quench differs at order one
    ql, qg = kg.kg_green_keldysh(si.handle, sf.handle, orbs, dt, nt, opts)
    assert np.max(np.abs(ql - Gl)) > 1e-3
    K = kg.Keldysh(si, sf, orbs, dt, nt, opts, dparams=dp)
    for k in reversed(range(nt)):
        dl, dg = K.row(k)
        assert np.max(np.abs(dl - rl[k, k])) < G_TOL and np.max(np.abs(dg - rg[k, k])) < G_TOL
    Sl, Sg = K.gram()
    assert np.max(np.abs(Sl - Gl)) < 1e-12 and np.max(np.abs(Sg - Gg)) < 1e-12
    K.close()


def test_driven_constant_offsets_equal_shifted_quench():
    ini, fin = driven_case()
    orbs = [(0, 0), (1, 1)]
    dt, nt, n_sub = 0.25, 5, 2
    p0 = W.periodic_drive(6)(0.41)
    dp = np.tile(p0, ((nt - 1) * n_sub, 2, 1))
    si, sf = kg.Sector(ini), kg.Sector(fin)
    sf2 = kg.Sector(oracle._shifted(fin, p0))
    opts = kg.kg_opts_default(dt_internal=dt / n_sub)
    Gl, Gg = kg.kg_green_keldysh_td(si.handle, sf.handle, orbs, dt, nt, dp, opts)
    Ql, Qg = kg.kg_green_keldysh(si.handle, sf2.handle, orbs, dt, nt, opts)
    assert np.max(np.abs(Gl - Ql)) < 1e-11 and np.max(np.abs(Gg - Qg)) < 1e-11
    # sum rule at every time
    for k in range(nt):
        assert np.max(np.abs(1j * (np.diagonal(Gg[k, k]) - np.diagonal(Gl[k, k])) - 1.0)) < 1e-11


def test_driven_memory_plan_host_phi():
    """Chain of 8 sites, (4,4), d = 4,900: with a 1 MB budget Phi(t_k) lives
    in host memory and rows keep no columns; the driven rows still match the
    oracle, and the one-shot call (one block at a time) gives its grid."""
    ini, fin = driven_case(8, 4, 4)
    orbs = [(0, 0), (0, 1)]
    dt, nt, n_sub = 0.1, 5, 2
    dp = W.drive_samples(W.periodic_drive(8, sites=range(4)), dt, nt, n_sub, oracle.CF4_C)
    rl, rg, _ = oracle.green_keldysh_td(ini, fin, orbs, dt, nt, dp, n_sub=n_sub)
    si, sf = kg.Sector(ini), kg.Sector(fin)
    opts = kg.kg_opts_default(dt_internal=dt / n_sub, mem_budget_mb=1)
    K = kg.Keldysh(si, sf, orbs, dt, nt, opts, dparams=dp)
    plan = K.plan()
    assert plan["phi_on_host"] in (1, 2) and plan["stores_kept"] == 0, plan
    for k in range(nt):
        dl, dg = K.row(k)
        assert np.max(np.abs(dl - rl[k, k])) < G_TOL and np.max(np.abs(dg - rg[k, k])) < G_TOL, k
    K.close()
    Gl, Gg = kg.kg_green_keldysh_td(si.handle, sf.handle, orbs, dt, nt, dp, opts)
    assert np.max(np.abs(Gl - rl)) < G_TOL and np.max(np.abs(Gg - rg)) < G_TOL


def test_driven_bad_inputs():
    ini, fin = driven_case()
    si, sf = kg.Sector(ini), kg.Sector(fin)
    dt, nt = 0.2, 3
    dp = W.drive_samples(W.periodic_drive(6), dt, nt, 1, oracle.CF4_C)
    bad = dp.copy()
    bad[1, 0, 4] = np.nan
    with pytest.raises(kg.KGError) as e:
        kg.kg_green_keldysh_td(si.handle, sf.handle, [(0, 0)], dt, nt, bad)
    assert e.value.code == kg.KG_EINVAL
    with pytest.raises(kg.KGError) as e:
        kg.kg_green_keldysh_td(si.handle, sf.handle, [(0, 0)], dt, nt, None)
    assert e.value.code == kg.KG_EINVAL
    # one time: no step, no drive needed; G(0,0) of the initial state
    Gl, Gg = kg.kg_green_keldysh_td(si.handle, sf.handle, [(0, 0)], dt, 1, None)
    Ql, Qg = kg.kg_green_keldysh(si.handle, sf.handle, [(0, 0)], dt, 1)
    assert np.array_equal(Gl, Ql) and np.array_equal(Gg, Qg)
