"""The 16-site chain of the local-magnetic-excitation quench at full size
(sector (7,7), d = 130,873,600, 2.1 GB per vector; neighbour sectors of
91.6M and 147.2M states).

* The GPU ground state of H_ini, checked with the oracle's own H*psi of it:
  the Rayleigh quotient must equal the GPU's E0 and the residual must meet
  the requested tolerance.  The oracle cannot run a Lanczos or a propagation
  at this size in test time, but one H*psi (and its basis) it can.
* The nonequilibrium G of Section 4 for the first grid times (t_k = 0.2 k,
  k < 3, internal Krylov step 0.05), every block (both spins, both kinds), in
  two memory plans: Phi(t_k) on the device with the Gram-Schmidt planes, and
  Phi(t_k) in host memory with rows that keep no columns and workspaces
  without planes.  Both must agree to rounding, satisfy the sum rule
  i(G^> - G^<)(t,t) = 1 at every time for both spins, and (first plan) give
  a Hermitian grid whose diagonal blocks are the rows' own.
"""
import time

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1109_1205_gb300 as kg  # noqa: E402

GS_TOL = 1e-10


@pytest.fixture(scope="module")
def c3():
    cfg = W.config_c3()
    si, sf = kg.Sector(cfg["ini"]), kg.Sector(cfg["fin"])
    assert si.dim == 130_873_600
    E0, res, gap = si.ground_state(kg.kg_opts_default(M_gs=40, tol_resid=GS_TOL, max_restarts=400))
    return cfg, si, sf, E0, res


def test_c3_ground_state_full_size(c3):
    cfg, si, _, E0, res = c3
    assert res <= GS_TOL * max(1.0, abs(E0))
    psi = si.ground_state_vector()
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-10  # FP64 sums over 1.3e8 components
    o = oracle.Sector(cfg["ini"])
    assert o.dim == psi.size
    hpsi = o.hpsi(psi)
    rq = float(np.vdot(psi, hpsi).real)
    assert abs(rq - E0) <= 1e-12 * abs(E0)
    r = float(np.linalg.norm(hpsi - E0 * psi))
    assert r <= 2 * GS_TOL * max(1.0, abs(E0)), (r, E0)


def _rows(cfg, si, sf, n_t, budget_mb):
    opts = kg.kg_opts_default(M=cfg["M"], dt_internal=cfg["dt_internal"], mem_budget_mb=budget_mb)
    K = kg.Keldysh(si, sf, cfg["orbitals"], cfg["dt"], n_t, opts)
    plan = K.plan()
    rows, secs = [], []
    for k in range(n_t):
        t0 = time.perf_counter()
        rows.append(K.row(k))
        secs.append(time.perf_counter() - t0)
    return K, plan, rows, secs


def test_c3_keldysh_first_rows_two_memory_plans(c3):
    cfg, si, sf, _, _ = c3
    n_t = 3
    K, plan, rows, secs = _rows(cfg, si, sf, n_t, 0)
    assert plan["phi_on_host"] == 0 and plan["stores_kept"] == 1 and plan["planes"] == 1, plan
    Gl, Gg = K.gram()
    K.close()
    # 60 GB: Phi(t_k) moves to host memory, rows keep no columns, no planes
    K2, plan2, rows2, _ = _rows(cfg, si, sf, n_t, 60000)
    assert plan2["phi_on_host"] in (1, 2) and plan2["stores_kept"] == 0 and plan2["planes"] == 0, plan2
    with pytest.raises(kg.KGError) as e:
        K2.gram()
    assert e.value.code == kg.KG_EINVAL
    K2.close()
    for k in range(n_t):
        (dl, dg), (dl2, dg2) = rows[k], rows2[k]
        assert np.max(np.abs(dl - dl2)) < 1e-12 and np.max(np.abs(dg - dg2)) < 1e-12, k
        # sum rule for both spins of the impurity: i (G^> - G^<)(t,t) = 1
        assert np.max(np.abs(1j * (np.diag(dg) - np.diag(dl)) - 1.0)) < 1e-10, k
        # occupations are probabilities; opposite spins do not mix
        occ = (-1j * np.diag(dl)).real
        assert np.all(occ > 0) and np.all(occ < 1) and dl[0, 1] == 0 and dg[0, 1] == 0
        assert np.max(np.abs(Gl[k, k] - dl)) < 1e-12 and np.max(np.abs(Gg[k, k] - dg)) < 1e-12
    for G in (Gl, Gg):
        assert np.max(np.abs(np.conj(G) + G.transpose(1, 0, 3, 2))) < 1e-12
    # the field of H_ini polarises the impurity at t = 0 (up favoured)
    occ0 = (-1j * np.diag(rows[0][0])).real
    assert occ0[0] > occ0[1]
    # G-steps of the last row: k * (dt / dt_internal) steps for every column
    n_sub = int(round(cfg["dt"] / cfg["dt_internal"]))
    print("c3 row %d: %d G-steps (4 columns, d = 91.6M / 147.2M) in %.2f s"
          % (n_t - 1, 4 * (n_t - 1) * n_sub, secs[-1]))
