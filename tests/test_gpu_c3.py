"""The 16-site chain of the local-magnetic-excitation quench at full size
(sector (7,7), d = 130,873,600, 2.1 GB per vector): the GPU ground state of
H_ini checked with the oracle's own H*psi of it -- the Rayleigh quotient must
equal the GPU's E0 and the residual must meet the requested tolerance.  The
oracle cannot run a Lanczos or a propagation at this size in test time, but
one H*psi (and its basis) it can."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1109_1205_gb300 as kg  # noqa: E402


def test_c3_ground_state_full_size():
    cfg = W.config_c3()
    s = kg.Sector(cfg["ini"])
    assert s.dim == 130_873_600
    tol = 1e-10
    E0, res, gap = s.ground_state(kg.kg_opts_default(M_gs=40, tol_resid=tol, max_restarts=400))
    assert res <= tol * max(1.0, abs(E0))
    psi = s.ground_state_vector()
    del s
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-10  # FP64 sums over 1.3e8 components
    o = oracle.Sector(cfg["ini"])
    assert o.dim == psi.size
    hpsi = o.hpsi(psi)
    rq = float(np.vdot(psi, hpsi).real)
    assert abs(rq - E0) <= 1e-12 * abs(E0)
    r = float(np.linalg.norm(hpsi - E0 * psi))
    assert r <= 2 * tol * max(1.0, abs(E0)), (r, E0)
