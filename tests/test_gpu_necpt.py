"""GPU parity of the nonequilibrium cluster-perturbation theory (Section 5,
Eq. (cpteq)): the cluster components from the library's GPU routines, the
contour matrices and their LU solve on the device, against the oracle's
NE-CPT on the same contour (trapezoidal, beta = 15).

* The 4-site impurity cluster of the paper's application (U = T = V = 1, field
  0.2 switched off at t = 0) coupled to a 100-site bath: every occupation
  n_{i sigma}(t_k) at 1e-10, the bar of the Green's functions (measured:
  1.1e-15).
* V = 0 returns the isolated cluster's occupations of the four-step method.
* Bad arguments are KG_EINVAL.
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

N_TOL = 1e-10


def cluster(L=4, U=1.0, h=0.2):
    ini = W.siam_chain(L, U, L // 2, L // 2, field=h)
    fin = W.siam_chain(L, U, L // 2, L // 2, field=0.0)
    return ini, fin


def test_necpt_parity_with_oracle():
    ini, fin = cluster()
    args = (100, 1.0, 1.0, 0.1, 6, 15.0, 150)
    ref = oracle.necpt_occupations(ini, fin, *args)
    si, sf = kg.Sector(ini), kg.Sector(fin)
    n = kg.kg_necpt_occupations(si, sf, *args)
    assert n.shape == ref.shape == (2, 6, 4)
    assert np.max(np.abs(n - ref)) < N_TOL, np.max(np.abs(n - ref))
    m = n[0] - n[1]
    assert m[0, 0] > 0.2  # the field polarises the impurity at t = 0


def test_necpt_decoupled_is_the_isolated_cluster():
    ini, fin = cluster()
    si, sf = kg.Sector(ini), kg.Sector(fin)
    n = kg.kg_necpt_occupations(si, sf, 50, 1.0, 0.0, 0.1, 5, 15.0, 150)
    orbs = [(i, s) for s in (0, 1) for i in range(4)]
    Gl, _ = kg.kg_green_keldysh(si.handle, sf.handle, orbs, 0.1, 5)
    for k in range(5):
        occ = (-1j * np.diagonal(Gl[k, k])).real
        assert np.max(np.abs(n[0, k] - occ[:4])) < 1e-12 and np.max(np.abs(n[1, k] - occ[4:])) < 1e-12


def test_necpt_bad_arguments():
    ini, fin = cluster()
    si, sf = kg.Sector(ini), kg.Sector(fin)
    for args in ((0, 1.0, 1.0, 0.1, 3, 15.0, 10), (10, 1.0, 1.0, 0.1, 0, 15.0, 10), (10, 1.0, 1.0, 0.1, 3, 0.0, 10),
                 (10, 1.0, 1.0, -0.1, 3, 15.0, 10), (10, 1.0, 1.0, 0.1, 3, 15.0, 1),
                 (10, 1.0, 1.0, 0.1, 3000, 15.0, 100)):
        with pytest.raises(kg.KGError) as e:
            kg.kg_necpt_occupations(si, sf, *args)
        assert e.value.code == kg.KG_EINVAL
