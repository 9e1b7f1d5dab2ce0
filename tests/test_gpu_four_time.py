"""GPU parity of the four-time correlation functions (the higher-order
Green's functions of the outlook in Section 6):
G(t1, t2, t3, t4) = <0|A1(t1) A2(t2) A3(t3) A4(t4)|0> after the quench.

* The CUDA path against the oracle on every one of the 5^4 time combinations
  at 1e-10, for operator sets of both spins and both orderings, with internal
  sub-steps; and in equilibrium (H_ini = H_fin) on a complex-hopping model.
* Operators that change the particle numbers give zero; bad arguments are
  KG_EINVAL.
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
OPS = [[(0, 0, 0), (2, 1, 0), (1, 1, 1), (0, 0, 1)],
       [(1, 0, 1), (1, 0, 0), (0, 1, 1), (4, 1, 0)],
       [(0, 0, 1), (3, 0, 0), (5, 0, 1), (0, 0, 0)]]


@pytest.mark.parametrize("ops", OPS, ids=["cc_cdcd", "cdc_cdc", "one_spin"])
def test_four_time_quench_parity(ops):
    ini = W.siam_chain(6, 2.0, 3, 3, field=0.3)
    fin = W.siam_chain(6, 2.0, 3, 3, field=0.0)
    dt, nt = 0.2, 5
    ref = oracle.green_four_time(ini, fin, ops, dt, nt)
    si, sf = kg.Sector(ini), kg.Sector(fin)
    G = kg.kg_green_four_time(si.handle, sf.handle, ops, dt, nt, kg.kg_opts_default(dt_internal=0.1))
    assert np.max(np.abs(ref)) > 1e-2
    assert np.max(np.abs(G - ref)) < G_TOL


def test_four_time_equilibrium_complex_hopping():
    m = W.random_model(5, 2, 3, seed=17, complex_hopping=True)
    ops = [(1, 1, 0), (4, 0, 1), (2, 0, 0), (3, 1, 1)]
    dt, nt = 0.15, 4
    ref = oracle.green_four_time(m, m, ops, dt, nt)
    s = kg.Sector(m)
    G = kg.kg_green_four_time(s.handle, s.handle, ops, dt, nt)
    assert np.max(np.abs(ref)) > 1e-3
    assert np.max(np.abs(G - ref)) < G_TOL


def test_four_time_zero_and_bad_arguments():
    ini = W.siam_chain(4, 2.0, 2, 2, field=0.3)
    fin = W.siam_chain(4, 2.0, 2, 2, field=0.0)
    si, sf = kg.Sector(ini), kg.Sector(fin)
    G = kg.kg_green_four_time(si.handle, sf.handle, [(0, 0, 0), (1, 0, 0), (2, 0, 0), (0, 0, 1)], 0.1, 3)
    assert G.shape == (3, 3, 3, 3) and np.all(G == 0)
    for ops, nt in (([(4, 0, 0), (1, 0, 0), (2, 0, 1), (0, 0, 1)], 3),
                    ([(0, 2, 0), (1, 0, 0), (2, 0, 1), (0, 0, 1)], 3),
                    ([(0, 0, 0), (1, 0, 0), (2, 0, 1), (0, 0, 1)], 0)):
        with pytest.raises(kg.KGError) as e:
            kg.kg_green_four_time(si.handle, sf.handle, ops, 0.1, nt)
        assert e.value.code == kg.KG_EINVAL
