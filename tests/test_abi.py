"""CPU-only checks of the C ABI: the library loads, exports every function
that include/krylovgf.h declares, and rejects bad arguments before touching
the GPU.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "krylovgf.h")


@pytest.fixture(scope="module")
def kg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1109_1205_gb300 as kg
    return kg


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kg_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["kg_build_sector", "kg_ground_state", "kg_green_equilibrium", "kg_green_keldysh",
                     "kg_hpsi", "kg_apply_cop", "kg_propagate"]:
        assert required in names


def test_every_declared_symbol_is_exported(kg):
    lib = ctypes.CDLL(kg.library_path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", kg.library_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (kg_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_declares_every_signature(kg):
    """The ctypes binding gives every declared function its argument types,
    so no pointer or 64-bit size goes through ctypes' default int conversion."""
    from paper_1109_1205_gb300 import _lib
    for name in declared_functions():
        assert name in _lib._sig, name
        assert getattr(kg.lib, name).argtypes is not None, name


def test_options_and_status_strings(kg):
    o = kg.kg_opts_default()
    assert (o.M, o.M_gs, o.reorth, o.use_graphs, o.seed, o.mem_budget_mb) == (20, 100, 1, 1, 1234, 0)
    assert o.tol_resid == 1e-12 and o.stream is None
    for code in range(0, -9, -1):
        assert kg.kg_strerror(code) != "unknown status"
    assert kg.kg_strerror(-42) == "unknown status"


def test_argument_validation_before_device_use(kg):
    lib = kg.lib
    out = ctypes.c_void_p()
    z = np.zeros(64)
    # bad sizes
    for L, nu, nd in [(0, 0, 0), (33, 1, 1), (4, 5, 1), (4, 1, -1)]:
        rc = lib.kg_build_sector(L, nu, nd, z.ctypes.data, None, z.ctypes.data, z.ctypes.data, ctypes.byref(out))
        assert rc == kg.KG_EINVAL
    # non-Hermitian hopping
    h = np.array([[0.0, 1.0], [2.0, 0.0]])
    rc = lib.kg_build_sector(2, 1, 1, h.ctypes.data, None, z.ctypes.data, z.ctypes.data, ctypes.byref(out))
    assert rc == kg.KG_EINVAL and "Hermitian" in kg.kg_last_error()
    # complex hopping must be anti-symmetric in its imaginary part
    hi = np.array([[0.0, 0.5], [0.5, 0.0]])
    hr = np.array([[0.0, 1.0], [1.0, 0.0]])
    rc = lib.kg_build_sector(2, 1, 1, hr.ctypes.data, hi.ctypes.data, z.ctypes.data, z.ctypes.data, ctypes.byref(out))
    assert rc == kg.KG_EINVAL
    # non-finite parameters (a NaN also passes a Hermiticity comparison, so it
    # is rejected on its own)
    for bad_h, bad_e, bad_u in [(np.nan, 0.0, 0.0), (np.inf, 0.0, 0.0), (0.0, np.nan, 0.0), (0.0, 0.0, -np.inf)]:
        hh = np.array([[0.0, bad_h], [bad_h, 0.0]])
        ee = np.full(4, bad_e)
        uu = np.full(2, bad_u)
        rc = lib.kg_build_sector(2, 1, 1, hh.ctypes.data, None, ee.ctypes.data, uu.ctypes.data, ctypes.byref(out))
        assert rc == kg.KG_EINVAL and "not finite" in kg.kg_last_error()
    hi = np.array([[0.0, np.nan], [-np.nan, 0.0]])
    rc = lib.kg_build_sector(2, 1, 1, hr.ctypes.data, hi.ctypes.data, z.ctypes.data, z.ctypes.data, ctypes.byref(out))
    assert rc == kg.KG_EINVAL
    # dimension beyond 2^31
    big = np.zeros(32 * 32)
    rc = lib.kg_build_sector(32, 16, 16, big.ctypes.data, None, z.ctypes.data, z.ctypes.data, ctypes.byref(out))
    assert rc == kg.KG_ENOMEM
    # NULL handles are rejected, never dereferenced
    assert lib.kg_hpsi(None, None, None, None) == kg.KG_EINVAL
    assert lib.kg_ground_state(None, None, None, None, None) == kg.KG_EINVAL
    assert lib.kg_keldysh_row(None, 0, None, None) == kg.KG_EINVAL
    assert lib.kg_green_lanczos(None, None, 0, 0, None, 0, 0.0, None, None, None, None) == kg.KG_EINVAL


def test_fourier_validation_and_empty_cases(kg):
    """kg_green_fourier rejects bad sizes and non-finite scalars before any
    device call; the empty and single-sample cases need no device either."""
    lib = kg.lib
    g = np.ones(8, dtype=np.complex128)
    w = np.linspace(-1.0, 1.0, 3)
    out = np.zeros(3, dtype=np.complex128)
    for n_series, n_t, dt, eta in [(-1, 4, 0.1, 0.0), (1, 0, 0.1, 0.0), (1, 4, 0.0, 0.0), (1, 4, -0.1, 0.0),
                                   (1, 4, float("nan"), 0.0), (1, 4, 0.1, -1.0), (1, 4, 0.1, float("inf")),
                                   (70000, 4, 0.1, 0.0)]:
        rc = lib.kg_green_fourier(g.ctypes.data, n_series, n_t, dt, w.ctypes.data, 3, eta, None, out.ctypes.data)
        assert rc == kg.KG_EINVAL, (n_series, n_t, dt, eta)
    assert lib.kg_green_fourier(None, 1, 4, 0.1, w.ctypes.data, 3, 0.0, None, out.ctypes.data) == kg.KG_EINVAL
    bad = np.array([0.0, float("nan"), 1.0])
    assert lib.kg_green_fourier(g.ctypes.data, 1, 4, 0.1, bad.ctypes.data, 3, 0.0, None,
                                out.ctypes.data) == kg.KG_EINVAL
    assert "omega[1]" in kg.kg_last_error()
    # nothing to transform, and a single sample (an empty time interval)
    assert kg.kg_green_fourier(np.zeros((2, 5)), 0.1, [], 0.2).shape == (2, 0)
    assert kg.kg_green_fourier(np.zeros((0, 5)), 0.1, w, 0.2).shape == (0, 3)
    z = kg.kg_green_fourier(np.array([[1.0 + 2.0j], [3.0j]]), 0.1, w, 0.2)
    assert z.shape == (2, 3) and np.all(z == 0)
    lib.kg_free_sector(None)
    lib.kg_keldysh_free(None)


def test_every_handle_entry_rejects_null(kg):
    """Each entry point that takes a handle or buffers returns KG_EINVAL for
    NULL before any device call (and the free functions accept NULL)."""
    lib = kg.lib
    o = kg.kg_opts_default()
    ob = ctypes.byref(o)
    buf = np.zeros(64)
    b = buf.ctypes.data
    orb = np.zeros(2, dtype=np.int32)
    ll = ctypes.c_longlong()
    E = kg.KG_EINVAL
    assert lib.kg_sector_dims(None, None, None, None) == E
    assert lib.kg_sector_strings(None, None, None) == E
    assert lib.kg_neighbour_dim(None, 0, 1, ctypes.byref(ll)) == E
    assert lib.kg_apply_cop(None, 0, 0, 1, b, b, None) == E
    assert lib.kg_copy_ground_state(None, b, 1) == E
    assert lib.kg_propagate(None, b, 0.1, 1, ob) == E
    assert lib.kg_green_equilibrium(None, orb.ctypes.data, 1, 0.1, 1, ob, b, b) == E
    assert lib.kg_green_equilibrium_fine(None, orb.ctypes.data, 1, 0.1, 1, 2, ob, b, b) == E
    assert lib.kg_green_equilibrium_batched(None, 0, orb.ctypes.data, 1, 0.1, 1, ob, b, b, None) == E
    nulls = (ctypes.c_void_p * 2)()
    assert lib.kg_green_equilibrium_batched(nulls, 2, orb.ctypes.data, 1, 0.1, 1, ob, b, b, None) == E
    assert "NULL sector" in kg.kg_last_error()
    assert lib.kg_green_equilibrium_vjp(None, orb.ctypes.data, 1, 0.1, 1, ob, 0, None, None, b, b, b, b) == E
    assert lib.kg_green_keldysh(None, None, orb.ctypes.data, 1, 0.1, 1, ob, b, b) == E
    assert lib.kg_keldysh_create(None, None, orb.ctypes.data, 1, 0.1, 1, ob, None) == E
    assert lib.kg_keldysh_gram(None, b, b) == E
    assert lib.kg_keldysh_plan(None, None, None, None, None) == E
    assert lib.kg_green_mixed(None, None, orb.ctypes.data, 1, 0.1, 1, 0.0, 0.1, 1, ob, b, b) == E
    assert lib.kg_green_restarted(None, orb.ctypes.data, 1, 10, 1, 1, 0.1, ob, b, b) == E
    assert lib.kg_keldysh_get_phi(None, 0, b) == E
    assert lib.kg_keldysh_set_phi(None, 0, b) == E
    assert lib.kg_overlaps(None, 1, b, 1, 4, b, None) == E
    assert lib.kg_overlaps(b, 0, b, 1, 4, b, None) == E
    assert lib.kg_overlaps(b, 33, b, 1, 4, b, None) == E
    assert lib.kg_overlaps_noalloc(b, 1, None, 1, 4, b, None) == E
    assert lib.kg_overlaps_noalloc(b, 1, b, 65, 4, b, None) == E
    assert lib.kg_green_matsubara(None, orb.ctypes.data, 1, 10, 0.0, b, 1, ob, b, b) == E
    assert lib.kg_green_matsubara_steps(None, orb.ctypes.data, 1, 0.0, 0.1, 1, ob, b, b) == E
    assert lib.kg_probe_fp64(None, None) == E
    assert lib.kg_green_keldysh_td(None, None, orb.ctypes.data, 1, 0.1, 3, b, ob, b, b) == E
    assert lib.kg_keldysh_create_td(None, None, orb.ctypes.data, 1, 0.1, 3, b, ob, None) == E
    ops = np.zeros(12, dtype=np.int32)
    assert lib.kg_green_four_time(None, None, ops.ctypes.data, 0.1, 2, ob, b) == E
    assert lib.kg_necpt_occupations(None, None, 10, 1.0, 1.0, 0.1, 2, 15.0, 10, ob, b) == E
    lib.kg_free_sector(None)
    lib.kg_keldysh_free(None)
    lib.kg_opts_default(None)
