"""ctypes marshalling for libkrylovgf (see include/krylovgf.h for semantics).

Host arrays are numpy complex128 / float64; device vectors are anything with
a `data_ptr()` (torch CUDA tensors) or a raw integer device address.  Complex
vectors are interleaved (re, im), i.e. numpy/torch complex128 layout.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "_build", "libkrylovgf.so")

if not os.path.exists(library_path):
    raise ImportError(
        "libkrylovgf.so is not built (%s); run __graft_entry__.build() or "
        "python paper_1109_1205_gb300/build.py" % library_path)
lib = ctypes.CDLL(library_path)

KG_OK, KG_EINVAL, KG_ENOMEM, KG_ENOCONV, KG_EDEGEN = 0, -1, -2, -3, -4
KG_EBREAKDOWN, KG_ENUMERIC, KG_ETIMEOUT, KG_ECUDA = -5, -6, -7, -8


class Opts(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int),
        ("M_gs", ctypes.c_int),
        ("max_restarts", ctypes.c_int),
        ("tol_resid", ctypes.c_double),
        ("reorth", ctypes.c_int),
        ("mem_budget_mb", ctypes.c_int),
        ("schedule", ctypes.c_int),
        ("use_graphs", ctypes.c_int),
        ("dt_internal", ctypes.c_double),
        ("seed", ctypes.c_ulonglong),
        ("stream", ctypes.c_void_p),
    ]


class KGError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = lib.kg_last_error().decode()
        super().__init__("%s: %s (%d): %s" % (where, lib.kg_strerror(code).decode(), code, msg))


_P, _I, _D, _LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
_sig = {
    "kg_opts_default": (None, [ctypes.POINTER(Opts)]),
    "kg_build_sector": (_I, [_I, _I, _I, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "kg_free_sector": (None, [_P]),
    "kg_sector_dims": (_I, [_P, ctypes.POINTER(_LL), ctypes.POINTER(_LL), ctypes.POINTER(_LL)]),
    "kg_sector_strings": (_I, [_P, _P, _P]),
    "kg_hpsi": (_I, [_P, _P, _P, _P]),
    "kg_neighbour_dim": (_I, [_P, _I, _I, ctypes.POINTER(_LL)]),
    "kg_apply_cop": (_I, [_P, _I, _I, _I, _P, _P, _P]),
    "kg_overlaps": (_I, [_P, _I, _P, _I, _LL, _P, _P]),
    "kg_overlaps_noalloc": (_I, [_P, _I, _P, _I, _LL, _P, _P]),
    "kg_ground_state": (_I, [_P, ctypes.POINTER(Opts), ctypes.POINTER(_D), ctypes.POINTER(_D),
                             ctypes.POINTER(_D)]),
    "kg_copy_ground_state": (_I, [_P, _P, _I]),
    "kg_propagate": (_I, [_P, _P, _D, _I, ctypes.POINTER(Opts)]),
    "kg_green_equilibrium": (_I, [_P, _P, _I, _D, _I, ctypes.POINTER(Opts), _P, _P]),
    "kg_green_keldysh": (_I, [_P, _P, _P, _I, _D, _I, ctypes.POINTER(Opts), _P, _P]),
    "kg_green_equilibrium_batched": (_I, [_P, _I, _P, _I, _D, _I, ctypes.POINTER(Opts), _P, _P, _P]),
    "kg_green_equilibrium_vjp": (_I, [_P, _P, _I, _D, _I, ctypes.POINTER(Opts), _I, _P, _P, _P, _P, _P, _P]),
    "kg_green_lanczos": (_I, [_P, _P, _I, _I, _P, _I, _D, ctypes.POINTER(Opts), _P, _P, _P]),
    "kg_green_equilibrium_fine": (_I, [_P, _P, _I, _D, _I, _I, ctypes.POINTER(Opts), _P, _P]),
    "kg_green_fourier": (_I, [_P, _I, _I, _D, _P, _I, _D, _P, _P]),
    "kg_green_matsubara": (_I, [_P, _P, _I, _I, _D, _P, _I, ctypes.POINTER(Opts), _P, _P]),
    "kg_green_matsubara_steps": (_I, [_P, _P, _I, _D, _D, _I, ctypes.POINTER(Opts), _P, _P]),
    "kg_keldysh_create": (_I, [_P, _P, _P, _I, _D, _I, ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "kg_green_keldysh_td": (_I, [_P, _P, _P, _I, _D, _I, _P, ctypes.POINTER(Opts), _P, _P]),
    "kg_green_four_time": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(Opts), _P]),
    "kg_necpt_occupations": (_I, [_P, _P, _I, _D, _D, _D, _I, _D, _I, ctypes.POINTER(Opts), _P]),
    "kg_keldysh_create_td": (_I, [_P, _P, _P, _I, _D, _I, _P, ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "kg_green_mixed": (_I, [_P, _P, _P, _I, _D, _I, _D, _D, _I, ctypes.POINTER(Opts), _P, _P]),
    "kg_green_restarted": (_I, [_P, _P, _I, _I, _I, _I, _D, ctypes.POINTER(Opts), _P, _P]),
    "kg_keldysh_row": (_I, [_P, _I, _P, _P]),
    "kg_keldysh_gram": (_I, [_P, _P, _P]),
    "kg_keldysh_plan": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                             ctypes.POINTER(_LL)]),
    "kg_keldysh_get_phi": (_I, [_P, _I, _P]),
    "kg_keldysh_set_phi": (_I, [_P, _I, _P]),
    "kg_keldysh_free": (None, [_P]),
    "kg_strerror": (ctypes.c_char_p, [_I]),
    "kg_last_error": (ctypes.c_char_p, []),
    "kg_launch_count": (ctypes.c_ulonglong, []),
    "kg_profile_start": (_I, []),
    "kg_profile_stop": (_I, []),
    "kg_profile_count": (_I, []),
    "kg_profile_get": (_I, [_I, ctypes.c_char_p, _I, ctypes.POINTER(_LL), ctypes.POINTER(_D)]),
    "kg_probe_fp64": (_I, [ctypes.POINTER(_D), _P]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _check(rc, where):
    if rc != KG_OK:
        raise KGError(rc, where)
    return rc


def _addr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("expected a device tensor, numpy array or address, got %r" % type(x))


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return getattr(stream, "cuda_stream", stream)


def _orb_array(orbitals):
    return np.ascontiguousarray(np.asarray(orbitals, dtype=np.int32).reshape(-1, 2))


# ------------------------------------------------ same-name thin wrappers
def kg_opts_default(**overrides):
    o = Opts()
    lib.kg_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "stream":
            v = _stream(v)
        setattr(o, k, v)
    return o


def kg_build_sector(L, n_up, n_dn, h, eps, U):
    h = np.asarray(h, dtype=np.complex128).reshape(L, L)
    h_re = np.ascontiguousarray(h.real, dtype=np.float64)
    h_im = np.ascontiguousarray(h.imag, dtype=np.float64)
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(2 * L))
    U = np.ascontiguousarray(np.broadcast_to(np.asarray(U, dtype=np.float64), (L,)))
    out = _P()
    _check(lib.kg_build_sector(L, n_up, n_dn, h_re.ctypes.data, h_im.ctypes.data if np.any(h_im) else None,
                               eps.ctypes.data, U.ctypes.data, ctypes.byref(out)), "kg_build_sector")
    return out.value


def kg_free_sector(handle):
    lib.kg_free_sector(handle)


def kg_sector_dims(handle):
    d, du, dd = _LL(), _LL(), _LL()
    _check(lib.kg_sector_dims(handle, ctypes.byref(d), ctypes.byref(du), ctypes.byref(dd)), "kg_sector_dims")
    return d.value, du.value, dd.value


def kg_sector_strings(handle):
    _, du, dd = kg_sector_dims(handle)
    up = np.empty(du, dtype=np.uint32)
    dn = np.empty(dd, dtype=np.uint32)
    _check(lib.kg_sector_strings(handle, up.ctypes.data, dn.ctypes.data), "kg_sector_strings")
    return up, dn


def kg_hpsi(handle, x_dev, y_dev, stream=None):
    _check(lib.kg_hpsi(handle, _addr(x_dev), _addr(y_dev), _stream(stream)), "kg_hpsi")


def kg_neighbour_dim(handle, spin, dagger):
    d = _LL()
    _check(lib.kg_neighbour_dim(handle, spin, 1 if dagger else 0, ctypes.byref(d)), "kg_neighbour_dim")
    return d.value


def kg_apply_cop(handle, site, spin, dagger, x_dev, y_dev, stream=None):
    _check(lib.kg_apply_cop(handle, site, spin, 1 if dagger else 0, _addr(x_dev), _addr(y_dev), _stream(stream)),
           "kg_apply_cop")


def kg_overlaps(X_dev, n_x, Y_dev, n_y, d, G_dev, stream=None):
    """G[b][a] = <x_a|y_b> on the device (complex [n_y][n_x])."""
    _check(lib.kg_overlaps(_addr(X_dev), int(n_x), _addr(Y_dev), int(n_y), int(d), _addr(G_dev), _stream(stream)),
           "kg_overlaps")


def kg_overlaps_noalloc(X_dev, n_x, Y_dev, n_y, d, G_dev, stream=None):
    """kg_overlaps without device allocation (library-held scratch, n_y <= 64)."""
    _check(lib.kg_overlaps_noalloc(_addr(X_dev), int(n_x), _addr(Y_dev), int(n_y), int(d), _addr(G_dev),
                                   _stream(stream)), "kg_overlaps_noalloc")


def kg_ground_state(handle, opts=None):
    o = opts if opts is not None else kg_opts_default()
    e0, res, gap = _D(), _D(), _D()
    rc = lib.kg_ground_state(handle, ctypes.byref(o), ctypes.byref(e0), ctypes.byref(res), ctypes.byref(gap))
    _check(rc, "kg_ground_state")
    return e0.value, res.value, gap.value


def kg_copy_ground_state(handle, out, to_host=True):
    _check(lib.kg_copy_ground_state(handle, _addr(out), 1 if to_host else 0), "kg_copy_ground_state")
    return out


def kg_propagate(handle, x_dev, dt, n_steps, opts=None):
    o = opts if opts is not None else kg_opts_default()
    _check(lib.kg_propagate(handle, _addr(x_dev), float(dt), int(n_steps), ctypes.byref(o)), "kg_propagate")


def kg_green_equilibrium(handle, orbitals, dt, n_steps, opts=None):
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    n = orb.shape[0]
    Gg = np.zeros((n_steps + 1, n, n), dtype=np.complex128)
    Gl = np.zeros_like(Gg)
    _check(lib.kg_green_equilibrium(handle, orb.ctypes.data, n, float(dt), int(n_steps), ctypes.byref(o),
                                    Gg.ctypes.data, Gl.ctypes.data), "kg_green_equilibrium")
    return Gg, Gl


def kg_green_equilibrium_fine(handle, orbitals, dt, n_steps, fine, opts=None):
    """Equilibrium G on the grid t_k = k dt with one Krylov space per `fine`
    output times (Krylov step fine*dt); same layout as kg_green_equilibrium."""
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    n = orb.shape[0]
    Gg = np.zeros((n_steps + 1, n, n), dtype=np.complex128)
    Gl = np.zeros_like(Gg)
    _check(lib.kg_green_equilibrium_fine(handle, orb.ctypes.data, n, float(dt), int(n_steps), int(fine),
                                         ctypes.byref(o), Gg.ctypes.data, Gl.ctypes.data), "kg_green_equilibrium_fine")
    return Gg, Gl


def kg_green_equilibrium_batched(handles, orbitals, dt, n_steps, opts=None):
    """Equilibrium G of many sectors in one batch; returns (G_gtr, G_les, status)
    with G of shape [n_inst, n_steps+1, n_orb, n_orb]."""
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    n = orb.shape[0]
    arr = (_P * len(handles))(*handles)
    Gg = np.zeros((len(handles), n_steps + 1, n, n), dtype=np.complex128)
    Gl = np.zeros_like(Gg)
    status = np.zeros(len(handles), dtype=np.int32)
    _check(lib.kg_green_equilibrium_batched(ctypes.cast(arr, _P), len(handles), orb.ctypes.data, n, float(dt),
                                            int(n_steps), ctypes.byref(o), Gg.ctypes.data, Gl.ctypes.data,
                                            status.ctypes.data), "kg_green_equilibrium_batched")
    return Gg, Gl, status


def kg_green_equilibrium_vjp(handle, L, orbitals, dt, n_steps, dG_gtr=None, dG_les=None, opts=None, checkpoint=0):
    """Gradients (g_eps [2, L], g_hre [L, L], g_him [L, L], g_U [L]) of a loss
    whose cotangents with respect to G^> and G^< are dG_gtr, dG_les."""
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    n = orb.shape[0]
    shape = (n_steps + 1, n, n)
    dg = None if dG_gtr is None else np.ascontiguousarray(np.asarray(dG_gtr, dtype=np.complex128).reshape(shape))
    dl = None if dG_les is None else np.ascontiguousarray(np.asarray(dG_les, dtype=np.complex128).reshape(shape))
    g_eps = np.zeros((2, L))
    g_hre = np.zeros((L, L))
    g_him = np.zeros((L, L))
    g_U = np.zeros(L)
    _check(lib.kg_green_equilibrium_vjp(handle, orb.ctypes.data, n, float(dt), int(n_steps), ctypes.byref(o),
                                        int(checkpoint), None if dg is None else dg.ctypes.data,
                                        None if dl is None else dl.ctypes.data, g_eps.ctypes.data, g_hre.ctypes.data,
                                        g_him.ctypes.data, g_U.ctypes.data), "kg_green_equilibrium_vjp")
    return g_eps, g_hre, g_him, g_U


def kg_green_lanczos(handle, orbitals, n, omega, eta, opts=None):
    """Lanczos (continued-fraction) Green's function of the diagonal orbitals:
    returns (G_gtr, G_les, coef) with G of shape [n_orb, n_omega] (complex) and
    coef [n_orb, 2, 2n] (particle / hole; a_0..a_{n-1}, b_0..b_{n-1})."""
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    n_orb = orb.shape[0]
    w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).ravel())
    Gg = np.zeros((n_orb, w.size), dtype=np.complex128)
    Gl = np.zeros_like(Gg)
    coef = np.zeros((n_orb, 2, 2 * n), dtype=np.float64)
    _check(lib.kg_green_lanczos(handle, orb.ctypes.data, n_orb, int(n), w.ctypes.data if w.size else None, w.size,
                                float(eta), ctypes.byref(o), Gg.ctypes.data, Gl.ctypes.data, coef.ctypes.data),
           "kg_green_lanczos")
    return Gg, Gl, coef


def kg_green_matsubara(handle, orbitals, n, mu, tau, opts=None):
    """Zero-temperature Matsubara function of the diagonal orbitals from
    n-step Lanczos runs: returns (G_plus, G_minus), real [n_orb, n_tau], with
    G_plus[a, j] = G^M_aa(+tau_j) and G_minus[a, j] = G^M_aa(-tau_j)."""
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    n_orb = orb.shape[0]
    t = np.ascontiguousarray(np.asarray(tau, dtype=np.float64).ravel())
    Gp = np.zeros((n_orb, t.size), dtype=np.float64)
    Gm = np.zeros_like(Gp)
    _check(lib.kg_green_matsubara(handle, orb.ctypes.data, n_orb, int(n), float(mu), t.ctypes.data if t.size else None,
                                  t.size, ctypes.byref(o), Gp.ctypes.data if Gp.size else None,
                                  Gm.ctypes.data if Gm.size else None), "kg_green_matsubara")
    return Gp, Gm


def kg_green_matsubara_steps(handle, orbitals, mu, dtau, n_steps, opts=None):
    """Zero-temperature Matsubara function on tau_k = k dtau by imaginary-time
    Krylov steps: returns (G_plus, G_minus), complex [n_steps+1, n_orb, n_orb]
    with G_plus[k, a, b] = G^M_ab(+tau_k) and G_minus[k, a, b] = G^M_ab(-tau_k)."""
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    n = orb.shape[0]
    Gp = np.zeros((n_steps + 1, n, n), dtype=np.complex128)
    Gm = np.zeros_like(Gp)
    _check(lib.kg_green_matsubara_steps(handle, orb.ctypes.data, n, float(mu), float(dtau), int(n_steps),
                                        ctypes.byref(o), Gp.ctypes.data, Gm.ctypes.data), "kg_green_matsubara_steps")
    return Gp, Gm


def kg_green_fourier(G_t, dt, omega, eta, stream=None):
    """Damped Fourier transform sum_k w_k e^{i(omega + i eta) t_k} G(t_k),
    t_k = k dt, trapezoidal weights, of each row of G_t (complex [n_series,
    n_t], or one series [n_t]); returns complex [n_series, n_omega] (or
    [n_omega] for one series)."""
    g = np.ascontiguousarray(np.asarray(G_t, dtype=np.complex128))
    one = g.ndim == 1
    g = g.reshape(1, -1) if one else g.reshape(g.shape[0], g.shape[-1])
    w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).ravel())
    out = np.zeros((g.shape[0], w.size), dtype=np.complex128)
    _check(lib.kg_green_fourier(g.ctypes.data if g.size else None, g.shape[0], g.shape[1], float(dt),
                                w.ctypes.data if w.size else None, w.size, float(eta), _stream(stream),
                                out.ctypes.data if out.size else None), "kg_green_fourier")
    return out[0] if one else out


def kg_green_keldysh(h_ini, h_fin, orbitals, dt, n_t, opts=None):
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    n = orb.shape[0]
    Gl = np.zeros((n_t, n_t, n, n), dtype=np.complex128)
    Gg = np.zeros_like(Gl)
    _check(lib.kg_green_keldysh(h_ini, h_fin, orb.ctypes.data, n, float(dt), int(n_t), ctypes.byref(o),
                                Gl.ctypes.data, Gg.ctypes.data), "kg_green_keldysh")
    return Gl, Gg


def _dparams_array(dparams):
    if dparams is None:
        return None
    return np.ascontiguousarray(np.asarray(dparams, dtype=np.float64))


def kg_green_keldysh_td(h_ini, h_fin, orbitals, dt, n_t, dparams, opts=None):
    """Keldysh G^<, G^> for the driven H(t): dparams [(n_t-1) n_sub, 2, 3L]
    (offsets of eps_up, eps_dn, U at the two Gauss nodes of each internal step)."""
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    n = orb.shape[0]
    dp = _dparams_array(dparams)
    Gl = np.zeros((n_t, n_t, n, n), dtype=np.complex128)
    Gg = np.zeros_like(Gl)
    _check(lib.kg_green_keldysh_td(h_ini, h_fin, orb.ctypes.data, n, float(dt), int(n_t),
                                   dp.ctypes.data if dp is not None and dp.size else None, ctypes.byref(o),
                                   Gl.ctypes.data, Gg.ctypes.data), "kg_green_keldysh_td")
    return Gl, Gg


def kg_green_four_time(h_ini, h_fin, ops, dt, n_t, opts=None):
    """<0|A1(t1) A2(t2) A3(t3) A4(t4)|0> on t_k = k dt: ops = four (site, spin,
    dagger) triples; returns complex [n_t, n_t, n_t, n_t]."""
    o = opts if opts is not None else kg_opts_default()
    op = np.ascontiguousarray(np.asarray(ops, dtype=np.int32).reshape(12))
    G = np.zeros((n_t,) * 4, dtype=np.complex128)
    _check(lib.kg_green_four_time(h_ini, h_fin, op.ctypes.data, float(dt), int(n_t), ctypes.byref(o),
                                  G.ctypes.data), "kg_green_four_time")
    return G


def kg_necpt_occupations(ini, fin, L_b, T_b, V, dt, n_t, beta, n_tau, opts=None):
    """NE-CPT occupations n[spin, k, i] of the cluster sites (Sector objects
    ini, fin) coupled to the bath chain (Section 5), on t_k = k dt."""
    o = opts if opts is not None else kg_opts_default()
    out = np.zeros((2, int(n_t), fin.L))
    _check(lib.kg_necpt_occupations(ini.handle, fin.handle, int(L_b), float(T_b), float(V), float(dt), int(n_t),
                                    float(beta), int(n_tau), ctypes.byref(o), out.ctypes.data), "kg_necpt_occupations")
    return out


def kg_keldysh_create_td(h_ini, h_fin, orbitals, dt, n_t, dparams, opts=None):
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    dp = _dparams_array(dparams)
    out = _P()
    _check(lib.kg_keldysh_create_td(h_ini, h_fin, orb.ctypes.data, orb.shape[0], float(dt), int(n_t),
                                    dp.ctypes.data if dp is not None and dp.size else None, ctypes.byref(o),
                                    ctypes.byref(out)), "kg_keldysh_create_td")
    return out.value


def kg_green_restarted(handle, orbitals, n, f, q, dt, opts=None):
    """Equilibrium G^>, G^< on t_k = k dt, k = 0..f q, one Krylov space of
    dimension n per interval of q steps; arrays [f q + 1, n_orb, n_orb]."""
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    m = orb.shape[0]
    Gg = np.zeros((f * q + 1, m, m), dtype=np.complex128)
    Gl = np.zeros_like(Gg)
    _check(lib.kg_green_restarted(handle, orb.ctypes.data, m, int(n), int(f), int(q), float(dt), ctypes.byref(o),
                                  Gg.ctypes.data, Gl.ctypes.data), "kg_green_restarted")
    return Gg, Gl


def kg_green_mixed(h_ini, h_fin, orbitals, dt, n_t, mu, dtau, n_tau, opts=None):
    """Mixed components (G_right [n_t, n_tau+1, n, n], G_left [n_tau+1, n_t, n, n])."""
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    n = orb.shape[0]
    Gr = np.zeros((n_t, n_tau + 1, n, n), dtype=np.complex128)
    Gl = np.zeros((n_tau + 1, n_t, n, n), dtype=np.complex128)
    _check(lib.kg_green_mixed(h_ini, h_fin, orb.ctypes.data, n, float(dt), int(n_t), float(mu), float(dtau),
                              int(n_tau), ctypes.byref(o), Gr.ctypes.data, Gl.ctypes.data), "kg_green_mixed")
    return Gr, Gl


def kg_keldysh_create(h_ini, h_fin, orbitals, dt, n_t, opts=None):
    o = opts if opts is not None else kg_opts_default()
    orb = _orb_array(orbitals)
    out = _P()
    _check(lib.kg_keldysh_create(h_ini, h_fin, orb.ctypes.data, orb.shape[0], float(dt), int(n_t),
                                 ctypes.byref(o), ctypes.byref(out)), "kg_keldysh_create")
    return out.value


def kg_keldysh_row(handle, k, n_orb):
    Gl = np.zeros((n_orb, n_orb), dtype=np.complex128)
    Gg = np.zeros_like(Gl)
    _check(lib.kg_keldysh_row(handle, int(k), Gl.ctypes.data, Gg.ctypes.data), "kg_keldysh_row")
    return Gl, Gg


def kg_keldysh_gram(handle, n_t, n_orb):
    Gl = np.zeros((n_t, n_t, n_orb, n_orb), dtype=np.complex128)
    Gg = np.zeros_like(Gl)
    _check(lib.kg_keldysh_gram(handle, Gl.ctypes.data, Gg.ctypes.data), "kg_keldysh_gram")
    return Gl, Gg


def kg_keldysh_plan(handle):
    """The Keldysh memory plan: dict with phi_on_host (0 device, 1 pinned host,
    2 pageable host), stores_kept, planes and budget (bytes)."""
    a, b, c, d = _I(), _I(), _I(), _LL()
    _check(lib.kg_keldysh_plan(handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
           "kg_keldysh_plan")
    return {"phi_on_host": a.value, "stores_kept": b.value, "planes": c.value, "budget": d.value}


def kg_keldysh_get_phi(handle, k, out):
    _check(lib.kg_keldysh_get_phi(handle, int(k), _addr(out)), "kg_keldysh_get_phi")
    return out


def kg_keldysh_set_phi(handle, k, phi):
    _check(lib.kg_keldysh_set_phi(handle, int(k), _addr(phi)), "kg_keldysh_set_phi")


def kg_keldysh_free(handle):
    lib.kg_keldysh_free(handle)


def kg_strerror(code):
    return lib.kg_strerror(code).decode()


def kg_last_error():
    return lib.kg_last_error().decode()


def kg_launch_count():
    return int(lib.kg_launch_count())


def kg_profile_start():
    _check(lib.kg_profile_start(), "kg_profile_start")


def kg_profile_stop():
    """Stops the profiler; returns {kernel name: (launches, total ms)}."""
    _check(lib.kg_profile_stop(), "kg_profile_stop")
    out = {}
    buf = ctypes.create_string_buffer(128)
    for i in range(lib.kg_profile_count()):
        n, ms = _LL(), _D()
        _check(lib.kg_profile_get(i, buf, 128, ctypes.byref(n), ctypes.byref(ms)), "kg_profile_get")
        out[buf.value.decode()] = (n.value, ms.value)
    return out


def kg_probe_fp64(stream=None):
    t = _D()
    _check(lib.kg_probe_fp64(ctypes.byref(t), _stream(stream)), "kg_probe_fp64")
    return t.value


# ------------------------------------------------------------ handles
class Sector:
    """Owning wrapper of a kg_sector handle built from a workloads-style model."""

    def __init__(self, model=None, *, L=None, n_up=None, n_dn=None, h=None, eps=None, U=None):
        if model is not None:
            L, n_up, n_dn = model["L"], model["n_up"], model["n_dn"]
            h, eps, U = model["h"], model["eps"], model["U"]
        self.L, self.n_up, self.n_dn = L, n_up, n_dn
        self.handle = kg_build_sector(L, n_up, n_dn, h, eps, U)
        self.dim, self.D_up, self.D_dn = kg_sector_dims(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            kg_free_sector(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def strings(self):
        return kg_sector_strings(self.handle)

    def hpsi(self, x_dev, y_dev, stream=None):
        kg_hpsi(self.handle, x_dev, y_dev, stream)

    def neighbour_dim(self, spin, dagger):
        return kg_neighbour_dim(self.handle, spin, dagger)

    def apply_cop(self, site, spin, dagger, x_dev, y_dev, stream=None):
        kg_apply_cop(self.handle, site, spin, dagger, x_dev, y_dev, stream)

    def ground_state(self, opts=None):
        return kg_ground_state(self.handle, opts)

    def ground_state_vector(self):
        out = np.empty(self.dim, dtype=np.complex128)
        return kg_copy_ground_state(self.handle, out, True)

    def propagate(self, x_dev, dt, n_steps, opts=None):
        kg_propagate(self.handle, x_dev, dt, n_steps, opts)

    def green_equilibrium(self, orbitals, dt, n_steps, opts=None):
        return kg_green_equilibrium(self.handle, orbitals, dt, n_steps, opts)

    def green_restarted(self, orbitals, n, f, q, dt, opts=None):
        return kg_green_restarted(self.handle, orbitals, n, f, q, dt, opts)

    def green_equilibrium_fine(self, orbitals, dt, n_steps, fine, opts=None):
        return kg_green_equilibrium_fine(self.handle, orbitals, dt, n_steps, fine, opts)

    def green_lanczos(self, orbitals, n, omega, eta, opts=None):
        return kg_green_lanczos(self.handle, orbitals, n, omega, eta, opts)

    def green_matsubara(self, orbitals, n, mu, tau, opts=None):
        return kg_green_matsubara(self.handle, orbitals, n, mu, tau, opts)

    def green_matsubara_steps(self, orbitals, mu, dtau, n_steps, opts=None):
        return kg_green_matsubara_steps(self.handle, orbitals, mu, dtau, n_steps, opts)

    def spectrum_td(self, orbitals, dt, n_steps, omega, eta, fine=1, opts=None):
        """Time-dependent Lanczos G(omega) of the diagonal orbitals: the
        equilibrium G(t_k), k = 0..n_steps (one Krylov space per `fine`
        times), then its damped Fourier transform.  Returns (G_gtr, G_les),
        complex [n_orb, n_omega], in the convention of green_lanczos."""
        if fine == 1:
            Gg, Gl = kg_green_equilibrium(self.handle, orbitals, dt, n_steps, opts)
        else:
            Gg, Gl = kg_green_equilibrium_fine(self.handle, orbitals, dt, n_steps, fine, opts)
        n = Gg.shape[1]
        series = np.concatenate([Gg[:, range(n), range(n)].T, -Gl[:, range(n), range(n)].T])
        out = kg_green_fourier(series, dt, omega, eta, None if opts is None else opts.stream)
        return out[:n], out[n:]


class Keldysh:
    """Staged four-step Keldysh calculation (create = steps (i)-(ii))."""

    def __init__(self, ini, fin, orbitals, dt, n_t, opts=None, dparams=None):
        """dparams: the driven H(t) of kg_keldysh_create_td (None: the quench)."""
        self.n_orb = len(orbitals)
        self.n_t = n_t
        self.ini, self.fin = ini, fin  # the sectors must outlive this handle
        if dparams is None:
            self.handle = kg_keldysh_create(ini.handle, fin.handle, orbitals, dt, n_t, opts)
        else:
            self.handle = kg_keldysh_create_td(ini.handle, fin.handle, orbitals, dt, n_t, dparams, opts)

    def row(self, k):
        return kg_keldysh_row(self.handle, k, self.n_orb)

    def gram(self):
        return kg_keldysh_gram(self.handle, self.n_t, self.n_orb)

    def plan(self):
        return kg_keldysh_plan(self.handle)

    def get_phi(self, k):
        out = np.empty(self.fin.dim, dtype=np.complex128)
        return kg_keldysh_get_phi(self.handle, k, out)

    def set_phi(self, k, phi):
        kg_keldysh_set_phi(self.handle, k, np.ascontiguousarray(phi, dtype=np.complex128))

    def close(self):
        if getattr(self, "handle", None):
            kg_keldysh_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
