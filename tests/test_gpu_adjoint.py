"""The adjoint of the equilibrium Green's function.

The library's vector-Jacobian product is checked against
* the oracle's analytic gradient (first-order perturbation theory of the
  Lehmann form from dense eigen-decompositions) on the bath-fitting star at
  L = 6 and L = 8 (d = 400 and 4,900, 401 times) and on a complex-hopping
  model, to 1e-8 relative;
* central finite differences (h = 1e-6) of the CPU oracle's forward (an
  independent Chebyshev propagation) on small models with every cotangent
  path active;
* at the full size of the bath-fitting workload (star SIAM L = 10, (5,5),
  d = 63,504): central differences of the oracle's forward on a short grid,
  and central differences of the GPU forward on all 401 times (checkpoints
  every 20 steps).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1109_1205_gb300 as kg  # noqa: E402
from paper_1109_1205_gb300.autograd import green_equilibrium  # noqa: E402

FD_H = 1e-6


def linear_loss(Gg, Gl, A, B):
    return float(np.sum((np.conj(A) * Gg).real) + np.sum((np.conj(B) * Gl).real))


def sector_dim(m):
    return math.comb(m["L"], m["n_up"]) * math.comb(m["L"], m["n_dn"])


def oracle_loss(model, orbs, dt, n, A, B):
    # a Krylov space as large as the sector makes the oracle ground state
    # exact to rounding, so the difference quotients see no convergence noise
    Gg, Gl, _ = oracle.green_equilibrium(model, orbs, dt, n, K=max(80, sector_dim(model)), tol=1e-14)
    return linear_loss(Gg, Gl, A, B)


def perturbed(model, kind, idx, delta):
    m = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in model.items()}
    if kind == "eps":
        m["eps"][idx] += delta
    elif kind == "U":
        m["U"][idx] += delta
    elif kind == "re":
        a, b = idx
        m["h"][a, b] += delta
        m["h"][b, a] += delta
    elif kind == "im":
        a, b = idx
        m["h"][a, b] += 1j * delta
        m["h"][b, a] -= 1j * delta
    return m


def fd(model, kind, idx, loss):
    return (loss(perturbed(model, kind, idx, FD_H)) - loss(perturbed(model, kind, idx, -FD_H))) / (2 * FD_H)


def check_case(model, orbs, dt, n, checkpoint, seed, kinds):
    rng = np.random.default_rng(seed)
    shape = (n + 1, len(orbs), len(orbs))
    A = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    B = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    L = model["L"]
    s = kg.Sector(model)
    g_eps, g_hre, g_him, g_U = kg.kg_green_equilibrium_vjp(s.handle, L, orbs, dt, n, A, B, checkpoint=checkpoint)
    loss = lambda m: oracle_loss(m, orbs, dt, n, A, B)  # noqa: E731
    checked = 0
    for kind in kinds:
        if kind == "eps":
            items = [((sg, i), g_eps[sg, i]) for sg in range(2) for i in range(L)]
        elif kind == "U":
            items = [(i, g_U[i]) for i in range(L)]
        else:
            items = [((a, b), (g_hre if kind == "re" else g_him)[a, b])
                     for a in range(L) for b in range(a + 1, L) if model["h"][a, b] != 0]
        for idx, g in items:
            ref = fd(model, kind, idx, loss)
            assert abs(g - ref) <= 1e-6 * max(1.0, abs(ref)), (kind, idx, g, ref)
            checked += 1
    return checked


def test_vjp_vs_oracle_fd_real_star():
    m = W.siam_star(-1.5, 3.0, [-1.0, 0.3, 1.2, 2.0], [0.5, 0.7, 0.4, 0.6], 2, 3)
    n = check_case(m, [(0, 0), (0, 1), (2, 0)], 0.05, 30, 7, 11, ["eps", "U", "re"])
    assert n == 10 + 5 + 4


def test_vjp_vs_oracle_fd_complex_hopping():
    m = W.random_model(4, 2, 1, seed=31, complex_hopping=True)
    check_case(m, [(0, 0), (3, 1)], 0.07, 16, 5, 12, ["eps", "U", "re", "im"])


def c5_like(L, seed, eps_d=-2.0):
    rng = np.random.default_rng(seed)
    U = float(rng.uniform(1, 8))
    ek, vk = rng.uniform(-3, 3, L - 1), rng.uniform(0.2, 1.0, L - 1)
    return W.siam_star(eps_d, U, ek, vk, L // 2, L // 2), ek, vk, U


@pytest.mark.parametrize("L,tol", [(6, 1e-6), (8, 1e-5)])
def test_autograd_bath_fit_vs_oracle_fd(L, tol):
    """The bath-fitting loss sum_t |G_imp(t) - G_target(t)|^2 (G_imp the
    retarded impurity function) through the torch.autograd.Function, against
    oracle central differences in the fitted parameters (eps_k, V_k, U)."""
    dt, n = 0.05, 60 if L == 6 else 24
    tgt, *_ = c5_like(L, 7)
    m, ek, vk, U = c5_like(L, 8)
    Tg, Tl, _ = oracle.green_equilibrium(tgt, [(0, 0)], dt, n, K=120, tol=1e-14)
    T = torch.from_numpy((Tg - Tl)[:, 0, 0])

    def torch_loss(ek_t, vk_t, U_t):
        h = torch.zeros(L, L, dtype=torch.float64)
        h[0, 1:] = vk_t
        h[1:, 0] = vk_t
        eps = torch.zeros(2, L, dtype=torch.float64)
        eps[:, 0] = -2.0
        eps[:, 1:] = ek_t
        Uv = torch.zeros(L, dtype=torch.float64)
        Uv[0] = U_t
        Gg, Gl = green_equilibrium(h, eps, Uv, L, L // 2, L // 2, [(0, 0)], dt, n, checkpoint=7)
        return torch.sum(torch.abs(Gg[:, 0, 0] - Gl[:, 0, 0] - T) ** 2)

    ek_t = torch.tensor(ek, requires_grad=True)
    vk_t = torch.tensor(vk, requires_grad=True)
    U_t = torch.tensor(U, dtype=torch.float64, requires_grad=True)  # a bare float would give float32
    loss = torch_loss(ek_t, vk_t, U_t)
    loss.backward()

    def oracle_l(ek_, vk_, U_):
        mm = W.siam_star(-2.0, U_, ek_, vk_, L // 2, L // 2)
        # restarted Lanczos to a residual of a few 1e-14 (gap ~1): G to ~1e-15
        Gg, Gl, _ = oracle.green_equilibrium(mm, [(0, 0)], dt, n, K=120, tol=1e-14)
        return float(np.sum(np.abs((Gg - Gl)[:, 0, 0] - T.numpy()) ** 2))

    assert abs(loss.item() - oracle_l(ek, vk, U)) < 1e-9
    for k in range(L - 1):
        for arr, grad in ((ek, ek_t.grad), (vk, vk_t.grad)):
            p, q = arr.copy(), arr.copy()
            p[k] += FD_H
            q[k] -= FD_H
            args_p = (p, vk, U) if arr is ek else (ek, p, U)
            args_q = (q, vk, U) if arr is ek else (ek, q, U)
            ref = (oracle_l(*args_p) - oracle_l(*args_q)) / (2 * FD_H)
            assert abs(grad[k].item() - ref) <= tol * max(1.0, abs(ref)), (k, grad[k].item(), ref)
    ref = (oracle_l(ek, vk, U + FD_H) - oracle_l(ek, vk, U - FD_H)) / (2 * FD_H)
    assert abs(U_t.grad.item() - ref) <= tol * max(1.0, abs(ref))


def test_c5_full_size_vs_gpu_fd():
    """The full bath-fitting workload (d = 63,504, 401 times, checkpoints every
    20 steps): adjoint gradient against central differences of the GPU
    forward in the 19 fitted parameters.  The difference step is 1e-4: each
    perturbed forward converges its own ground state to a residual of about
    1e-13, which puts ~1e-10 of noise into the loss -- 1e-6 relative at this
    step, against a truncation error of ~1e-8."""
    cfg = W.config_c5()
    L, dt, n, orbs = 10, cfg["dt"], cfg["n_steps"], cfg["orbitals"]
    opts = kg.kg_opts_default(M=cfg["M"], tol_resid=1e-14, max_restarts=1000)
    h = 1e-4
    Tg, Tl = kg.Sector(cfg["target"]).green_equilibrium(orbs, dt, n, opts)
    T = (Tg - Tl)[:, 0, 0]
    m = cfg["start"]

    def gpu_loss(model):
        Gg, Gl = kg.Sector(model).green_equilibrium(orbs, dt, n, opts)
        return float(np.sum(np.abs((Gg - Gl)[:, 0, 0] - T) ** 2)), Gg, Gl

    L0, Gg, Gl = gpu_loss(m)
    r = 2.0 * ((Gg - Gl)[:, 0, 0] - T)
    dGg = np.zeros_like(Gg)
    dGl = np.zeros_like(Gl)
    dGg[:, 0, 0] = r
    dGl[:, 0, 0] = -r
    s = kg.Sector(m)
    g_eps, g_hre, _, g_U = kg.kg_green_equilibrium_vjp(s.handle, L, orbs, dt, n, dGg, dGl, opts, checkpoint=20)
    grads = {("U", 0): g_U[0]}
    for k in range(1, L):
        grads[("e", k)] = g_eps[0, k] + g_eps[1, k]
        grads[("v", k)] = g_hre[0, k]
    for (kind, k), g in grads.items():
        def pert(delta):
            mm = {kk: (v.copy() if isinstance(v, np.ndarray) else v) for kk, v in m.items()}
            if kind == "U":
                mm["U"][0] += delta
            elif kind == "e":
                mm["eps"][:, k] += delta
            else:
                mm["h"][0, k] += delta
                mm["h"][k, 0] += delta
            return mm
        ref = (gpu_loss(pert(h))[0] - gpu_loss(pert(-h))[0]) / (2 * h)
        assert abs(g - ref) <= 2e-5 * max(1.0, abs(ref)), (kind, k, g, ref)


# ------------------------------------------- the dense-oracle gradient
def _compare(got, ref, tol, model):
    """All eps and U gradients, and the hopping gradients of the model's bonds
    and the diagonal (the library returns zero for pairs absent from the
    model, which the oracle differentiates too)."""
    bonds = (model["h"] != 0) | np.eye(model["L"], dtype=bool)
    ref = (ref[0], np.where(bonds, ref[1], 0.0), np.where(bonds, ref[2], 0.0), ref[3])
    scale = max(1.0, max(float(np.max(np.abs(r))) for r in ref))
    for name, g, r in zip(("eps", "hre", "him", "U"), got, ref):
        assert np.max(np.abs(np.asarray(g) - r)) <= tol * scale, (name, np.max(np.abs(np.asarray(g) - r)), scale)


@pytest.mark.parametrize("L", [6, 8])
def test_vjp_vs_dense_oracle_gradient_bath_fit(L):
    """The bath-fitting gradient of the adjoint workload's star model (401
    times, checkpoints every 20 steps) at L = 6 (d = 400) and L = 8 (d = 4,900)
    against the oracle's analytic gradient, every parameter (eps of both spins,
    U, every hopping pair's real and imaginary part)."""
    dt, n = 0.05, 400
    tgt, *_ = c5_like(L, 7)
    m, *_ = c5_like(L, 8)
    orbs = [(0, 0)]
    Tg, Tl, _ = oracle.green_equilibrium(tgt, orbs, dt, n, K=120, tol=1e-14)
    Gg, Gl, _ = oracle.green_equilibrium(m, orbs, dt, n, K=120, tol=1e-14)
    r = 2.0 * ((Gg - Gl) - (Tg - Tl))
    ref = oracle.green_equilibrium_grad_dense(m, orbs, dt, n, r, -r)
    s = kg.Sector(m)
    got = kg.kg_green_equilibrium_vjp(s.handle, L, orbs, dt, n, r, -r, checkpoint=20)
    _compare(got, ref, 1e-8, m)


def test_vjp_vs_dense_oracle_gradient_complex_two_spins():
    """Random complex cotangents on both parts, orbitals of both spins and a
    complex Hermitian hopping matrix with some bonds absent (d = 300, 200
    times)."""
    m = W.random_model(6, 3, 2, seed=44, complex_hopping=True, density=0.7)
    orbs = [(0, 0), (3, 0), (2, 1)]
    dt, n = 0.05, 200
    rng = np.random.default_rng(45)
    shape = (n + 1, len(orbs), len(orbs))
    A = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    B = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = oracle.green_equilibrium_grad_dense(m, orbs, dt, n, A, B)
    s = kg.Sector(m)
    got = kg.kg_green_equilibrium_vjp(s.handle, 6, orbs, dt, n, A, B, checkpoint=13)
    _compare(got, ref, 1e-8, m)


def test_c5_full_size_vs_oracle_fd():
    """The full-size bath-fitting sector (d = 63,504) on a short grid (41
    times): the adjoint against central differences of the oracle's forward
    in U, one eps_k and one V_k.  Step 1e-4: the oracle's ground state is
    converged to a residual of 1e-14, which leaves ~1e-12 of noise in the
    loss, 1e-8 after the division; the truncation error is ~1e-8."""
    cfg = W.config_c5()
    L, dt, n, orbs = 10, cfg["dt"], 40, cfg["orbitals"]
    h = 1e-4
    Tg, Tl, _ = oracle.green_equilibrium(cfg["target"], orbs, dt, n, K=80, tol=1e-14)
    T = (Tg - Tl)[:, 0, 0]
    m = cfg["start"]

    def loss(model):
        Gg, Gl, _ = oracle.green_equilibrium(model, orbs, dt, n, K=80, tol=1e-14)
        return float(np.sum(np.abs((Gg - Gl)[:, 0, 0] - T) ** 2)), Gg, Gl

    _, Gg, Gl = loss(m)
    r = 2.0 * ((Gg - Gl)[:, 0, 0] - T)
    dGg = np.zeros_like(Gg)
    dGl = np.zeros_like(Gl)
    dGg[:, 0, 0] = r
    dGl[:, 0, 0] = -r
    s = kg.Sector(m)
    opts = kg.kg_opts_default(M=cfg["M"], tol_resid=1e-14, max_restarts=1000)
    g_eps, g_hre, _, g_U = kg.kg_green_equilibrium_vjp(s.handle, L, orbs, dt, n, dGg, dGl, opts, checkpoint=20)
    for kind, k, g in (("U", 0, g_U[0]), ("e", 4, g_eps[0, 4] + g_eps[1, 4]), ("v", 7, g_hre[0, 7])):
        def pert(delta):
            mm = {kk: (v.copy() if isinstance(v, np.ndarray) else v) for kk, v in m.items()}
            if kind == "U":
                mm["U"][0] += delta
            elif kind == "e":
                mm["eps"][:, k] += delta
            else:
                mm["h"][0, k] += delta
                mm["h"][k, 0] += delta
            return mm
        ref = (loss(pert(h))[0] - loss(pert(-h))[0]) / (2 * h)
        assert abs(g - ref) <= 2e-6 * max(1.0, abs(ref)), (kind, k, g, ref)


def test_autograd_frees_the_sector_without_backward(monkeypatch):
    """A forward whose graph is dropped without a backward releases its sector
    handle; CUDA inputs give CUDA outputs."""
    import gc

    from paper_1109_1205_gb300 import _lib
    freed = []
    orig = _lib.kg_free_sector
    monkeypatch.setattr(_lib, "kg_free_sector", lambda hdl: (freed.append(hdl), orig(hdl))[1])
    m = W.siam_star(-1.5, 3.0, [-1.0, 0.3, 1.2], [0.5, 0.7, 0.4], 2, 2)
    h = torch.tensor(m["h"].real, device="cuda", requires_grad=True)
    eps = torch.tensor(m["eps"], device="cuda")
    Uv = torch.tensor(m["U"], device="cuda")
    Gg, Gl = green_equilibrium(h, eps, Uv, 4, 2, 2, [(0, 0)], 0.1, 5)
    assert Gg.is_cuda and Gl.is_cuda
    del Gg, Gl
    gc.collect()
    assert len(freed) == 1
    Gg, Gl = green_equilibrium(h, eps, Uv, 4, 2, 2, [(0, 0)], 0.1, 5)
    (Gg.abs().sum() + Gl.abs().sum()).backward()
    assert len(freed) == 2 and h.grad is not None and h.grad.is_cuda
