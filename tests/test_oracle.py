"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every check here uses a route independent of the oracle's own arithmetic:
values printed in the paper, closed forms, torch autograd (Hessian traces,
Jacobians), finite differences, or a dense Kronecker solve.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import kfac_oracle as ko
from synth import inputs as si
from tests import torch_ref as tr

HERE = os.path.dirname(os.path.abspath(__file__))


def _theta(d, widths, seed=0, bias_scale=0.3):
    """Xavier weights plus non-zero biases, so that bias terms are exercised."""
    th = si.xavier_theta(d, widths, seed)
    rng = np.random.default_rng(seed + 100)
    Ws = ko.unpack_theta(th, d, widths)
    for W in Ws:
        W[:, -1] = bias_scale * rng.standard_normal(W.shape[0])
    return ko.pack_theta(Ws)


# --------------------------------------------------------------------------
# Bookkeeping: the parameter counts printed in App. A
# --------------------------------------------------------------------------
def test_param_counts_match_paper():
    with open(os.path.join(HERE, "golden", "param_counts.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        assert si.param_count(c["d"], c["widths"]) == c["D"], c
        Ws = ko.unpack_theta(np.zeros(c["D"]), c["d"], c["widths"])
        assert sum(W.size for W in Ws) == c["D"]


def test_pack_unpack_column_stacking():
    d, widths = 3, (4, 2, 1)
    th = np.arange(si.param_count(d, widths), dtype=float)
    Ws = ko.unpack_theta(th, d, widths)
    # first index fastest: W̃_1[i, j] = theta[i + h_1 * j]
    assert Ws[0][1, 0] == 1.0 and Ws[0][0, 1] == 4.0
    np.testing.assert_array_equal(ko.pack_theta(Ws), th)


# --------------------------------------------------------------------------
# Forward Laplacian (Eq. 6)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d,widths", [(2, (5, 4, 1)), (3, (6, 1)), (4, (3, 5, 2, 1))])
def test_forward_laplacian_vs_autograd_hessian_trace(d, widths):
    th = _theta(d, widths, seed=d)
    X = np.random.default_rng(1).uniform(size=(7, d))
    u, g, lap = ko.forward_laplacian(ko.unpack_theta(th, d, widths), X)
    u_r, g_r, lap_r = tr.value_grad_lap(th, d, widths, X)
    np.testing.assert_allclose(u, u_r, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(g, g_r, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(lap, lap_r, rtol=1e-11, atol=1e-12)


def test_partial_laplacian_heat_vs_autograd():
    d, widths = 5, (6, 4, 1)
    th = _theta(d, widths, seed=3)
    X = np.random.default_rng(2).uniform(size=(5, d))
    u, g, lap = ko.forward_laplacian(ko.unpack_theta(th, d, widths), X, op="heat")
    _, _, lap_r = tr.value_grad_lap(th, d, widths, X, lap_coords=range(1, d))
    np.testing.assert_allclose(lap, lap_r, rtol=1e-11, atol=1e-12)


def test_forward_laplacian_vs_central_differences():
    d, widths = 3, (5, 5, 1)
    th = _theta(d, widths, seed=7)
    Ws = ko.unpack_theta(th, d, widths)
    X = np.random.default_rng(3).uniform(size=(4, d))
    u, g, lap = ko.forward_laplacian(Ws, X)
    h = 1e-4
    for n in range(X.shape[0]):
        lap_fd, g_fd = 0.0, np.zeros(d)
        for i in range(d):
            e = np.zeros(d); e[i] = h
            up = ko.forward_laplacian(Ws, (X[n] + e)[None])[0][0]
            um = ko.forward_laplacian(Ws, (X[n] - e)[None])[0][0]
            lap_fd += (up - 2 * u[n] + um) / h ** 2
            g_fd[i] = (up - um) / (2 * h)
        assert abs(lap_fd - lap[n]) < 1e-5 * max(1.0, abs(lap[n]))
        np.testing.assert_allclose(g_fd, g[n], rtol=1e-6, atol=1e-8)


def test_linear_net_has_zero_laplacian():
    # One linear layer (L = 1): u = W x + b, so ∇u = W and Δu = 0.
    d = 4
    th = np.random.default_rng(0).standard_normal(si.param_count(d, (1,)))
    Ws = ko.unpack_theta(th, d, (1,))
    X = np.random.default_rng(1).uniform(size=(6, d))
    u, g, lap = ko.forward_laplacian(Ws, X)
    np.testing.assert_allclose(u, X @ Ws[0][0, :d] + Ws[0][0, d], rtol=1e-14)
    np.testing.assert_allclose(g, np.broadcast_to(Ws[0][0, :d], g.shape), rtol=1e-14)
    assert np.all(lap == 0.0)


def test_one_hidden_layer_closed_form():
    # u = Σ_j v_j tanh(w_j·x + b_j) + c  ⇒  Δu = Σ_j v_j σ''(a_j) ‖w_j‖²
    d, h = 3, 7
    th = _theta(d, (h, 1), seed=11)
    W1, W2 = ko.unpack_theta(th, d, (h, 1))
    X = np.random.default_rng(5).uniform(size=(9, d))
    a = X @ W1[:, :d].T + W1[:, d]
    y = np.tanh(a)
    s2 = -2 * y * (1 - y * y)
    lap_cf = (W2[0, :h] * s2 * (W1[:, :d] ** 2).sum(axis=1)).sum(axis=1)
    grad_cf = (W2[0, :h] * (1 - y * y)) @ W1[:, :d]
    u, g, lap = ko.forward_laplacian([W1, W2], X)
    np.testing.assert_allclose(lap, lap_cf, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(g, grad_cf, rtol=1e-13, atol=1e-14)


# --------------------------------------------------------------------------
# Manufactured solutions (Eq. 11, Eq. 13, App. A.3, A.6)
# --------------------------------------------------------------------------
def _check_problem(prob, n=5, seed=0):
    import torch
    rng = np.random.default_rng(seed)
    X = rng.uniform(size=(n, prob.d))
    for x in X:
        xt = torch.as_tensor(x, dtype=torch.float64)

        def u_t(z):
            return torch.as_tensor(0.0, dtype=torch.float64) + _torch_u(prob, z)
        H = torch.autograd.functional.hessian(u_t, xt)
        gr = torch.autograd.functional.jacobian(u_t, xt)
        if prob.op == "heat":
            res = float(gr[0] - prob.kappa * sum(H[i, i] for i in range(1, prob.d)))
            assert abs(res - prob.f(x[None])[0]) < 1e-10
        else:
            assert abs(float(-torch.trace(H)) - prob.f(x[None])[0]) < 1e-9
        assert abs(float(u_t(xt)) - prob.u_star(x[None])[0]) < 1e-12


def _torch_u(prob, z):
    import torch
    pi = math.pi
    if prob.name == "poisson2d_sin":
        return torch.sin(pi * z[0]) * torch.sin(pi * z[1])
    if prob.name == "poisson5d_cos":
        return torch.cos(pi * z).sum()
    if prob.name == "poisson100d_norm":
        return (z * z).sum()
    if prob.name == "heat4d_sin":
        return torch.exp(-pi * pi * z[0]) * torch.prod(torch.sin(pi * z[1:]))
    raise KeyError(prob.name)


@pytest.mark.parametrize("name", sorted(si.PROBLEMS))
def test_manufactured_solutions(name):
    _check_problem(si.PROBLEMS[name])


def test_boundary_data_is_solution_on_faces():
    for name, prob in si.PROBLEMS.items():
        _, _, xb, g = si.make_batch(prob, 10, 64, seed=1)
        np.testing.assert_allclose(g, prob.u_star(xb), atol=1e-12)
        on_face = np.any((xb == 0.0) | (xb == 1.0), axis=1)
        assert on_face.all()


# --------------------------------------------------------------------------
# Backward pass: J_W r_n = Σ_s g_{n,s} T̂_{n,s}ᵀ (Sec. 3.2) and ∇L
# --------------------------------------------------------------------------
@pytest.mark.parametrize("op", ["laplace", "heat"])
def test_residual_jacobian_vs_autograd(op):
    d, widths = (3 if op == "laplace" else 4), (5, 4, 1)
    kappa = 0.25 if op == "heat" else 0.0
    th = _theta(d, widths, seed=21)
    Ws = ko.unpack_theta(th, d, widths)
    rng = np.random.default_rng(4)
    X = rng.uniform(size=(4, d))
    f = rng.standard_normal(4)
    fp = ko.taylor_forward(Ws, X, op)
    zb = ko.taylor_adjoint(Ws, fp, ko.residual_seed(fp.S, op, kappa, True), op)
    J = np.concatenate([np.stack([ko.weight_jacobian(zb[l], fp.T_in[l])[n].reshape(-1, order="F")
                                  for n in range(4)]) for l in range(len(Ws))], axis=1)
    J_ref = tr.residual_jacobians(th, d, widths, X, f, op, kappa, interior=True)
    np.testing.assert_allclose(J, J_ref, rtol=1e-10, atol=1e-11)
    r = ko.interior_residual(fp, f, op, kappa)
    np.testing.assert_allclose(r, tr.residuals(th, d, widths, X, f, op, kappa, True), rtol=1e-12, atol=1e-12)


def test_boundary_jacobian_vs_autograd():
    d, widths = 3, (6, 3, 1)
    th = _theta(d, widths, seed=5)
    Ws = ko.unpack_theta(th, d, widths)
    X = np.random.default_rng(6).uniform(size=(5, d))
    g = np.random.default_rng(7).standard_normal(5)
    fp = ko.taylor_forward(Ws, X, with_derivatives=False)
    zb = ko.taylor_adjoint(Ws, fp, ko.residual_seed(1, "laplace", 0.0, False))
    J = np.concatenate([np.stack([ko.weight_jacobian(zb[l], fp.T_in[l])[n].reshape(-1, order="F")
                                  for n in range(5)]) for l in range(len(Ws))], axis=1)
    np.testing.assert_allclose(J, tr.residual_jacobians(th, d, widths, X, g, interior=False),
                               rtol=1e-12, atol=1e-13)


def test_adjoint_vs_finite_differences_of_intermediate():
    # g^{(l)}_{n,s} = ∂r_n/∂Z^{(l)}_{n,s}: perturb one entry of Z^{(l)} and re-run
    # the remaining layers (central differences).
    d, widths = 2, (4, 3, 1)
    th = _theta(d, widths, seed=9)
    Ws = ko.unpack_theta(th, d, widths)
    X = np.random.default_rng(8).uniform(size=(1, d))
    fp = ko.taylor_forward(Ws, X)
    zb = ko.taylor_adjoint(Ws, fp, ko.residual_seed(fp.S, "laplace", 0.0, True))
    lap_set = ko.operator_matrix(d, "laplace")

    def r_from(l, Z):
        T = ko.append_bias_row(ko.tanh_taylor(Z, lap_set))
        for k in range(l + 1, len(Ws)):
            Z = np.matmul(Ws[k][None], T)
            if k < len(Ws) - 1:
                T = ko.append_bias_row(ko.tanh_taylor(Z, lap_set))
        return -Z[0, 0, -1]

    h = 1e-6
    for l in range(len(Ws) - 1):
        for i in range(Ws[l].shape[0]):
            for s in range(fp.S):
                Zp = fp.Z[l].copy(); Zp[0, i, s] += h
                Zm = fp.Z[l].copy(); Zm[0, i, s] -= h
                fd = (r_from(l, Zp) - r_from(l, Zm)) / (2 * h)
                assert abs(fd - zb[l][0, i, s]) < 1e-6 * max(1, abs(fd)), (l, i, s)


@pytest.mark.parametrize("op", ["laplace", "heat"])
def test_loss_gradient_vs_autograd(op):
    import torch
    d, widths = 3, (5, 4, 1)
    kappa = 0.25 if op == "heat" else 0.0
    th = _theta(d, widths, seed=2)
    rng = np.random.default_rng(10)
    Xi, Xb = rng.uniform(size=(6, d)), rng.uniform(size=(4, d))
    f, g = rng.standard_normal(6), rng.standard_normal(4)
    cfg = ko.KfacConfig(d=d, widths=widths, op=op, kappa=kappa)
    cg = ko.curvature_and_gradient(cfg, ko.unpack_theta(th, d, widths), Xi, f, Xb, g)
    rf = tr.residual_fn(d, widths, op, kappa)
    tht = torch.as_tensor(th).clone().requires_grad_(True)
    Li = sum(rf(tht, torch.as_tensor(x), float(t), True) ** 2 for x, t in zip(Xi, f)) / (2 * 6)
    Lb = sum(rf(tht, torch.as_tensor(x), float(t), False) ** 2 for x, t in zip(Xb, g)) / (2 * 4)
    (gr,) = torch.autograd.grad(Li + Lb, tht)
    np.testing.assert_allclose(ko.pack_theta(cg["grads"]), gr.numpy(), rtol=1e-10, atol=1e-12)
    assert abs(cg["loss"][0] - float(Li + Lb)) < 1e-12 * max(1, float(Li + Lb))


# --------------------------------------------------------------------------
# Kronecker factors (Eq. 3, Eq. 7, Eq. 8)
# --------------------------------------------------------------------------
def test_single_point_boundary_kfac_is_exact_ggn_block():
    # N = 1 and S = 1: A ⊗ B equals the exact GGN block (Eq. 3 without the
    # expectation approximation), brute-forced from autograd Jacobians.
    d, widths = 3, (4, 3, 1)
    th = _theta(d, widths, seed=13)
    Ws = ko.unpack_theta(th, d, widths)
    X = np.random.default_rng(14).uniform(size=(1, d))
    fp = ko.taylor_forward(Ws, X, with_derivatives=False)
    zb = ko.taylor_adjoint(Ws, fp, ko.residual_seed(1, "laplace", 0.0, False))
    J = tr.residual_jacobians(th, d, widths, X, [0.0], interior=False)[0]
    off = 0
    for l in range(len(Ws)):
        A, B = ko.factors_expand(fp.T_in[l], zb[l])
        p = Ws[l].size
        block = np.outer(J[off:off + p], J[off:off + p])
        np.testing.assert_allclose(np.kron(A, B), block, rtol=1e-11, atol=1e-13)
        off += p


def test_exact_interior_block_vs_autograd():
    d, widths = 2, (4, 3, 1)
    th = _theta(d, widths, seed=15)
    Ws = ko.unpack_theta(th, d, widths)
    X = np.random.default_rng(16).uniform(size=(5, d))
    fp = ko.taylor_forward(Ws, X)
    zb = ko.taylor_adjoint(Ws, fp, ko.residual_seed(fp.S, "laplace", 0.0, True))
    J = tr.residual_jacobians(th, d, widths, X, np.zeros(5), interior=True)
    off = 0
    for l in range(len(Ws)):
        p = Ws[l].size
        G_ref = J[:, off:off + p].T @ J[:, off:off + p] / 5
        np.testing.assert_allclose(ko.exact_interior_block(fp.T_in[l], zb[l]), G_ref,
                                   rtol=1e-10, atol=1e-12)
        off += p


def test_full_ggn_vs_autograd():
    d, widths = 2, (3, 2, 1)
    th = _theta(d, widths, seed=17)
    rng = np.random.default_rng(18)
    Xi, Xb = rng.uniform(size=(4, d)), rng.uniform(size=(3, d))
    cfg = ko.KfacConfig(d=d, widths=widths)
    G = ko.full_ggn(cfg, ko.unpack_theta(th, d, widths), Xi, np.zeros(4), Xb, np.zeros(3))
    Ji = tr.residual_jacobians(th, d, widths, Xi, np.zeros(4), interior=True)
    Jb = tr.residual_jacobians(th, d, widths, Xb, np.zeros(3), interior=False)
    np.testing.assert_allclose(G, Ji.T @ Ji / 4 + Jb.T @ Jb / 3, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("variant", ["expand", "reduce"])
def test_factor_structure(variant):
    d, widths = 3, (6, 5, 1)
    th = _theta(d, widths, seed=19)
    rng = np.random.default_rng(20)
    N, Nb = 11, 7
    Xi, Xb = rng.uniform(size=(N, d)), rng.uniform(size=(Nb, d))
    cfg = ko.KfacConfig(d=d, widths=widths, variant=variant)
    cg = ko.curvature_and_gradient(cfg, ko.unpack_theta(th, d, widths), Xi, np.zeros(N), Xb, np.zeros(Nb))
    Ai, Bi, Ab, Bb = cg["factors"]
    S = d + 2
    for M in Ai + Bi + Ab + Bb:
        np.testing.assert_allclose(M, M.T, atol=1e-15)
        assert np.linalg.eigvalsh(M).min() >= -1e-12 * max(1.0, np.abs(M).max())
    # Layer-1 input factor in closed form.
    ones = np.ones((N, 1))
    if variant == "expand":
        A1 = np.block([[Xi.T @ Xi + N * np.eye(d), Xi.T @ ones], [ones.T @ Xi, np.array([[float(N)]])]]) / (N * S)
        assert abs(Ai[1][-1, -1] - 1.0 / S) < 1e-15          # bias entry 1/S
    else:
        abar = np.concatenate([Xi + 1.0, ones], axis=1) / S
        abar[:, -1] = 1.0 / S
        A1 = abar.T @ abar / N
    np.testing.assert_allclose(Ai[0], A1, rtol=1e-13, atol=1e-15)
    Xb1 = np.concatenate([Xb, np.ones((Nb, 1))], axis=1)
    np.testing.assert_allclose(Ab[0], Xb1.T @ Xb1 / Nb, rtol=1e-13)
    assert abs(Ab[1][-1, -1] - 1.0) < 1e-15                    # boundary bias entry 1
    # Last layer: g^{(L)} is the seed, so B^{(L)} = Σ_s c_s² (expand) or (Σ_s c_s)² (reduce).
    assert abs(Bi[-1][0, 0] - 1.0) < 1e-15 and abs(Bb[-1][0, 0] - 1.0) < 1e-15


def test_heat_last_layer_factor():
    d, widths = 5, (4, 1)
    th = _theta(d, widths, seed=1)
    rng = np.random.default_rng(2)
    Xi, Xb = rng.uniform(size=(3, d)), rng.uniform(size=(2, d))
    for variant, expect in (("expand", 1.0 + 0.25 ** 2), ("reduce", (1.0 - 0.25) ** 2)):
        cfg = ko.KfacConfig(d=d, widths=widths, op="heat", kappa=0.25, variant=variant)
        cg = ko.curvature_and_gradient(cfg, ko.unpack_theta(th, d, widths), Xi, np.zeros(3), Xb, np.zeros(2))
        assert abs(cg["factors"][1][-1][0, 0] - expect) < 1e-15


def test_reduce_equals_expand_for_one_column():
    rng = np.random.default_rng(3)
    T = rng.standard_normal((9, 5, 1))
    G = rng.standard_normal((9, 4, 1))
    for x, y in zip(ko.factors_expand(T, G), ko.factors_reduce(T, G)):
        np.testing.assert_allclose(x, y, rtol=1e-14)


def test_reduce_exact_when_shared_inputs_coincide():
    # If all S input columns of the single point are equal, the exact block
    # (Eq. 7) factorises as ā āᵀ ⊗ ḡ ḡᵀ, which is what KFAC-reduce returns.
    rng = np.random.default_rng(4)
    t = rng.standard_normal(5)
    T = np.repeat(t[None, :, None], 6, axis=2)
    G = rng.standard_normal((1, 3, 6))
    A, B = ko.factors_reduce(T, G)
    np.testing.assert_allclose(np.kron(A, B), ko.exact_interior_block(T, G), rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# Damped Kronecker-sum inverse (Sec. 3.4)
# --------------------------------------------------------------------------
def _spd(n, rng, rank=None):
    M = rng.standard_normal((n, rank or n))
    return M @ M.T / n


@pytest.mark.parametrize("damping_sqrt", [False, True])
def test_kron_sum_inverse_vs_dense_solve(damping_sqrt):
    rng = np.random.default_rng(30)
    na, nb, lam = 5, 4, 1e-3
    Ai, Ab = _spd(na, rng, 3), _spd(na, rng, 2)
    Bi, Bb = _spd(nb, rng, 2), _spd(nb, rng, 4)
    G = rng.standard_normal((nb, na))
    D = ko.kron_sum_inverse_apply(Ai, Bi, Ab, Bb, G, lam, damping_sqrt)
    e = math.sqrt(lam) if damping_sqrt else lam
    K = np.kron(Ai + e * np.eye(na), Bi + e * np.eye(nb)) + np.kron(Ab + e * np.eye(na), Bb + e * np.eye(nb))
    ref = -np.linalg.solve(K, G.reshape(-1, order="F")).reshape(nb, na, order="F")
    np.testing.assert_allclose(D, ref, rtol=1e-9, atol=1e-12)


def test_kron_sum_inverse_large_damping_limit():
    rng = np.random.default_rng(31)
    Ai, Ab, Bi, Bb = _spd(4, rng), _spd(4, rng), _spd(3, rng), _spd(3, rng)
    G = rng.standard_normal((3, 4))
    lam = 1e7
    D = ko.kron_sum_inverse_apply(Ai, Bi, Ab, Bb, G, lam)
    np.testing.assert_allclose(D, -G / (2 * lam * lam), rtol=1e-5)


def test_generalized_eig_diagonalises():
    rng = np.random.default_rng(32)
    P, Q = _spd(6, rng) + np.eye(6), _spd(6, rng, 2)
    V, w = ko.generalized_eig(P, Q)
    np.testing.assert_allclose(V.T @ P @ V, np.eye(6), atol=1e-12)
    np.testing.assert_allclose(V.T @ Q @ V, np.diag(w), atol=1e-12)


# --------------------------------------------------------------------------
# One KFAC step (Algorithm 1 with fixed learning rate)
# --------------------------------------------------------------------------
def test_kfac_step_matches_dense_preconditioning():
    d, widths = 2, (4, 3, 1)
    th = _theta(d, widths, seed=40)
    prob = si.PROBLEMS["poisson2d_sin"]
    Xi, f, Xb, g = si.make_batch(prob, 8, 6, seed=3)
    cfg = ko.KfacConfig(d=d, widths=widths, lam=1e-2, lr=0.5, momentum=0.3, beta=0.0)
    st = ko.init_state(cfg)
    res = ko.kfac_step(cfg, st, th, Xi, f, Xb, g)
    Ws = ko.unpack_theta(th, d, widths)
    # Dense per-layer Kronecker-sum system assembled from the fresh factors.
    Ai, Bi, Ab, Bb = res.factors
    for l, W in enumerate(Ws):
        na, nb = Ai[l].shape[0], Bi[l].shape[0]
        K = (np.kron(Ai[l] + cfg.lam * np.eye(na), Bi[l] + cfg.lam * np.eye(nb))
             + np.kron(Ab[l] + cfg.lam * np.eye(na), Bb[l] + cfg.lam * np.eye(nb)))
        ref = -np.linalg.solve(K, res.grads[l].reshape(-1, order="F"))
        np.testing.assert_allclose(res.direction[l].reshape(-1, order="F"), ref, rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(res.theta_new, th + cfg.lr * ko.pack_theta(res.direction), rtol=1e-14)
    # Second step: momentum on the previous update, δ_1 = lr (μ δ_0 + Δ_1).
    prev = [u.copy() for u in res.update]
    res2 = ko.kfac_step(cfg, st, res.theta_new, Xi, f, Xb, g)
    for l in range(len(Ws)):
        np.testing.assert_allclose(res2.update[l], cfg.lr * (cfg.momentum * prev[l] + res2.direction[l]),
                                   rtol=1e-14)


def test_ema_and_identity_init():
    d, widths = 2, (3, 1)
    th = _theta(d, widths, seed=41)
    prob = si.PROBLEMS["poisson2d_sin"]
    Xi, f, Xb, g = si.make_batch(prob, 5, 4, seed=4)
    cfg = ko.KfacConfig(d=d, widths=widths, beta=0.75, init_identity=True)
    st = ko.init_state(cfg)
    res = ko.kfac_step(cfg, st, th, Xi, f, Xb, g)
    cg = ko.curvature_and_gradient(cfg, ko.unpack_theta(th, d, widths), Xi, f, Xb, g)
    for l in range(2):
        n = cg["factors"][0][l].shape[0]
        np.testing.assert_allclose(st.A_int[l], 0.75 * np.eye(n) + 0.25 * cg["factors"][0][l], rtol=1e-14)


def test_kfac_direction_is_descent_poisson2d():
    # The damped Kronecker sum is positive definite, so Δ is a descent
    # direction: gᵀΔ < 0 and a short step along Δ lowers the loss (Eq. 1).
    wl = si.WORKLOADS["poisson2d_small"]
    prob = wl.prob
    th = si.xavier_theta(prob.d, wl.widths, 0)
    Xi, f, Xb, g = si.make_batch(prob, 200, 60, seed=0)
    cfg = ko.KfacConfig(d=prob.d, widths=wl.widths, lam=1e-3, lr=2.0 ** -8, beta=0.0)
    st = ko.init_state(cfg)
    res = ko.kfac_step(cfg, st, th, Xi, f, Xb, g)
    assert ko.pack_theta(res.grads) @ ko.pack_theta(res.direction) < 0
    nxt = ko.curvature_and_gradient(cfg, ko.unpack_theta(res.theta_new, prob.d, wl.widths), Xi, f, Xb, g)
    assert nxt["loss"][0] < res.loss[0]


# --------------------------------------------------------------------------
# Log-grid line search (Sec. 3.4; App. B)
# --------------------------------------------------------------------------
def _linear_loss_closed_form(w, b, Xi, f, Xb, g):
    # u = wᵀx + b has Δu = 0, so the Poisson residuals are r_Ω = -f and
    # r_∂ = wᵀx + b - g; Eq. 1 with 1/(2N) on each term.
    li = (f ** 2).sum() / (2 * f.size)
    lb = ((Xb @ w + b - g) ** 2).sum() / (2 * g.size)
    return li + lb


def test_line_search_grid_argmin_closed_form():
    # A single linear layer: L(θ + αδ̂) is a quadratic in α known in closed
    # form.  With δ̂ = 0.37 × (the exact minimiser − θ) the minimum over α is at
    # 1/0.37 > 1, so the grid's answer is α = 1; with 3.1 × it sits at
    # 1/3.1 and the grid picks whichever of 2^-1, 2^-2 is closer in loss.
    d = 3
    prob = si.poisson_cos_problem(d)
    Xi, f, Xb, g = si.make_batch(prob, 20, 15, seed=11)
    cfg = ko.KfacConfig(d=d, widths=(1,), line_search=True)
    th = np.array([0.3, -0.2, 0.5, 0.1])                 # (w_1, w_2, w_3, b)
    Aug = np.hstack([Xb, np.ones((Xb.shape[0], 1))])
    opt = np.linalg.lstsq(Aug, g, rcond=None)[0]
    for scale in (0.37, 3.1):
        dhat = scale * (opt - th)
        alpha, losses = ko.line_search(cfg, th, dhat, Xi, f, Xb, g)
        ref = [_linear_loss_closed_form((th + a * dhat)[:3], (th + a * dhat)[3], Xi, f, Xb, g)
               for a in ko.LINE_SEARCH_GRID]
        np.testing.assert_allclose(losses[:, 0], ref, rtol=1e-12)
        assert alpha == ko.LINE_SEARCH_GRID[int(np.argmin(ref))]
    assert len(ko.LINE_SEARCH_GRID) == 31
    assert ko.LINE_SEARCH_GRID[0] == 1.0 and ko.LINE_SEARCH_GRID[-1] == 2.0 ** -30


def test_line_search_ties_and_nonfinite():
    d = 2
    prob = si.PROBLEMS["poisson2d_sin"]
    Xi, f, Xb, g = si.make_batch(prob, 10, 8, seed=12)
    cfg = ko.KfacConfig(d=d, widths=(1,), line_search=True)
    th = np.array([0.1, 0.2, 0.3])
    # δ̂ = 0: every trial has the same loss, the larger α is kept.
    alpha, losses = ko.line_search(cfg, th, np.zeros(3), Xi, f, Xb, g)
    assert alpha == 1.0 and np.all(losses[:, 0] == losses[0, 0])
    # A huge δ̂ overflows the large-α trials; they never win.
    with np.errstate(over="ignore", invalid="ignore"):
        alpha, losses = ko.line_search(cfg, th, np.full(3, 1e160), Xi, f, Xb, g)
    assert not np.isfinite(losses[0, 0])
    assert np.isfinite(losses[-1, 0]) and alpha == 2.0 ** -30


def test_kfac_step_with_line_search_descends():
    # δ̂ is a descent direction (the damped curvature is positive definite),
    # so the grid minimum is below L(θ) and θ_{t+1} = θ_t + α* δ̂ attains it.
    wl = si.WORKLOADS["poisson2d_small"]
    prob = wl.prob
    th = si.xavier_theta(prob.d, wl.widths, 0)
    Xi, f, Xb, g = si.make_batch(prob, 100, 40, seed=1)
    cfg = ko.KfacConfig(d=prob.d, widths=wl.widths, lam=1e-3, momentum=0.5, line_search=True)
    st = ko.init_state(cfg)
    for step in range(2):
        res = ko.kfac_step(cfg, st, th, Xi, f, Xb, g)
        losses = res.extras["line_search_losses"]
        k = int(np.argmin(losses[:, 0]))
        assert res.extras["alpha"] == 2.0 ** -k
        after = ko.curvature_and_gradient(cfg, ko.unpack_theta(res.theta_new, prob.d, wl.widths),
                                          Xi, f, Xb, g)["loss"]
        np.testing.assert_allclose(after, losses[k], rtol=1e-12)
        assert after[0] < res.loss[0]
        th = res.theta_new


# --------------------------------------------------------------------------
# KFAC*: automatic learning rate and momentum (Sec. 3.4)
# --------------------------------------------------------------------------
def test_gramian_products_vs_full_ggn():
    d, widths = 2, (4, 3, 1)
    th = _theta(d, widths, seed=50)
    prob = si.PROBLEMS["poisson2d_sin"]
    Xi, f, Xb, g = si.make_batch(prob, 6, 5, seed=13)
    cfg = ko.KfacConfig(d=d, widths=widths)
    Ws = ko.unpack_theta(th, d, widths)
    G = ko.full_ggn(cfg, Ws, Xi, f, Xb, g)
    cg = ko.curvature_and_gradient(cfg, Ws, Xi, f, Xb, g)
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal(th.size), rng.standard_normal(th.size)
    ja = ko.residual_jvp(cg, ko.unpack_theta(a, d, widths))
    jb = ko.residual_jvp(cg, ko.unpack_theta(b, d, widths))
    np.testing.assert_allclose(ko.gramian_bilinear(ja, jb), a @ G @ b, rtol=1e-11)
    # the residual JVP is the directional derivative of the residuals
    h = 1e-6
    rp = ko.curvature_and_gradient(cfg, ko.unpack_theta(th + h * a, d, widths), Xi, f, Xb, g)
    rm = ko.curvature_and_gradient(cfg, ko.unpack_theta(th - h * a, d, widths), Xi, f, Xb, g)
    np.testing.assert_allclose(ja[0], (rp["r_i"] - rm["r_i"]) / (2 * h), rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(ja[1], (rp["r_b"] - rm["r_b"]) / (2 * h), rtol=1e-6, atol=1e-8)


def test_kfac_star_minimises_quadratic_model():
    d, widths = 2, (5, 4, 1)
    th = _theta(d, widths, seed=51)
    prob = si.PROBLEMS["poisson2d_sin"]
    Xi, f, Xb, g = si.make_batch(prob, 8, 6, seed=14)
    cfg = ko.KfacConfig(d=d, widths=widths, lam=1e-2, kfac_star=True)
    st = ko.init_state(cfg)
    res1 = ko.kfac_step(cfg, st, th, Xi, f, Xb, g)
    assert res1.extras["mu"] == 0.0                     # first step: α only
    res2 = ko.kfac_step(cfg, st, res1.theta_new, Xi, f, Xb, g)
    Ws = ko.unpack_theta(res1.theta_new, d, widths)
    G = ko.full_ggn(cfg, Ws, Xi, f, Xb, g) + cfg.lam * np.eye(th.size)
    gr = ko.pack_theta(res2.grads)
    Dl, dl = ko.pack_theta(res2.direction), ko.pack_theta(res1.update)

    def model(a, m):
        v = a * Dl + m * dl
        return v @ gr + 0.5 * v @ G @ v

    a, m = res2.extras["alpha"], res2.extras["mu"]
    np.testing.assert_allclose(ko.pack_theta(res2.update), a * Dl + m * dl, rtol=1e-14)
    best = model(a, m)
    for da, dm in ((1e-3, 0), (-1e-3, 0), (0, 1e-3), (0, -1e-3)):
        assert model(a + da * abs(a), m + dm * max(abs(m), 1.0)) > best
    # stationarity of the model in (α, μ) with the dense Gramian
    np.testing.assert_allclose([Dl @ (gr + G @ (a * Dl + m * dl)), dl @ (gr + G @ (a * Dl + m * dl))],
                               [0.0, 0.0], atol=1e-9 * abs(Dl @ gr))


# --------------------------------------------------------------------------
# General second-order operator Σ c_ij ∂²_ij (App. C.3)
# --------------------------------------------------------------------------
def _sym(d, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((d, d))
    return 0.5 * (M + M.T)       # indefinite in general


def test_general_operator_forward_vs_autograd():
    d, widths = 4, (7, 5, 1)
    th = _theta(d, widths, seed=60)
    X = np.random.default_rng(61).random((6, d))
    C = _sym(d, 62)
    Ws = ko.unpack_theta(th, d, widths)
    u, g, cu = ko.forward_laplacian(Ws, X, "general", C)
    np.testing.assert_allclose(cu, tr.operator_value(th, d, widths, X, C), rtol=1e-11, atol=1e-12)
    # c = I reproduces the Laplacian column, c = diag(0, 1, ..) the heat operator's
    _, _, lap = ko.forward_laplacian(Ws, X, "laplace")
    np.testing.assert_allclose(ko.forward_laplacian(Ws, X, "general", np.eye(d))[2], lap, rtol=1e-13)
    _, _, plap = ko.forward_laplacian(Ws, X, "heat")
    np.testing.assert_allclose(ko.forward_laplacian(Ws, X, "general", np.diag([0.0] + [1.0] * (d - 1)))[2],
                               plap, rtol=1e-13)


def test_general_operator_jacobian_and_gradient_vs_autograd():
    d, widths = 3, (6, 4, 1)
    th = _theta(d, widths, seed=63)
    rng = np.random.default_rng(64)
    Xi, f = rng.random((5, d)), rng.standard_normal(5)
    Xb, g = rng.random((4, d)), rng.standard_normal(4)
    C = _sym(d, 65)
    cfg = ko.KfacConfig(d=d, widths=widths, op="general", op_coef=C)
    cg = ko.curvature_and_gradient(cfg, ko.unpack_theta(th, d, widths), Xi, f, Xb, g)
    J = tr.residual_jacobians(th, d, widths, Xi, f, op="general", coef=C)
    Jo = np.stack([np.concatenate([ko.weight_jacobian(cg["zb_i"][l][n:n + 1], cg["fp_i"].T_in[l][n:n + 1])[0]
                                   .reshape(-1, order="F") for l in range(len(widths))]) for n in range(5)])
    np.testing.assert_allclose(Jo, J, rtol=1e-10, atol=1e-12)
    Jb = tr.residual_jacobians(th, d, widths, Xb, g, interior=False)
    grad = J.T @ cg["r_i"] / 5 + Jb.T @ cg["r_b"] / 4
    np.testing.assert_allclose(ko.pack_theta(cg["grads"]), grad, rtol=1e-10, atol=1e-12)
