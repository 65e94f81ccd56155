"""Pins of the oracle's general-residual KFAC (Sec. 3.3, Eq. 9-10): a residual
with M outputs that is quadratic in the network's Taylor outputs, with the
criterion l(r) = 1/2 r^T W r (Lambda = W).

Independent routes: torch autograd (residuals, their Jacobians, the loss
gradient and the exact GGN of Eq. 2 with Lambda), closed forms (the last
layer's B factor from the residual's own Jacobian), the KFLR rewrite of B
with W = L L^T (a second way to form Eq. 10), and the reduction to the
Poisson residual of Eq. 1."""
import numpy as np
import pytest

from oracle import kfac_oracle as ko
from synth import inputs as si
from tests import torch_ref as tr


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _case(M=2, seed=0, d=3, widths=(6, 5, 1), N=5, Nb=3, quad=True, op="laplace"):
    rng = np.random.default_rng(seed)
    S = d + 2
    b = rng.standard_normal((M, S))
    Q = None
    if quad:
        Q = rng.standard_normal((M, S, S))
        Q = 0.5 * (Q + np.transpose(Q, (0, 2, 1)))
    A = rng.standard_normal((M, M))
    W = A @ A.T + M * np.eye(M)
    th = si.xavier_theta(d, widths, seed)
    th = th + 0.05 * rng.standard_normal(th.size)      # non-zero biases
    Xi = rng.random((N, d))
    F = rng.standard_normal((N, M))
    Xb = rng.random((Nb, d))
    g = rng.standard_normal(Nb)
    res = ko.QuadraticResidual(b=b, Q=Q, W=W)
    cfg = ko.KfacConfig(d=d, widths=widths, op=op, residual=res, lam=1e-2)
    return cfg, th, Xi, F, Xb, g


@pytest.mark.parametrize("quad", [False, True])
def test_residual_and_gradient_vs_autograd(quad):
    cfg, th, Xi, F, Xb, g = _case(quad=quad)
    res = cfg.residual
    Ws = ko.unpack_theta(th, cfg.d, cfg.widths)
    cg = ko.curvature_and_gradient(cfg, Ws, Xi, F, Xb, g)
    r_ref, J_ref = tr.quadratic_residual_rows(th, cfg.d, cfg.widths, Xi, F, res.b, res.Q)
    assert rel(cg["r_i"], r_ref) < 1e-12
    # loss and its gradient: (1/N) sum_n J_n^T W r_n + boundary (Eq. 1)
    W = res.weight()
    N = Xi.shape[0]
    li = np.einsum("nk,kj,nj->", r_ref, W, r_ref) / (2 * N)
    Jb = tr.residual_jacobians(th, cfg.d, cfg.widths, Xb, g, interior=False)
    rb = tr.residuals(th, cfg.d, cfg.widths, Xb, g, interior=False)
    grad_ref = np.einsum("nkD,kj,nj->D", J_ref, W, r_ref) / N + Jb.T @ rb / Xb.shape[0]
    assert abs(cg["loss"][1] - li) <= 1e-12 * abs(li)
    assert rel(ko.pack_theta(cg["grads"]), grad_ref) < 1e-11


def test_full_ggn_vs_autograd():
    # Eq. 2 with Lambda = W: G = (1/N) sum_n J_n^T W J_n + (1/N_b) sum J_b^T J_b
    cfg, th, Xi, F, Xb, g = _case()
    Ws = ko.unpack_theta(th, cfg.d, cfg.widths)
    G = ko.full_ggn(cfg, Ws, Xi, F, Xb, g)
    _, J_ref = tr.quadratic_residual_rows(th, cfg.d, cfg.widths, Xi, F, cfg.residual.b, cfg.residual.Q)
    Jb = tr.residual_jacobians(th, cfg.d, cfg.widths, Xb, g, interior=False)
    G_ref = np.einsum("nkD,kj,njE->DE", J_ref, cfg.residual.weight(), J_ref) / Xi.shape[0] + Jb.T @ Jb / Xb.shape[0]
    assert rel(G, G_ref) < 1e-11


def test_last_layer_b_factor_closed_form():
    # h_L = 1: J_{Z^(L)_{n,s}} r_n is column s of the residual's own Jacobian, so
    # B^(L) = (1/N) sum_{n,s} J[n,:,s]^T W J[n,:,s] (Eq. 10) needs no adjoint pass
    cfg, th, Xi, F, Xb, g = _case(M=3, seed=4)
    Ws = ko.unpack_theta(th, cfg.d, cfg.widths)
    cg = ko.curvature_and_gradient(cfg, Ws, Xi, F, Xb, g)
    z = cg["fp_i"].Z[-1][:, 0, :]
    J = ko.quadratic_residual_jacobian(cfg.residual, z)
    W = cfg.residual.weight()
    BL = np.einsum("nks,kj,njs->", J, W, J) / Xi.shape[0]
    assert abs(cg["factors"][1][-1][0, 0] - BL) <= 1e-12 * abs(BL)


def test_kflr_form_of_b_with_cholesky_of_w():
    # W = L L^T: B = (1/N) sum_{n,s,m} g_m g_m^T with g_m = sum_k L[k,m] g_k
    # (the outer-product rewrite of Sec. 3.3), the route of the CUDA path
    cfg, th, Xi, F, Xb, g = _case(M=3, seed=5)
    Ws = ko.unpack_theta(th, cfg.d, cfg.widths)
    cg = ko.curvature_and_gradient(cfg, Ws, Xi, F, Xb, g)
    Lc = np.linalg.cholesky(cfg.residual.weight())
    N = Xi.shape[0]
    for l in range(len(cfg.widths)):
        Gk = [np.transpose(zb[l], (0, 2, 1)).reshape(-1, zb[l].shape[1]) for zb in cg["zb_i_k"]]
        B = sum((sum(Lc[k, m] * Gk[k] for k in range(len(Gk)))).T @ (sum(Lc[k, m] * Gk[k] for k in range(len(Gk))))
                for m in range(len(Gk))) / N
        assert rel(cg["factors"][1][l], B) < 1e-12


def test_reduces_to_the_poisson_residual():
    # M = 1, r = -Laplacian(u) - f, W = 1: exactly the residual of Eq. 1
    d, widths = 3, (6, 5, 1)
    prob = si.poisson_cos_problem(d)
    th = si.xavier_theta(d, widths, 3)
    Xi, f, Xb, g = si.make_batch(prob, 7, 4, seed=1)
    b = np.zeros((1, d + 2))
    b[0, -1] = -1.0
    plain = ko.KfacConfig(d=d, widths=widths, lam=1e-2)
    gen = ko.KfacConfig(d=d, widths=widths, lam=1e-2, residual=ko.QuadraticResidual(b=b))
    Ws = ko.unpack_theta(th, d, widths)
    a = ko.curvature_and_gradient(plain, Ws, Xi, f, Xb, g)
    c = ko.curvature_and_gradient(gen, Ws, Xi, f[:, None], Xb, g)
    assert rel(ko.pack_theta(c["grads"]), ko.pack_theta(a["grads"])) < 1e-14
    for fa, fc in zip(a["factors"], c["factors"]):
        for x, y in zip(fa, fc):
            assert rel(y, x) < 1e-14
    np.testing.assert_allclose(c["loss"], a["loss"], rtol=1e-14)


def test_heat_operator_with_first_order_terms():
    # a convection term b_i du/dx_i next to the heat operator's second-order column
    cfg, th, Xi, F, Xb, g = _case(M=1, seed=6, d=4, quad=False, op="heat")
    Ws = ko.unpack_theta(th, cfg.d, cfg.widths)
    cg = ko.curvature_and_gradient(cfg, Ws, Xi, F, Xb, g)
    r_ref, _ = tr.quadratic_residual_rows(th, cfg.d, cfg.widths, Xi, F, cfg.residual.b, op="heat")
    assert rel(cg["r_i"], r_ref) < 1e-12


def test_kfac_star_with_general_residual_minimises_the_model():
    # (alpha*, mu*) of the quadratic model with the exact damped GGN (Eq. 2 with
    # Lambda = W) built densely from the autograd Jacobians
    cfg, th, Xi, F, Xb, g = _case(seed=7)
    cfg.kfac_star = True
    st = ko.init_state(cfg)
    res0 = ko.kfac_step(cfg, st, th, Xi, F, Xb, g)
    res1 = ko.kfac_step(cfg, st, res0.theta_new, Xi, F, Xb, g)
    Ws = ko.unpack_theta(res0.theta_new, cfg.d, cfg.widths)
    G = ko.full_ggn(cfg, Ws, Xi, F, Xb, g) + cfg.lam * np.eye(res0.theta_new.size)
    D = ko.pack_theta(res1.direction)
    dp = ko.pack_theta(res0.update)
    grad = ko.pack_theta(res1.grads)
    A = np.array([[D @ G @ D, D @ G @ dp], [D @ G @ dp, dp @ G @ dp]])
    alpha, mu = -np.linalg.solve(A, [D @ grad, dp @ grad])
    assert abs(res1.extras["alpha"] - alpha) <= 1e-9 * abs(alpha)
    assert abs(res1.extras["mu"] - mu) <= 1e-9 * max(abs(mu), 1e-3)
