"""Reverse mode through the forward Laplacian (kfac_pinn_forward_laplacian_backward
and the ForwardLaplacian autograd.Function) against double autograd and
central finite differences (h = 1e-6, FP64).

phi = Σ_n a_n u_n + b_nᵀ∇u_n + c_n Δu_n with random weights, so every output
channel is seeded.
"""
import numpy as np
import pytest
import torch

from synth import inputs as si
from tests import torch_ref as tr

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _theta(d, widths, seed):
    th = si.xavier_theta(d, widths, seed)
    rng = np.random.default_rng(seed + 1)
    return th + 0.05 * rng.standard_normal(th.size)   # non-zero biases


def double_autograd(theta, d, widths, X, a, b, c, lap_coords):
    """phi and its gradients by autograd of autograd (CPU, float64)."""
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    net = tr.mlp_from_flat(th, d, widths)
    phi = 0.0
    for n in range(X.shape[0]):
        x = Xt[n]
        u = net(x)
        (g,) = torch.autograd.grad(u, x, create_graph=True)
        lap = 0.0
        for i in lap_coords:
            (gi,) = torch.autograd.grad(g[i], x, create_graph=True)
            lap = lap + gi[i]
        phi = phi + a[n] * u + (torch.tensor(b[n]) * g).sum() + c[n] * lap
    dth, dX = torch.autograd.grad(phi, (th, Xt))
    return float(phi.detach()), dth.numpy(), dX.numpy()


def _opt(d, widths, op="laplace", kappa=0.0, **kw):
    from paper_2405_15603_gb300.api import KfacPinn
    return KfacPinn(d, widths, device=DEV, op=op, kappa=kappa, **kw)


CASES = [
    ("poisson3d_3-16-12-1", 3, (16, 12, 1), "laplace", list(range(3))),
    ("heat4d_5-16-16-8-1", 5, (16, 16, 8, 1), "heat", list(range(1, 5))),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_backward_vs_double_autograd(case):
    _, d, widths, op, lap_coords = case
    rng = np.random.default_rng(7)
    N = 24
    X = rng.random((N, d))
    a, b, c = rng.standard_normal(N), rng.standard_normal((N, d)), rng.standard_normal(N)
    th = _theta(d, widths, 3)
    phi_ref, dth_ref, dX_ref = double_autograd(th, d, widths, X, a, b, c, lap_coords)
    opt = _opt(d, widths, op=op, kappa=0.25, max_n_int=N, max_n_bdy=1)
    theta = torch.tensor(th, device=DEV)
    dth, dX = opt.forward_laplacian_backward(theta, X, a, b, c, need_dX=True)
    torch.cuda.synchronize()
    assert rel(dth.cpu(), dth_ref) < 1e-11
    assert rel(dX.cpu(), dX_ref) < 1e-11
    assert opt.sync_status() == "KFAC_OK"


def test_backward_vs_central_differences():
    d, widths = 4, (24, 24, 1)
    rng = np.random.default_rng(8)
    N = 200
    X = rng.random((N, d))
    a, b, c = rng.standard_normal(N), rng.standard_normal((N, d)), rng.standard_normal(N)
    th = _theta(d, widths, 5)
    opt = _opt(d, widths, max_n_int=N, max_n_bdy=1)
    A, B, Cc = (torch.tensor(v, device=DEV) for v in (a, b, c))

    def phi(t):
        u, g, lap = opt.forward_laplacian(t, X)
        return float((A * u).sum() + (B * g).sum() + (Cc * lap).sum())

    theta = torch.tensor(th, device=DEV)
    dth, _ = opt.forward_laplacian_backward(theta, X, a, b, c)
    h = 1e-6
    for k in range(3):
        v = torch.tensor(rng.standard_normal(th.size), device=DEV)
        fd = (phi(theta + h * v) - phi(theta - h * v)) / (2 * h)
        an = float(dth @ v)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1.0), (fd, an)


def test_autograd_function_and_chunking():
    from paper_2405_15603_gb300.api import ForwardLaplacian
    d, widths = 3, (20, 10, 1)
    rng = np.random.default_rng(9)
    N = 150
    X = rng.random((N, d))
    th = _theta(d, widths, 11)
    small = _opt(d, widths, max_n_int=64, max_n_bdy=1)     # three chunks of the pass
    big = _opt(d, widths, max_n_int=N, max_n_bdy=1)
    a = torch.tensor(rng.standard_normal(N), device=DEV)
    c = torch.tensor(rng.standard_normal(N), device=DEV)
    grads = []
    for opt in (small, big):
        theta = torch.tensor(th, device=DEV, requires_grad=True)
        Xt = torch.tensor(X, device=DEV, requires_grad=True)
        u, g, lap = ForwardLaplacian.apply(theta, Xt, opt)
        phi = (a * u).sum() + g.pow(2).sum() + (c * lap).sum()
        grads.append([t.detach().cpu().numpy() for t in torch.autograd.grad(phi, (theta, Xt))])
    assert rel(grads[0][0], grads[1][0]) < 1e-13
    assert rel(grads[0][1], grads[1][1]) < 1e-13
    # against double autograd (b = 2 ∇u at the current parameters)
    ref_u = tr.value_grad_lap(th, d, widths, X)
    phi_ref, dth_ref, dX_ref = double_autograd(th, d, widths, X, a.cpu().numpy(), 2 * ref_u[1],
                                               c.cpu().numpy(), list(range(d)))
    assert rel(grads[1][0], dth_ref) < 1e-11
    assert rel(grads[1][1], dX_ref) < 1e-11


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_split", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_backward_mixed_precision(case, precision):
    # Reduced precisions against double autograd at their gradient bounds:
    # BF16 tangent and adjoint rows 2e-2, split-BF16 everywhere and FP32 1e-4
    _, d, widths, op, lap_coords = case
    rng = np.random.default_rng(17)
    N = 96
    X = rng.random((N, d))
    a, b, c = rng.standard_normal(N), rng.standard_normal((N, d)), rng.standard_normal(N)
    th = _theta(d, widths, 19)
    phi_ref, dth_ref, dX_ref = double_autograd(th, d, widths, X, a, b, c, lap_coords)
    opt = _opt(d, widths, op=op, kappa=0.25, precision=precision, max_n_int=64, max_n_bdy=1)
    dth, dX = opt.forward_laplacian_backward(torch.tensor(th, device=DEV), X, a, b, c, need_dX=True)
    torch.cuda.synchronize()
    tol = 2e-2 if precision == "mixed_bf16" else 1e-4
    assert rel(dth.cpu(), dth_ref) < tol
    assert rel(dX.cpu(), dX_ref) < tol
    assert opt.sync_status() == "KFAC_OK"


def test_backward_mixed_general_operator_vs_fp64():
    d, widths, N = 5, (64, 32, 1), 80
    rng = np.random.default_rng(21)
    M = rng.standard_normal((d, d))
    C = 0.5 * (M + M.T)
    X = rng.random((N, d))
    a, b, c = rng.standard_normal(N), rng.standard_normal((N, d)), rng.standard_normal(N)
    th = torch.tensor(_theta(d, widths, 23), device=DEV)
    out = {}
    for prec in ("fp64", "mixed_bf16"):
        opt = _opt(d, widths, op="general", precision=prec, op_coef=C, max_n_int=N, max_n_bdy=1)
        out[prec] = [t.cpu().numpy() for t in opt.forward_laplacian_backward(th, X, a, b, c, need_dX=True)]
    assert rel(out["mixed_bf16"][0], out["fp64"][0]) < 2e-2
    assert rel(out["mixed_bf16"][1], out["fp64"][1]) < 2e-2


def test_store_forward_matches_recompute():
    # Reverse mode reusing the stored activations of the forward pass gives the
    # same gradient as recomputing them, with fewer kernels; a step in between
    # discards the stored pass.
    from paper_2405_15603_gb300.api import ForwardLaplacian
    d, widths = 4, (32, 24, 1)
    rng = np.random.default_rng(12)
    N = 120
    X = torch.tensor(rng.random((N, d)), device=DEV)
    th = torch.tensor(_theta(d, widths, 13), device=DEV)
    a = torch.tensor(rng.standard_normal(N), device=DEV)
    out = {}
    for store in (False, True):
        opt = _opt(d, widths, max_n_int=N, max_n_bdy=4)
        opt.set_store_forward(store)
        theta = th.clone().requires_grad_(True)
        u, g, lap = ForwardLaplacian.apply(theta, X, opt)
        phi = (a * lap).sum() + u.sum() + g.sum()
        n0 = opt.launch_count()
        (gr,) = torch.autograd.grad(phi, theta)
        torch.cuda.synchronize()
        out[store] = (gr.cpu().numpy(), opt.launch_count() - n0)
    assert np.array_equal(out[True][0], out[False][0])
    assert out[True][1] < out[False][1]
    # a step in between discards the stored activations: still the right gradient
    opt = _opt(d, widths, max_n_int=N, max_n_bdy=4)
    opt.set_store_forward(True)
    theta = th.clone().requires_grad_(True)
    u, g, lap = ForwardLaplacian.apply(theta, X, opt)
    prob = si.poisson_cos_problem(d)
    Xi, f, Xb, gb = si.make_batch(prob, N, 4, seed=1)
    opt.step(th.clone(), Xi, f, Xb, gb)
    (gr,) = torch.autograd.grad((a * lap).sum() + u.sum() + g.sum(), theta)
    assert np.array_equal(gr.cpu().numpy(), out[False][0])
