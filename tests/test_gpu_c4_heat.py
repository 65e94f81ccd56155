"""The (4+1)-d heat workload (5 -> 128 -> 128 -> 64 -> 1, 4000 interior and
1000 initial/boundary points, kappa = 1/4) in the precision it is specified
in, FP32, against the FP64 oracle; and its reverse mode, the hand-written
adjoint of the Taylor pass behind torch.autograd.Function, at the full point
count in FP32 and FP64.

FP32 bounds: one SIMT FP32 operation rounds to 2^-24 relative; the Taylor
pass chains a few hundred of them per output and the Grams sum up to
S N = 28,000 rows in FP32 chunks of at most a few hundred rows, combined in
FP64, so forward outputs, loss, gradient and factors land near 1e-6 and are
held to the reduced-precision bounds (1e-4; the update 1e-3, which the damped
inverse's ~330-fold amplification of factor errors on this problem leaves
well inside).  Reverse mode: FP64 against central differences (h = 1e-6) and
double autograd; FP32 against FP64 to 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import kfac_oracle as ko
from synth import inputs as si
from tests import torch_ref as tr

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
WL = si.WORKLOADS["heat4d"]
PROB, WIDTHS = WL.prob, WL.widths


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _opt(precision, N, Nb, **kw):
    from paper_2405_15603_gb300.api import KfacPinn
    return KfacPinn(PROB.d, WIDTHS, device=DEV, precision=precision, op=PROB.op, kappa=PROB.kappa,
                    max_n_int=N, max_n_bdy=Nb, **kw)


@pytest.mark.parametrize("variant", ["expand", "reduce"])
def test_heat_step_fp32_vs_oracle(variant):
    N, Nb = WL.n_int, WL.n_bdy
    th = si.xavier_theta(PROB.d, WIDTHS, 0)
    Xi, f, Xb, g = si.make_batch(PROB, N, Nb, seed=0)
    kw = dict(lam=1e-3, lr=0.1, beta=0.0, variant=variant)
    cfg = ko.KfacConfig(d=PROB.d, widths=WIDTHS, op=PROB.op, kappa=PROB.kappa, **kw)
    ref = ko.kfac_step(cfg, ko.init_state(cfg), th, Xi, f, Xb, g)
    opt = _opt("fp32", N, Nb, **kw)
    theta = torch.tensor(th, device=DEV)
    u, gu, lap = (t.cpu().numpy() for t in opt.forward_laplacian(theta, Xi))
    ru, rg, rl = ko.forward_laplacian(ko.unpack_theta(th, PROB.d, WIDTHS), Xi, PROB.op)
    assert rel(u, ru) < 1e-5 and rel(gu, rg) < 1e-5 and rel(lap, rl) < 1e-5
    loss = opt.step(theta, Xi, f, Xb, g).cpu().numpy()
    assert opt.sync_status() == "KFAC_OK"
    assert rel(loss, np.array(ref.loss)) < 1e-5
    assert rel(opt.gradient().cpu(), ko.pack_theta(ref.grads)) < 1e-4
    for which, refs in zip(("A_int", "B_int", "A_bdy", "B_bdy"), ref.factors):
        for l in range(len(WIDTHS)):
            assert rel(opt.get_factor(l + 1, which).cpu(), refs[l]) < 1e-4, (which, l)
    assert rel(theta.cpu().numpy() - th, ref.theta_new - th) < 1e-3


@pytest.mark.parametrize("update", ["line_search", "kfac_star"])
def test_heat_steps_fp32_updates(update):
    # three steps of the paper's two update rules in FP32 against the oracle
    N, Nb = 1000, 250
    kw = dict(lam=1e-3, beta=0.9, init_identity=True, momentum=0.6 if update == "line_search" else 0.0)
    cfg = ko.KfacConfig(d=PROB.d, widths=WIDTHS, op=PROB.op, kappa=PROB.kappa,
                        line_search=update == "line_search", kfac_star=update == "kfac_star", **kw)
    st = ko.init_state(cfg)
    opt = _opt("fp32", N, Nb, update=update, **kw)
    th = si.xavier_theta(PROB.d, WIDTHS, 1)
    for step in range(3):
        Xi, f, Xb, g = si.make_batch(PROB, N, Nb, seed=2, step=step)
        res = ko.kfac_step(cfg, st, th, Xi, f, Xb, g)
        theta = torch.tensor(th, device=DEV)
        opt.step(theta, Xi, f, Xb, g)
        torch.cuda.synchronize()
        assert rel(theta.cpu().numpy() - th, res.theta_new - th) < 1e-3, step
        th = res.theta_new
    assert opt.sync_status() == "KFAC_OK"


def test_heat_reverse_mode_full_size():
    # phi = sum_n a_n u_n + b_n^T grad u_n + c_n (partial Laplacian)_n over the
    # workload's 4000 interior points, through ForwardLaplacian.apply
    from paper_2405_15603_gb300.api import ForwardLaplacian
    N = WL.n_int
    rng = np.random.default_rng(31)
    X = si.make_batch(PROB, N, 8, seed=3)[0]
    th0 = si.xavier_theta(PROB.d, WIDTHS, 4)
    th = th0 + 0.05 * rng.standard_normal(th0.size)      # non-zero biases
    a, b, c = (torch.tensor(v, device=DEV) for v in
               (rng.standard_normal(N), rng.standard_normal((N, PROB.d)), rng.standard_normal(N)))
    grads = {}
    for prec in ("fp64", "fp32"):
        opt = _opt(prec, N, 8)
        theta = torch.tensor(th, device=DEV, requires_grad=True)
        Xt = torch.tensor(X, device=DEV, requires_grad=True)
        u, g, lap = ForwardLaplacian.apply(theta, Xt, opt)
        phi = (a * u).sum() + (b * g).sum() + (c * lap).sum()
        grads[prec] = [t.detach().cpu().numpy() for t in torch.autograd.grad(phi, (theta, Xt))]
        assert opt.sync_status() == "KFAC_OK"
        if prec == "fp64":
            # central differences of phi along random directions (FP64 path)
            def phi_at(t):
                uu, gg, ll = opt.forward_laplacian(t, X)
                return float((a * uu).sum() + (b * gg).sum() + (c * ll).sum())
            h = 1e-6
            base = torch.tensor(th, device=DEV)
            for k in range(3):
                v = torch.tensor(rng.standard_normal(th.size), device=DEV)
                fd = (phi_at(base + h * v) - phi_at(base - h * v)) / (2 * h)
                an = float(torch.tensor(grads["fp64"][0], device=DEV) @ v)
                assert abs(fd - an) <= 1e-6 * max(abs(an), 1.0), (fd, an)
    assert rel(grads["fp32"][0], grads["fp64"][0]) < 1e-5
    assert rel(grads["fp32"][1], grads["fp64"][1]) < 1e-5
    # double autograd on the first 64 points (the CPU reference loops over points)
    n = 64
    ref = _double_autograd(th, X[:n], a.cpu().numpy()[:n], b.cpu().numpy()[:n], c.cpu().numpy()[:n])
    opt = _opt("fp64", n, 8)
    dth, dX = opt.forward_laplacian_backward(torch.tensor(th, device=DEV), X[:n], a[:n], b[:n], c[:n],
                                             need_dX=True)
    assert rel(dth.cpu(), ref[0]) < 1e-11 and rel(dX.cpu(), ref[1]) < 1e-11


def _double_autograd(theta, X, a, b, c):
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    net = tr.mlp_from_flat(th, PROB.d, WIDTHS)
    phi = 0.0
    for n in range(X.shape[0]):
        x = Xt[n]
        u = net(x)
        (gr,) = torch.autograd.grad(u, x, create_graph=True)
        lap = 0.0
        for i in range(1, PROB.d):          # the spatial coordinates; coordinate 0 is time
            (gi,) = torch.autograd.grad(gr[i], x, create_graph=True)
            lap = lap + gi[i]
        phi = phi + a[n] * u + (torch.tensor(b[n]) * gr).sum() + c[n] * lap
    dth, dX = torch.autograd.grad(phi, (th, Xt))
    return dth.numpy(), dX.numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_heat_store_forward_matches_recompute(precision):
    from paper_2405_15603_gb300.api import ForwardLaplacian
    N = 1000
    X = torch.tensor(si.make_batch(PROB, N, 8, seed=5)[0], device=DEV)
    th = torch.tensor(si.xavier_theta(PROB.d, WIDTHS, 6), device=DEV)
    out = {}
    for store in (False, True):
        opt = _opt(precision, N, 8)
        opt.set_store_forward(store)
        theta = th.clone().requires_grad_(True)
        u, g, lap = ForwardLaplacian.apply(theta, X, opt)
        (gr,) = torch.autograd.grad(lap.sum() + u.sum() + g.sum(), theta)
        out[store] = gr.cpu().numpy()
    assert np.array_equal(out[True], out[False])
