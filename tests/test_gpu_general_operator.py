"""GPU parity of the general second-order operator r = Σ_ij c_ij ∂²_ij u - f
(App. C.3): the Taylor pass runs along the eigenvectors of C with weights
equal to its eigenvalues; the oracle propagates the coordinate tangents and
the quadratic form Σ c_ij a_i a_j directly, as printed in the paper."""
import numpy as np
import pytest
import torch

from oracle import kfac_oracle as ko
from synth import inputs as si

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def _coef(d, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((d, d))
    return 0.5 * (M + M.T)            # symmetric, indefinite


def _opt(d, widths, C, **kw):
    from paper_2405_15603_gb300.api import KfacPinn
    return KfacPinn(d, widths, device=DEV, op="general", op_coef=C, **kw)


CASES = [("3-24-16-1", 3, (24, 16, 1), 150, 40), ("7-40-72-1", 7, (40, 72, 1), 67, 13),
         ("5-64-64-48-1", 5, (64, 64, 48, 1), 300, 60)]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_general_forward_and_steps_fp64(case):
    _, d, widths, N, Nb = case
    C = _coef(d, 1)
    prob = si.poisson_cos_problem(d)
    th = si.xavier_theta(d, widths, 2)
    X = si.sample_interior(N, d, np.random.default_rng(3))
    opt = _opt(d, widths, C, max_n_int=N, max_n_bdy=Nb, lam=1e-3, lr=0.1, beta=0.9, momentum=0.3,
               init_identity=True)
    u, g, cu = opt.forward_laplacian(torch.tensor(th, device=DEV), X)
    ru, rg, rc = ko.forward_laplacian(ko.unpack_theta(th, d, widths), X, "general", C)
    torch.cuda.synchronize()
    assert rel(u.cpu(), ru) < 1e-12
    assert rel(g.cpu(), rg) < 1e-11
    assert rel(cu.cpu(), rc) < 1e-10
    cfg = ko.KfacConfig(d=d, widths=widths, op="general", op_coef=C, lam=1e-3, lr=0.1, beta=0.9, momentum=0.3,
                        init_identity=True)
    st = ko.init_state(cfg)
    for step in range(2):
        Xi, f, Xb, gb = si.make_batch(prob, N, Nb, seed=4, step=step)
        res = ko.kfac_step(cfg, st, th, Xi, f, Xb, gb)
        theta = torch.tensor(th, device=DEV)
        loss = opt.step(theta, Xi, f, Xb, gb)
        grad = opt.gradient().cpu().numpy()
        torch.cuda.synchronize()
        assert rel(loss.cpu().numpy(), np.array(res.loss)) < 1e-10
        assert rel(grad, ko.pack_theta(res.grads)) < 1e-9
        for l in range(1, len(widths) + 1):
            for which, ref in zip(("A_int", "B_int"), (st.A_int[l - 1], st.B_int[l - 1])):
                assert rel(opt.get_factor(l, which).cpu(), ref) < 1e-10, (l, which)
        assert rel(theta.cpu().numpy() - th, res.theta_new - th) < 1e-8
        th = res.theta_new
    assert opt.sync_status() == "KFAC_OK"


def test_general_minus_identity_equals_laplace():
    # C = -I gives r = -Δu - f, the Poisson residual
    from paper_2405_15603_gb300.api import KfacPinn
    d, widths, N, Nb = 4, (32, 24, 1), 100, 30
    prob = si.poisson_cos_problem(d)
    kw = dict(max_n_int=N, max_n_bdy=Nb, lam=1e-3, lr=0.1)
    gen = _opt(d, widths, -np.eye(d), **kw)
    lap = KfacPinn(d, widths, device=DEV, **kw)
    th = si.xavier_theta(d, widths, 5)
    t1, t2 = torch.tensor(th, device=DEV), torch.tensor(th, device=DEV)
    Xi, f, Xb, g = si.make_batch(prob, N, Nb, seed=6)
    l1 = gen.step(t1, Xi, f, Xb, g).cpu().numpy()
    l2 = lap.step(t2, Xi, f, Xb, g).cpu().numpy()
    assert rel(l1, l2) < 1e-13
    assert rel(t1.cpu().numpy() - th, t2.cpu().numpy() - th) < 1e-9


def test_general_mixed_precision():
    d, widths, N, Nb = 6, (64, 64, 1), 256, 64
    C = _coef(d, 7)
    prob = si.poisson_cos_problem(d)
    th = si.xavier_theta(d, widths, 8)
    X = si.sample_interior(N, d, np.random.default_rng(9))
    opt = _opt(d, widths, C, precision="mixed_bf16", max_n_int=N, max_n_bdy=Nb, lam=1e-3, lr=0.1)
    u, g, cu = opt.forward_laplacian(torch.tensor(th, device=DEV), X)
    ru, rg, rc = ko.forward_laplacian(ko.unpack_theta(th, d, widths), X, "general", C)
    torch.cuda.synchronize()
    assert rel(u.cpu(), ru) < 1e-4
    assert rel(g.cpu(), rg) < 1e-2
    assert rel(cu.cpu(), rc) < 2e-2
    Xi, f, Xb, gb = si.make_batch(prob, N, Nb, seed=10)
    cfg = ko.KfacConfig(d=d, widths=widths, op="general", op_coef=C, lam=1e-3, lr=0.1)
    res = ko.kfac_step(cfg, ko.init_state(cfg), th, Xi, f, Xb, gb)
    loss = opt.step(torch.tensor(th, device=DEV), Xi, f, Xb, gb)
    grad = opt.gradient().cpu().numpy()
    torch.cuda.synchronize()
    assert rel(loss.cpu().numpy(), np.array(res.loss)) < 1e-3
    assert rel(grad, ko.pack_theta(res.grads)) < 2e-2
    assert opt.sync_status() == "KFAC_OK"


def test_general_operator_rejects_reduce_and_asymmetric():
    from paper_2405_15603_gb300.api import KfacError
    with pytest.raises(KfacError):
        _opt(3, (8, 1), _coef(3, 1), variant="reduce", max_n_int=4, max_n_bdy=4)
    M = np.arange(9.0).reshape(3, 3)
    with pytest.raises(KfacError):
        _opt(3, (8, 1), M, max_n_int=4, max_n_bdy=4)
