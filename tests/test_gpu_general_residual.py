"""GPU parity of the general-residual KFAC (Sec. 3.3, Eq. 9-10) against the
oracle: M residual outputs that are polynomials of degree two in the
network's Taylor outputs, the criterion 1/2 r^T W r (Lambda = W).  The CUDA
path forms B_Omega from M adjoint passes seeded with the columns of the
Cholesky factor of W and the gradient from one seeded with W r_n; the oracle
forms Eq. 10 with W directly and is pinned to autograd and closed forms
(tests/test_oracle_general_residual.py).

FP64 to 1e-10 (parameters over several steps 1e-8); FP32 to the
reduced-precision bounds (1e-4 on loss, gradient and factors, 1e-3 on the
update)."""
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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _nonlinear_system(d=3, M=2, seed=0):
    rng = np.random.default_rng(seed)
    S = d + 2
    b = rng.standard_normal((M, S))
    Q = rng.standard_normal((M, S, S))
    Q = 0.25 * (Q + np.transpose(Q, (0, 2, 1)))
    A = rng.standard_normal((M, M))
    return dict(b=b, Q=Q, W=A @ A.T + M * np.eye(M))


def _log_fokker_planck_like(d=5):
    # r = du/dt - 1/2 Laplacian_x u - 1/2 |grad_x u|^2 - f  (coordinate 0 is t)
    S = d + 2
    b = np.zeros((1, S))
    b[0, 1] = 1.0
    b[0, S - 1] = -0.5
    Q = np.zeros((1, S, S))
    for i in range(2, d + 1):
        Q[0, i, i] = -1.0
    return dict(b=b, Q=Q, W=None)


def _convection_diffusion(d=4):
    # r = -Laplacian u + beta . grad u - f
    S = d + 2
    b = np.zeros((1, S))
    b[0, S - 1] = -1.0
    b[0, 1:d + 1] = np.linspace(0.5, -0.5, d)
    return dict(b=b, Q=None, W=None)


CASES = [
    ("system_M2_quadratic_3-16-12-1", "laplace", 3, (16, 12, 1), _nonlinear_system(3, 2), 67, 13),
    ("log_fokker_planck_like_5-24-24-1", "heat", 5, (24, 24, 1), _log_fokker_planck_like(5), 90, 30),
    ("convection_diffusion_4-20-1", "laplace", 4, (20, 1), _convection_diffusion(4), 40, 20),
]


def _data(d, M, N, Nb, seed):
    rng = np.random.default_rng(seed)
    return rng.random((N, d)), rng.standard_normal((N, M)), rng.random((Nb, d)), rng.standard_normal(Nb)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("update", ["fixed", "line_search"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_general_residual_steps_vs_oracle(case, update, precision):
    from paper_2405_15603_gb300.api import KfacPinn
    _, op, d, widths, res, N, Nb = case
    M = res["b"].shape[0]
    kw = dict(lam=1e-3, beta=0.9, init_identity=True, momentum=0.5, lr=0.05)
    cfg = ko.KfacConfig(d=d, widths=widths, op=op, kappa=0.0, line_search=update == "line_search",
                        residual=ko.QuadraticResidual(b=res["b"], Q=res["Q"], W=res["W"]), **kw)
    st = ko.init_state(cfg)
    opt = KfacPinn(d, widths, device=DEV, op=op, precision=precision, max_n_int=N, max_n_bdy=Nb,
                   update=update, residual=res, **kw)
    rng = np.random.default_rng(1)
    th = si.xavier_theta(d, widths, 2) + 0.05 * rng.standard_normal(opt.D)
    fp64 = precision == "fp64"
    for step in range(3):
        Xi, F, Xb, g = _data(d, M, N, Nb, 10 + step)
        ref = ko.kfac_step(cfg, st, th, Xi, F, Xb, g)
        theta = torch.tensor(th, device=DEV)
        loss = opt.step(theta, Xi, F, Xb, g)
        torch.cuda.synchronize()
        assert rel(loss.cpu().numpy(), np.array(ref.loss)) < (1e-10 if fp64 else 1e-5)
        assert rel(opt.gradient().cpu().numpy(), ko.pack_theta(ref.grads)) < (1e-10 if fp64 else 1e-4)
        for which, facs in zip(("A_int", "B_int", "A_bdy", "B_bdy"), ref.factors):
            for l in range(1, len(widths) + 1):
                got = opt.get_factor(l, which).cpu().numpy()
                assert rel(got, facs[l - 1]) < (1e-10 if fp64 else 1e-4), (step, which, l)
        if update == "line_search":
            ls = opt.line_search_losses().cpu().numpy()
            np.testing.assert_allclose(ls, ref.extras["line_search_losses"], rtol=1e-10 if fp64 else 1e-5)
        assert rel(theta.cpu().numpy() - th, ref.theta_new - th) < (1e-8 if fp64 else 1e-3), step
        th = ref.theta_new
    assert opt.sync_status() == "KFAC_OK"


def test_general_residual_host_batch_and_graph_mode_match_device_steps():
    # the interior data of every call hold N x M values: the host-batch step
    # and the staged graph replay must carry all of them
    from paper_2405_15603_gb300.api import KfacPinn
    _, op, d, widths, res, N, Nb = CASES[0]
    M = res["b"].shape[0]
    kw = dict(lam=1e-3, beta=0.9, init_identity=True, lr=0.05, residual=res, max_n_int=N, max_n_bdy=Nb)
    batches = [_data(d, M, N, Nb, 20 + k) for k in range(4)]
    th0 = si.xavier_theta(d, widths, 3)
    out = []
    for mode in ("device", "host", "graph"):
        opt = KfacPinn(d, widths, device=DEV, **kw)
        if mode == "graph":
            opt.set_graph(True)
        theta = torch.tensor(th0, device=DEV)
        for b in batches:
            if mode == "host":
                opt.step_host(theta, *b)
            else:
                opt.step(theta, *b)
        torch.cuda.synchronize()
        out.append(theta.cpu().numpy())
        assert opt.sync_status() == "KFAC_OK"
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_general_residual_rejected_combinations():
    from paper_2405_15603_gb300.api import KfacError, KfacPinn
    res = _nonlinear_system(3, 2)
    for kw in (dict(precision="mixed_split"), dict(update="kfac_star"), dict(variant="reduce"),
               dict(op="general", op_coef=np.eye(3))):
        with pytest.raises(KfacError):
            KfacPinn(3, (16, 12, 1), device=DEV, residual=res, max_n_int=8, max_n_bdy=8, **kw)
    bad_w = dict(res, W=-np.eye(2))
    bad_q = dict(res, Q=res["Q"] + np.arange(5.0)[None, :, None])
    for r in (bad_w, bad_q):
        with pytest.raises(KfacError):
            KfacPinn(3, (16, 12, 1), device=DEV, residual=r, max_n_int=8, max_n_bdy=8)
