"""Edge cases of the CUDA path: empty and one-point batches, the largest
factor size the library accepts (h + 1 = 1024), non-finite data, and the
degenerate operator cases (no hidden layer, a single output direction)."""
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


def _opt(d, widths, **kw):
    from paper_2405_15603_gb300.api import KfacPinn
    return KfacPinn(d, widths, device=DEV, **kw)


@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16"])
def test_empty_batches_are_rejected_and_empty_forward_is_a_no_op(precision):
    from paper_2405_15603_gb300.api import KfacError
    d, widths = 3, (16, 16, 1)
    opt = _opt(d, widths, precision=precision, max_n_int=8, max_n_bdy=8)
    th = torch.tensor(si.xavier_theta(d, widths, 0), device=DEV)
    empty = np.zeros((0, d))
    u, g, lap = opt.forward_laplacian(th, empty)
    assert u.numel() == 0 and g.shape == (0, d) and lap.numel() == 0
    one = np.zeros((1, d))
    with pytest.raises(KfacError) as e:
        opt.step(th, empty, np.zeros(0), one, np.zeros(1))
    assert e.value.status == "KFAC_BAD_ARG"
    with pytest.raises(KfacError):
        opt.step(th, one, np.zeros(1), empty, np.zeros(0))
    assert opt.sync_status() == "KFAC_OK"


def test_largest_factor_size():
    # widths up to 1023 and d + 1 <= 1024: factors of size 1024 reach the
    # eigensolver's largest problem (shared-memory back-transform, deepest
    # divide-and-conquer level)
    d, widths = 1023, (1023, 1)
    rng = np.random.default_rng(0)
    N, Nb = 3, 2
    Xi, Xb = rng.random((N, d)), rng.random((Nb, d))
    f, g = rng.standard_normal(N), rng.standard_normal(Nb)
    th = si.xavier_theta(d, widths, 1)
    cfg = ko.KfacConfig(d=d, widths=widths, lam=1e-2, lr=0.5, init_identity=True, beta=0.5)
    res = ko.kfac_step(cfg, ko.init_state(cfg), th, Xi, f, Xb, g)
    opt = _opt(d, widths, max_n_int=N, max_n_bdy=Nb, lam=1e-2, lr=0.5, init_identity=True, beta=0.5)
    theta = torch.tensor(th, device=DEV)
    loss = opt.step(theta, Xi, f, Xb, g)
    torch.cuda.synchronize()
    assert opt.sync_status() == "KFAC_OK"
    assert rel(loss.cpu().numpy(), np.array(res.loss)) < 1e-10
    assert rel(opt.direction().cpu().numpy(), ko.pack_theta(res.direction)) < 1e-8
    assert rel(theta.cpu().numpy() - th, res.theta_new - th) < 1e-8


def test_width_beyond_limit_is_rejected():
    from paper_2405_15603_gb300.api import KfacError
    with pytest.raises(KfacError):
        _opt(4, (1024, 1), max_n_int=2, max_n_bdy=2)
    with pytest.raises(KfacError):
        _opt(1024, (8, 1), max_n_int=2, max_n_bdy=2)


@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16"])
def test_nonfinite_data_latches_status(precision):
    d, widths = 2, (16, 16, 1)
    opt = _opt(d, widths, precision=precision, max_n_int=16, max_n_bdy=8, lr=0.1)
    prob = si.PROBLEMS["poisson2d_sin"]
    Xi, f, Xb, g = si.make_batch(prob, 16, 8, seed=1)
    f = f.copy()
    f[3] = np.nan
    th = torch.tensor(si.xavier_theta(d, widths, 0), device=DEV)
    opt.step(th, Xi, f, Xb, g)
    assert opt.sync_status() == "KFAC_NONFINITE"


def test_line_search_skips_a_step_when_every_trial_is_nonfinite():
    # Only the boundary data are huge: every trial loss overflows, so the step
    # is skipped (alpha = 0, theta unchanged) and NONFINITE is latched.
    d, widths = 2, (8, 1)
    opt = _opt(d, widths, max_n_int=8, max_n_bdy=4, update="line_search")
    prob = si.PROBLEMS["poisson2d_sin"]
    Xi, f, Xb, g = si.make_batch(prob, 8, 4, seed=2)
    g = np.full_like(g, 1e300)
    th0 = si.xavier_theta(d, widths, 0)
    th = torch.tensor(th0, device=DEV)
    opt.step(th, Xi, f, Xb, g)
    torch.cuda.synchronize()
    assert opt.sync_status() == "KFAC_NONFINITE"
    assert np.array_equal(th.cpu().numpy(), th0)
    assert opt.update_coefficients().cpu().numpy()[0] == 0.0


def test_no_hidden_layer_and_single_point():
    # L = 1 (a linear model, the Taylor pass has no activation) with one point each
    for op, kappa in (("laplace", 0.0), ("heat", 0.25)):
        d, widths = 3, (1,)
        prob = si.poisson_cos_problem(d)
        rng = np.random.default_rng(3)
        Xi, Xb = rng.random((1, d)), rng.random((1, d))
        f, g = rng.standard_normal(1), rng.standard_normal(1)
        th = rng.standard_normal(d + 1)
        cfg = ko.KfacConfig(d=d, widths=widths, op=op, kappa=kappa, lam=1e-2, lr=0.3)
        res = ko.kfac_step(cfg, ko.init_state(cfg), th, Xi, f, Xb, g)
        opt = _opt(d, widths, op=op, kappa=kappa, lam=1e-2, lr=0.3, max_n_int=1, max_n_bdy=1)
        theta = torch.tensor(th, device=DEV)
        opt.step(theta, Xi, f, Xb, g)
        assert rel(theta.cpu().numpy() - th, res.theta_new - th) < 1e-10
        assert opt.sync_status() == "KFAC_OK"


def test_split_mode_variants_and_updates():
    # split-BF16 everywhere runs every variant and update rule; the tensor-core
    # precisions need a hidden layer (create rejects L = 1 for them)
    from paper_2405_15603_gb300.api import KfacError
    for prec in ("mixed_split", "mixed_bf16"):
        with pytest.raises(KfacError):
            _opt(3, (1,), precision=prec, max_n_int=8, max_n_bdy=8)
    prob = si.poisson_cos_problem(3)
    Xi, f, Xb, g = si.make_batch(prob, 8, 8, seed=3)
    for kw in (dict(update="line_search"), dict(variant="reduce"), dict(update="kfac_star"),
               dict(variant="reduce", update="kfac_star")):
        opt = _opt(3, (16, 16, 1), precision="mixed_split", max_n_int=8, max_n_bdy=8, **kw)
        th = torch.tensor(si.xavier_theta(3, (16, 16, 1), 0), device=DEV)
        opt.step(th, Xi, f, Xb, g)
        assert opt.sync_status() == "KFAC_OK", kw
        assert torch.isfinite(th).all()
