"""GPU parity of the KFAC update with momentum and log-grid line search
(Sec. 3.4; App. B): δ̂ = μ δ_{t-1} + Δ_t, α* = argmin over
{2^0, .., 2^-30} of L(θ + α δ̂) on the step's batch, θ += α* δ̂.

FP64 path: trial losses to 1e-10, parameters to 1e-8 over several steps.
Mixed path: the trial losses are checked along the GPU's own δ̂ (the
direction itself carries BF16-level factor errors amplified by 1/λ, see
the mixed parity tests), at the loss tolerance of that path.
"""
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


def _opt(prob, widths, N, Nb, **kw):
    from paper_2405_15603_gb300.api import KfacPinn
    return KfacPinn(prob.d, widths, device=DEV, op=prob.op, kappa=prob.kappa, max_n_int=N,
                    max_n_bdy=Nb, line_search=True, **kw)


def _same_choice(k_gpu, losses_ref, tol):
    k_ref = int(np.argmin(np.where(np.isfinite(losses_ref), losses_ref, np.inf)))
    return k_gpu == k_ref or losses_ref[k_gpu] <= losses_ref[k_ref] * (1 + tol)


FP64_CASES = [
    ("poisson2d_2-32-32-1", si.PROBLEMS["poisson2d_sin"], (32, 32, 1), 900, 120),
    ("heat4d_5-128-128-64-1", si.PROBLEMS["heat4d_sin"], (128, 128, 64, 1), 120, 60),
    ("ragged_7-40-72-1", si.poisson_cos_problem(7), (40, 72, 1), 67, 13),
]


@pytest.mark.parametrize("variant", ["expand", "reduce"])
@pytest.mark.parametrize("case", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_line_search_steps_fp64(case, variant):
    _, prob, widths, N, Nb = case
    kw = dict(beta=0.9, lam=1e-3, momentum=0.6, init_identity=True, variant=variant)
    cfg = ko.KfacConfig(d=prob.d, widths=widths, op=prob.op, kappa=prob.kappa, line_search=True, **kw)
    st = ko.init_state(cfg)
    opt = _opt(prob, widths, N, Nb, **kw)
    th = si.xavier_theta(prob.d, widths, 0)
    for step in range(3):
        Xi, f, Xb, g = si.make_batch(prob, N, Nb, seed=4, step=step)
        res = ko.kfac_step(cfg, st, th, Xi, f, Xb, g)
        theta = torch.tensor(th, device=DEV)
        loss = opt.step(theta, Xi, f, Xb, g)
        ls = opt.line_search_losses().cpu().numpy()
        torch.cuda.synchronize()
        ref = res.extras["line_search_losses"]
        assert rel(loss.cpu().numpy(), np.array(res.loss)) < 1e-10
        fin = np.isfinite(ref[:, 0])
        assert np.array_equal(fin, np.isfinite(ls[:, 0]))
        np.testing.assert_allclose(ls[fin], ref[fin], rtol=1e-10, atol=0)
        k = int(np.argmin(np.where(np.isfinite(ls[:, 0]), ls[:, 0], np.inf)))
        assert _same_choice(k, ref[:, 0], 1e-10)
        assert rel(theta.cpu().numpy() - th, res.theta_new - th) < 1e-8
        th = res.theta_new
    assert opt.sync_status() == "KFAC_OK"


MIXED_CASES = [
    ("poisson5d_5-64-64-48-48-1", si.PROBLEMS["poisson5d_cos"], (64, 64, 48, 48, 1), 300, 50),
    ("heat4d_5-128-128-64-1", si.PROBLEMS["heat4d_sin"], (128, 128, 64, 1), 200, 100),
    ("poisson100d_small_batch", si.PROBLEMS["poisson100d_norm"], (768, 768, 512, 512, 1), 64, 32),
]


@pytest.mark.parametrize("precision", ["mixed_split", "mixed_bf16"])
@pytest.mark.parametrize("case", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_line_search_mixed_along_gpu_direction(case, precision):
    # The trial losses near theta carry the loss bound of the precision's trial
    # pass: split-BF16 on every row for d < 32; plain BF16 tangents otherwise
    # (mixed_bf16 always), whose roundings average over the d tangents of the
    # second-order row: 1e-4 for split-BF16 (d = 100 included), 2e-4 with BF16
    # tangents at d = 5.
    _, prob, widths, N, Nb = case
    cfg = ko.KfacConfig(d=prob.d, widths=widths, op=prob.op, kappa=prob.kappa, lam=1e-3,
                        line_search=True)
    opt = _opt(prob, widths, N, Nb, precision=precision, lam=1e-3)
    th = si.xavier_theta(prob.d, widths, 1)
    Xi, f, Xb, g = si.make_batch(prob, N, Nb, seed=5)
    theta = torch.tensor(th, device=DEV)
    opt.step(theta, Xi, f, Xb, g)
    dhat = opt.direction().cpu().numpy()           # first step: δ̂ = Δ
    ls = opt.line_search_losses().cpu().numpy()
    th_new = theta.cpu().numpy()
    assert opt.sync_status() == "KFAC_OK"
    _, ref = ko.line_search(cfg, th, dhat, Xi, f, Xb, g)
    # Near the starting point (loss within 1.5x of L(θ)) the trial losses
    # carry the loss tolerance of the mixed path; the long trials move the
    # weights far from θ, where larger pre-activations amplify the BF16
    # tangent errors through σ'' (Eq. 6), so they get 1e-2 up to 100x L(θ).
    start = ref[-1, 0]
    near = np.isfinite(ref[:, 0]) & (ref[:, 0] < 1.5 * start)
    far = np.isfinite(ref[:, 0]) & (ref[:, 0] < 100 * start)
    assert near.sum() >= 10
    np.testing.assert_allclose(ls[near, 0], ref[near, 0], rtol=1e-4 if precision == "mixed_split" else 2e-4,
                               atol=0)
    np.testing.assert_allclose(ls[far, 0], ref[far, 0], rtol=1e-2, atol=0)
    k = int(np.argmin(np.where(np.isfinite(ls[:, 0]), ls[:, 0], np.inf)))
    assert _same_choice(k, ref[:, 0], 1e-3)
    np.testing.assert_allclose(th_new, th + 2.0 ** -k * dhat, rtol=1e-13, atol=1e-15)
    assert ref[k, 0] < ko.batch_loss(cfg, th, Xi, f, Xb, g)[0]


@pytest.mark.parametrize("case", MIXED_CASES[:2], ids=[c[0] for c in MIXED_CASES[:2]])
def test_line_search_split_steps_vs_oracle(case):
    # Three line-search steps with momentum and EMA in split-BF16 against the
    # oracle's: the same grid point wins (or one whose oracle loss is within
    # 1e-3 of the oracle's minimum), and the update is within 1e-3.
    _, prob, widths, N, Nb = case
    kw = dict(beta=0.9, lam=1e-3, momentum=0.6, init_identity=True)
    cfg = ko.KfacConfig(d=prob.d, widths=widths, op=prob.op, kappa=prob.kappa, line_search=True, **kw)
    st = ko.init_state(cfg)
    opt = _opt(prob, widths, N, Nb, precision="mixed_split", **kw)
    th = si.xavier_theta(prob.d, widths, 2)
    for step in range(3):
        Xi, f, Xb, g = si.make_batch(prob, N, Nb, seed=11, step=step)
        res = ko.kfac_step(cfg, st, th, Xi, f, Xb, g)
        theta = torch.tensor(th, device=DEV)
        loss = opt.step(theta, Xi, f, Xb, g)
        ls = opt.line_search_losses().cpu().numpy()
        torch.cuda.synchronize()
        ref = res.extras["line_search_losses"]
        assert rel(loss.cpu().numpy(), np.array(res.loss)) < 1e-4
        k = int(np.argmin(np.where(np.isfinite(ls[:, 0]), ls[:, 0], np.inf)))
        assert _same_choice(k, ref[:, 0], 1e-3)
        upd, rupd = theta.cpu().numpy() - th, res.theta_new - th
        if res.extras["alpha"] == 2.0 ** -k:
            assert rel(upd, rupd) < 1e-3, (step, rel(upd, rupd))
        th = res.theta_new
    assert opt.sync_status() == "KFAC_OK"


def test_line_search_not_ready_and_fixed_lr_unchanged():
    from paper_2405_15603_gb300.api import KfacError
    prob = si.PROBLEMS["poisson2d_sin"]
    widths = (16, 1)
    opt = _opt(prob, widths, 50, 20)
    with pytest.raises(KfacError) as e:
        opt.line_search_losses()
    assert e.value.status == "KFAC_NOT_READY"
    # line_search=False keeps the fixed learning rate θ += lr Δ.
    from paper_2405_15603_gb300.api import KfacPinn
    plain = KfacPinn(prob.d, widths, device=DEV, max_n_int=50, max_n_bdy=20, lr=0.25)
    th = si.xavier_theta(prob.d, widths, 2)
    Xi, f, Xb, g = si.make_batch(prob, 50, 20, seed=6)
    theta = torch.tensor(th, device=DEV)
    plain.step(theta, Xi, f, Xb, g)
    d = plain.direction().cpu().numpy()
    np.testing.assert_allclose(theta.cpu().numpy(), th + 0.25 * d, rtol=1e-14, atol=1e-16)
    with pytest.raises(KfacError):
        plain.line_search_losses()
