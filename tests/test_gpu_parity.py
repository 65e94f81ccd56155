"""GPU parity: the CUDA path through the C-ABI against the FP64 CPU oracle.

Tolerances are normwise relative errors per result.  FP64 path: 1e-10 on the
Taylor pass, loss, gradient and factors; the preconditioned direction and the
update go through an inverse whose condition number is up to ‖A‖/λ per
factor (the damped factors have eigenvalues down to λ), which multiplies the
~1e-14 rounding of the factors and gradient by up to 1e4-1e5 at λ = 1e-3, so
they are held to 1e-9.
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
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _opt(d, widths, **kw):
    from paper_2405_15603_gb300.api import KfacPinn
    return KfacPinn(d, widths, device=DEV, **kw)


def _theta(d, widths, seed=0, bias=0.2):
    th = si.xavier_theta(d, widths, seed)
    Ws = ko.unpack_theta(th, d, widths)
    rng = np.random.default_rng(seed + 7)
    for W in Ws:
        W[:, -1] = bias * rng.standard_normal(W.shape[0])
    return ko.pack_theta(Ws)


CASES = [
    # (name, problem, widths, N_int, N_bdy)
    ("poisson2d_2-32-32-1", "poisson2d_sin", (32, 32, 1), 900, 120),
    ("poisson5d_5-64-64-48-48-1", "poisson5d_cos", (64, 64, 48, 48, 1), 300, 50),
    ("heat4d_5-128-128-64-1", "heat4d_sin", (128, 128, 64, 1), 200, 100),
    ("ragged_3-70-33-1", None, (70, 33, 1), 67, 13),
]


def _problem(name, d=3):
    if name is None:
        return si.poisson_cos_problem(d)
    return si.PROBLEMS[name]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_forward_laplacian_fp64(case):
    _, pname, widths, N, _ = case
    prob = _problem(pname)
    th = _theta(prob.d, widths, 1)
    X = si.sample_interior(N, prob.d, np.random.default_rng(3))
    opt = _opt(prob.d, widths, op=prob.op, kappa=prob.kappa, max_n_int=N, max_n_bdy=8)
    u, g, lap = opt.forward_laplacian(torch.tensor(th, device=DEV), X)
    torch.cuda.synchronize()
    ru, rg, rl = ko.forward_laplacian(ko.unpack_theta(th, prob.d, widths), X, prob.op)
    assert rel(u.cpu(), ru) < 1e-10
    assert rel(g.cpu(), rg) < 1e-10
    assert rel(lap.cpu(), rl) < 1e-10
    assert opt.sync_status() == "KFAC_OK"


def test_forward_laplacian_chunks_beyond_capacity():
    prob = si.PROBLEMS["poisson5d_cos"]
    widths = (16, 8, 1)
    th = _theta(prob.d, widths, 2)
    X = si.sample_interior(101, prob.d, np.random.default_rng(5))
    opt = _opt(prob.d, widths, max_n_int=32, max_n_bdy=4)
    u, g, lap = opt.forward_laplacian(torch.tensor(th, device=DEV), X)
    ru, rg, rl = ko.forward_laplacian(ko.unpack_theta(th, prob.d, widths), X)
    assert rel(u.cpu(), ru) < 1e-10 and rel(lap.cpu(), rl) < 1e-10 and rel(g.cpu(), rg) < 1e-10


def _factor_case(case, variant):
    _, pname, widths, N, Nb = case
    prob = _problem(pname)
    th = _theta(prob.d, widths, 4)
    Xi, f, Xb, g = si.make_batch(prob, N, Nb, seed=11)
    cfg = ko.KfacConfig(d=prob.d, widths=widths, op=prob.op, kappa=prob.kappa, variant=variant)
    ref = ko.curvature_and_gradient(cfg, ko.unpack_theta(th, prob.d, widths), Xi, f, Xb, g)
    opt = _opt(prob.d, widths, op=prob.op, kappa=prob.kappa, variant=variant, max_n_int=N, max_n_bdy=Nb)
    loss = opt.factors(torch.tensor(th, device=DEV), Xi, f, Xb, g)
    torch.cuda.synchronize()
    return prob, widths, ref, opt, loss


@pytest.mark.parametrize("variant", ["expand", "reduce"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_loss_gradient_factors_fp64(case, variant):
    prob, widths, ref, opt, loss = _factor_case(case, variant)
    assert rel(loss.cpu().numpy(), np.array(ref["loss"])) < 1e-10
    assert rel(opt.gradient().cpu(), ko.pack_theta(ref["grads"])) < 1e-10
    Ai, Bi, Ab, Bb = ref["factors"]
    for l in range(len(widths)):
        for which, M in (("A_int", Ai), ("B_int", Bi), ("A_bdy", Ab), ("B_bdy", Bb)):
            got = opt.get_factor(l + 1, which).cpu().numpy()
            assert rel(got, M[l]) < 1e-10, (l, which, rel(got, M[l]))
    assert opt.sync_status() == "KFAC_OK"


@pytest.mark.parametrize("damping_sqrt", [False, True])
@pytest.mark.parametrize("case", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_invert_precondition_fp64(case, damping_sqrt):
    _, pname, widths, N, Nb = case
    prob = _problem(pname)
    lam = 1e-3
    th = _theta(prob.d, widths, 6)
    Xi, f, Xb, g = si.make_batch(prob, N, Nb, seed=12)
    cfg = ko.KfacConfig(d=prob.d, widths=widths, op=prob.op, kappa=prob.kappa, lam=lam,
                        damping_sqrt=damping_sqrt)
    ref = ko.curvature_and_gradient(cfg, ko.unpack_theta(th, prob.d, widths), Xi, f, Xb, g)
    opt = _opt(prob.d, widths, op=prob.op, kappa=prob.kappa, lam=lam, damping_sqrt=damping_sqrt,
               max_n_int=N, max_n_bdy=Nb)
    opt.factors(torch.tensor(th, device=DEV), Xi, f, Xb, g)
    opt.invert()
    d_gpu = opt.precondition().cpu().numpy()
    Ai, Bi, Ab, Bb = ref["factors"]
    d_ref = ko.pack_theta([ko.kron_sum_inverse_apply(Ai[l], Bi[l], Ab[l], Bb[l], ref["grads"][l], lam,
                                                     damping_sqrt) for l in range(len(widths))])
    assert rel(d_gpu, d_ref) < 1e-9, rel(d_gpu, d_ref)
    assert opt.sync_status() == "KFAC_OK"


def test_precondition_given_factors_and_gradient():
    # Set random SPD factors directly and precondition an arbitrary gradient.
    d, widths = 4, (9, 6, 1)
    opt = _opt(d, widths, lam=1e-2, max_n_int=4, max_n_bdy=4)
    rng = np.random.default_rng(0)
    mats = {}
    dims = [d] + list(widths)
    for l in range(1, len(dims)):
        for which in ("A_int", "B_int", "A_bdy", "B_bdy"):
            n = dims[l - 1] + 1 if which[0] == "A" else dims[l]
            M = rng.standard_normal((n, n + 2))
            mats[(l, which)] = M @ M.T / n
            opt.set_factor(l, which, mats[(l, which)])
    G = rng.standard_normal(opt.D)
    opt.invert()
    out = opt.precondition(torch.tensor(G, device=DEV)).cpu().numpy()
    Gs = ko.unpack_theta(G, d, widths)
    ref = ko.pack_theta([ko.kron_sum_inverse_apply(mats[(l, "A_int")], mats[(l, "B_int")],
                                                   mats[(l, "A_bdy")], mats[(l, "B_bdy")], Gs[l - 1], 1e-2)
                         for l in range(1, len(dims))])
    assert rel(out, ref) < 1e-10


@pytest.mark.parametrize("dims,rank", [((50, (300, 129, 1)), None), ((100, (768, 512, 1)), 40)])
def test_eigensolver_large_and_low_rank_factors(dims, rank):
    # Sizes that exercise the blocked Cholesky (several 64-blocks), the
    # cooperative tridiagonalisation and every divide-and-conquer level;
    # low-rank boundary factors give clustered whitened spectra.
    d, widths = dims
    opt = _opt(d, widths, lam=1e-3, max_n_int=4, max_n_bdy=4)
    rng = np.random.default_rng(1)
    mats = {}
    full = [d] + list(widths)
    for l in range(1, len(full)):
        for which in ("A_int", "B_int", "A_bdy", "B_bdy"):
            n = full[l - 1] + 1 if which[0] == "A" else full[l]
            k = n + 3 if (rank is None or which.endswith("int")) else min(rank, n)
            M = rng.standard_normal((n, k))
            mats[(l, which)] = M @ M.T / k
            opt.set_factor(l, which, mats[(l, which)])
    G = rng.standard_normal(opt.D)
    opt.invert()
    out = opt.precondition(torch.tensor(G, device=DEV)).cpu().numpy()
    assert opt.sync_status() == "KFAC_OK"
    Gs = ko.unpack_theta(G, d, widths)
    ref = ko.pack_theta([ko.kron_sum_inverse_apply(mats[(l, "A_int")], mats[(l, "B_int")],
                                                   mats[(l, "A_bdy")], mats[(l, "B_bdy")], Gs[l - 1], 1e-3)
                         for l in range(1, len(full))])
    assert rel(out, ref) < 1e-9, rel(out, ref)


@pytest.mark.parametrize("variant", ["expand", "reduce"])
def test_kfac_steps_fp64(variant):
    # Three steps with EMA, momentum and identity initialisation.
    prob = si.PROBLEMS["poisson2d_sin"]
    widths = (32, 32, 1)
    kw = dict(beta=0.8, lam=1e-3, lr=0.05, momentum=0.5, init_identity=True, variant=variant)
    th0 = si.xavier_theta(prob.d, widths, 0)
    cfg = ko.KfacConfig(d=prob.d, widths=widths, **{k: v for k, v in kw.items()})
    st = ko.init_state(cfg)
    opt = _opt(prob.d, widths, max_n_int=900, max_n_bdy=120, **kw)
    theta = torch.tensor(th0, device=DEV)
    th = th0.copy()
    for step in range(3):
        Xi, f, Xb, g = si.make_batch(prob, 900, 120, seed=0, step=step)
        res = ko.kfac_step(cfg, st, th, Xi, f, Xb, g)
        loss = opt.step(theta, Xi, f, Xb, g)
        torch.cuda.synchronize()
        assert rel(loss.cpu().numpy(), np.array(res.loss)) < 1e-9
        assert rel(theta.cpu().numpy() - th, res.theta_new - th) < 1e-8
        th = res.theta_new
        theta = torch.tensor(th, device=DEV)   # continue from the oracle's parameters
    assert opt.sync_status() == "KFAC_OK"


def test_single_point_and_single_layer():
    # N = 1 interior and boundary point; L = 1 (a linear model, no tanh).
    for widths in ((1,), (5, 1)):
        d = 3
        prob = si.poisson_cos_problem(d)
        th = _theta(d, widths, 3)
        Xi, f, Xb, g = si.make_batch(prob, 1, 1, seed=5)
        cfg = ko.KfacConfig(d=d, widths=widths, lam=1e-2, lr=0.3)
        res = ko.kfac_step(cfg, ko.init_state(cfg), th, Xi, f, Xb, g)
        opt = _opt(d, widths, lam=1e-2, lr=0.3, max_n_int=1, max_n_bdy=1)
        theta = torch.tensor(th, device=DEV)
        opt.step(theta, Xi, f, Xb, g)
        assert rel(theta.cpu().numpy() - th, res.theta_new - th) < 1e-9
        assert opt.sync_status() == "KFAC_OK"


def test_step_host_matches_device_step():
    prob = si.PROBLEMS["poisson5d_cos"]
    widths = (24, 24, 1)
    th0 = si.xavier_theta(prob.d, widths, 1)
    Xi, f, Xb, g = si.make_batch(prob, 100, 30, seed=2)
    a = _opt(prob.d, widths, max_n_int=100, max_n_bdy=30)
    b = _opt(prob.d, widths, max_n_int=100, max_n_bdy=30)
    ta, tb = torch.tensor(th0, device=DEV), torch.tensor(th0, device=DEV)
    la = a.step(ta, Xi, f, Xb, g).cpu().numpy()
    lb = b.step_host(tb, Xi, f, Xb, g)
    assert np.array_equal(la, lb)
    assert torch.equal(ta, tb)


def test_bad_arguments_and_not_pd():
    from paper_2405_15603_gb300.api import KfacPinn, KfacError
    with pytest.raises(KfacError):
        KfacPinn(2, (4, 2), device=DEV)               # last width must be 1
    opt = _opt(2, (4, 1), max_n_int=8, max_n_bdy=4)
    prob = si.PROBLEMS["poisson2d_sin"]
    Xi, f, Xb, g = si.make_batch(prob, 9, 4, seed=0)
    th = torch.tensor(si.xavier_theta(2, (4, 1), 0), device=DEV)
    with pytest.raises(KfacError):
        opt.step(th, Xi, f, Xb, g)                    # 9 > max_n_int
    with pytest.raises(KfacError):
        opt.precondition()                            # before invert: not ready
    # A negative-definite interior factor: the Cholesky fails, status NOT_PD.
    opt.set_factor(1, "A_int", -np.eye(3))
    opt.invert()
    assert opt.sync_status() == "KFAC_NOT_PD"
    assert opt.sync_status() == "KFAC_OK"             # cleared by the read
