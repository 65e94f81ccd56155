"""Parity at the full size of the 100-d benchmark workload (2048 interior and
512 boundary points, 100-768-768-512-512-1).

1. Element by element against the oracle: one step on the benchmark's first
   batch with beta = 0 (no EMA history), so the oracle's curvature pass
   (about a minute and 30 GB of host memory at this size) gives every
   factor of all five layers, the gradient and the preconditioned direction
   exactly; compared normwise per result, in the benchmarked precision
   (split-BF16: factors, gradient and forward outputs to 1e-4, the direction
   to 1e-3) and in FP64 (1e-10; the direction 1e-8).  The split-BF16 handle
   runs as bench.py runs it: graph mode and the split-K autotuner, the
   compared step a replay of the captured graph with the tuned chunks.
2. Three steps in the configuration bench.py times (split-BF16, line search
   with momentum, factors from the identity with beta = 0.99, graph mode,
   autotuner), checked with tests/fullsize_checks.py: closed forms and
   identities that hold at any size (a line-search step of the oracle at this
   size takes tens of minutes); the forward Laplacian at the outgoing
   parameters against the oracle at 32 sampled points.
   (tests/test_fullsize_checks.py runs this same procedure on the oracle's
   own steps at a small size.)

Tolerances of the three-step check (split-BF16):
  * first-layer factors 1e-4: FP32 copies of the points, FP32 products;
  * last-layer factors within 1e-6 of 1;
  * symmetry to 1e-12 of the largest entry; eigenvalues at least beta^3 less
    1e-5 of the largest;
  * direction within 1e-3 of the FP64 Kronecker-sum inverse of the step's
    own factors applied to its own gradient (FP64 eigensolver, FP32
    preconditioning products);
  * boundary losses 1e-3: split-BF16 value channel (about 1e-5 of u),
    relative to a residual that may be a few times smaller than u;
  * the update identity in FP64, 1e-9;
  * sampled u, grad u and Laplacian 1e-4 normwise.
"""
import numpy as np
import pytest
import torch

import bench
from oracle import kfac_oracle as ko
from synth import inputs as si
from tests import fullsize_checks as fc

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = dict(A1=1e-4, BL=1e-6, sym=1e-12, eig=1e-5, dir=1e-3, lb=1e-3, upd_rtol=1e-9, upd_atol=1e-13)
FWD_TOL = dict(u=1e-4, grad_u=1e-4, lap_u=1e-4)


def run_full_size(make_opt, wl, device, sync, tol, fwd_tol, n_sample=32):
    """Three steps of wl's problem as bench.py runs them, then the checks."""
    prob, widths = wl.prob, wl.widths
    seed = bench.replica_seed(0)
    batches = [si.make_batch(prob, wl.n_int, wl.n_bdy, seed=seed, step=k) for k in range(3)]
    opt = make_opt(prob.d, widths, wl.n_int, wl.n_bdy)
    opt.set_graph(True)
    opt.set_autotune(True)
    theta = torch.tensor(si.xavier_theta(prob.d, widths, seed), device=device)
    thetas = [theta.cpu().numpy().copy()]
    for b in batches:
        loss = opt.step(theta, *(torch.tensor(a, device=device) for a in b))
        sync()
        thetas.append(theta.cpu().numpy().copy())
    assert opt.sync_status() == "KFAC_OK"
    assert opt.tuning(), "the autotuner measured nothing"

    factors = {(l, w): opt.get_factor(l, w).cpu().numpy() for l in range(1, len(widths) + 1) for w in fc.WHICH}
    obs = dict(theta=thetas, factors=factors, grad=opt.gradient().cpu().numpy(),
               direction=opt.direction().cpu().numpy(), coef=opt.update_coefficients().cpu().numpy(),
               ls=opt.line_search_losses().cpu().numpy(), loss=loss.cpu().numpy())
    fc.check_step(obs, prob.d, widths, bench.HYPER, batches, tol)

    X = batches[-1][0]
    u, gu, lap = (t.cpu().numpy() for t in opt.forward_laplacian(theta, X))
    sync()
    idx = np.sort(np.random.default_rng(0).choice(wl.n_int, min(n_sample, wl.n_int), replace=False))
    ru, rg, rl = ko.forward_laplacian(ko.unpack_theta(thetas[-1], prob.d, widths), X[idx], prob.op)
    assert fc.rel(u[idx], ru) < fwd_tol["u"], fc.rel(u[idx], ru)
    assert fc.rel(gu[idx], rg) < fwd_tol["grad_u"], fc.rel(gu[idx], rg)
    assert fc.rel(lap[idx], rl) < fwd_tol["lap_u"], fc.rel(lap[idx], rl)
    assert opt.sync_status() == "KFAC_OK"
    opt.close()
    return obs


def test_full_size_step_in_the_benchmark_configuration():
    from paper_2405_15603_gb300.api import KfacPinn

    def make_opt(d, widths, n_int, n_bdy):
        return KfacPinn(d, widths, device=DEV, precision="mixed_split", max_n_int=n_int, max_n_bdy=n_bdy,
                        **bench.HYPER)

    run_full_size(make_opt, bench.WORKLOAD, DEV, torch.cuda.synchronize, TOL, FWD_TOL)


@pytest.fixture(scope="module")
def oracle_first_batch():
    """The oracle's curvature pass, gradient and direction on the benchmark's
    first batch at the initial parameters (beta = 0, lambda = 1e-3)."""
    wl = bench.WORKLOAD
    prob, widths = wl.prob, wl.widths
    seed = bench.replica_seed(0)
    th = si.xavier_theta(prob.d, widths, seed)
    batch = si.make_batch(prob, wl.n_int, wl.n_bdy, seed=seed, step=0)
    cfg = ko.KfacConfig(d=prob.d, widths=widths, lam=bench.HYPER["lam"])
    cg = ko.curvature_and_gradient(cfg, ko.unpack_theta(th, prob.d, widths), *batch)
    Ai, Bi, Ab, Bb = cg["factors"]
    direction = [ko.kron_sum_inverse_apply(Ai[l], Bi[l], Ab[l], Bb[l], cg["grads"][l], cfg.lam)
                 for l in range(len(widths))]
    out = cg["fp_i"].Z[-1][:, 0, :]
    ref = dict(theta=th, batch=batch, factors=cg["factors"], grad=ko.pack_theta(cg["grads"]),
               direction=ko.pack_theta(direction), loss=np.array(cg["loss"]),
               u=out[:, 0].copy(), grad_u=out[:, 1:-1].copy(), lap_u=out[:, -1].copy())
    del cg
    return ref


@pytest.mark.parametrize("precision", ["mixed_split", "fp64"])
def test_full_size_elementwise_vs_oracle(oracle_first_batch, precision):
    from paper_2405_15603_gb300.api import KfacPinn
    ref = oracle_first_batch
    wl = bench.WORKLOAD
    prob, widths = wl.prob, wl.widths
    split = precision == "mixed_split"
    tol, dtol = (1e-4, 1e-3) if split else (1e-10, 1e-8)
    opt = KfacPinn(prob.d, widths, device=DEV, precision=precision, max_n_int=wl.n_int, max_n_bdy=wl.n_bdy,
                   lam=bench.HYPER["lam"], beta=0.0, lr=0.1)
    batch = [torch.tensor(a, device=DEV) for a in ref["batch"]]
    theta = torch.tensor(ref["theta"], device=DEV)
    runs = 1
    if split:                     # as bench.py: autotuned chunks, eager, captured, replayed
        opt.set_graph(True)
        opt.set_autotune(True)
        runs = 3
    for _ in range(runs):         # beta = 0 and no momentum: every step is the same step
        theta.copy_(torch.tensor(ref["theta"], device=DEV))
        loss = opt.step(theta, *batch)
    torch.cuda.synchronize()
    assert opt.sync_status() == "KFAC_OK"
    if split:
        assert opt.tuning(), "the autotuner measured nothing"
    errs = {"loss": fc.rel(loss.cpu().numpy(), ref["loss"]),
            "gradient": fc.rel(opt.gradient().cpu().numpy(), ref["grad"])}
    for which, facs in zip(fc.WHICH, ref["factors"]):
        for l in range(1, len(widths) + 1):
            errs[f"{which}_{l}"] = fc.rel(opt.get_factor(l, which).cpu().numpy(), facs[l - 1])
    errs["direction"] = fc.rel(opt.direction().cpu().numpy(), ref["direction"])
    u, gu, lap = (t.cpu().numpy() for t in opt.forward_laplacian(torch.tensor(ref["theta"], device=DEV),
                                                                 ref["batch"][0]))
    errs["u"], errs["grad_u"], errs["lap_u"] = (fc.rel(u, ref["u"]), fc.rel(gu, ref["grad_u"]),
                                                fc.rel(lap, ref["lap_u"]))
    print()
    print(precision, " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v < (dtol if k == "direction" else tol), (k, v)
    opt.close()
