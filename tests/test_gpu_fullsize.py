"""Parity at the full size of the 100-d benchmark workload (2048 interior and
512 boundary points, 100-768-768-512-512-1) in the configuration bench.py
times: mixed_bf16, the line-search update with momentum, factors from the
identity with β = 0.99, graph mode and the split-K autotuner.

Three steps run as bench.py's warm-up does (eager with the autotuner
measuring, captured, replayed).  The replayed step is checked with
tests/fullsize_checks.py: closed forms and identities that hold at any size,
because a whole step of the oracle at this size takes tens of minutes.  The
forward Laplacian of the step's batch at the outgoing parameters is compared
with the oracle at 32 sampled points.  (tests/test_fullsize_checks.py runs
this same procedure on the oracle's own steps at a small size.)

Tolerances (mixed_bf16):
  * first-layer factors 1e-4: FP32 copies of the points, FP32 products;
  * last-layer factors within 1e-6 of 1;
  * symmetry to 1e-12 of the largest entry; eigenvalues at least β³ less
    1e-5 of the largest;
  * direction within 1e-3 of the FP64 Kronecker-sum inverse of the step's
    own factors applied to its own gradient (FP64 eigensolver, FP32
    preconditioning products);
  * boundary losses 1e-3: split-BF16 value channel (about 1e-5 of u),
    relative to a residual that may be a few times smaller than u;
  * the update identity in FP64, 1e-9;
  * sampled u 1e-3, ∇u 2e-2, Δu 2e-2 normwise (BF16 tangent channel; the
    per-result errors of this net are in tests/test_gpu_error_report.py).
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
FWD_TOL = dict(u=1e-3, grad_u=2e-2, lap_u=2e-2)


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
        return KfacPinn(d, widths, device=DEV, precision="mixed_bf16", max_n_int=n_int, max_n_bdy=n_bdy,
                        **bench.HYPER)

    run_full_size(make_opt, bench.WORKLOAD, DEV, torch.cuda.synchronize, TOL, FWD_TOL)
