"""Checks of KFAC steps at sizes where the oracle cannot take the whole step.

A step of the FP64 oracle on the 100-d benchmark workload (2048 interior and
512 boundary points, 100-768-768-512-512-1) takes tens of minutes on the host,
so the step of the CUDA path at that size is checked through what the oracle
computes in closed form or point by point, and through identities that hold
at any size:

  * the first layer's factors A_Ω^{(1)}, A_∂^{(1)} depend on the points alone
    (the Taylor input matrix of Sec. 3.1), so their EMA (Sec. 3.4) over the
    steps has a closed form (Eq. 8 interior, Eq. 3 boundary);
  * the last layer's factors B_Ω^{(L)} = B_∂^{(L)} = 1: the residual seed has
    unit norm for the Poisson residual and for u - g (Eq. 1);
  * every EMA factor started from the identity is symmetric with eigenvalues
    at least β^t (a convex combination of the identity and PSD Grams);
  * the direction is the damped Kronecker-sum inverse (Sec. 3.4) of the
    step's own factors applied to its own gradient, recomputed in FP64;
  * the line search (Sec. 3.4) picks the grid point of the smallest finite
    trial loss (ties: the larger step), with δ_t = α*(μ δ_{t-1} + Δ_t);
  * L = L_Ω + L_∂, and the boundary loss of Eq. 1 needs only plain forward
    passes of the boundary points.

The functions take plain arrays, so the same checks run on the CUDA path
(tests/test_gpu_fullsize.py) and on the oracle's own steps at a small size
(tests/test_oracle.py), where they must hold to rounding.
"""
import math

import numpy as np

from oracle import kfac_oracle as ko

WHICH = ("A_int", "B_int", "A_bdy", "B_bdy")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def first_layer_factor_ema(batches, beta, interior):
    """A^{(1)} after one EMA update per batch, started from the identity."""
    A = None
    for X_int, _, X_bdy, _ in batches:
        T = ko.input_taylor_matrix(X_int if interior else X_bdy, interior)
        A_hat = ko.factors_expand(T, np.zeros((T.shape[0], 1, T.shape[2])))[0]
        if A is None:
            A = np.eye(A_hat.shape[0])
        A = beta * A + (1.0 - beta) * A_hat
    return A


def boundary_loss(theta, d, widths, X_bdy, g):
    """L_∂ of Eq. 1 at theta: plain forward passes of the boundary points."""
    fp = ko.taylor_forward(ko.unpack_theta(theta, d, widths), X_bdy, "laplace", False)
    return ko.loss(np.zeros(1), ko.boundary_residual(fp, g))[2]


def check_step(obs, d, widths, hyper, batches, tol):
    """Check the last of len(batches) line-search KFAC steps of a Poisson
    problem whose factors started from the identity.

    obs: theta (parameters before and after each step, len(batches) + 1
    packed vectors), factors ({(layer, which): matrix} after the last step),
    grad and direction (packed, of the last step), coef ((c0, c1) of its
    update δ = c0 Δ + c1 δ_prev), ls (its 31 x 3 trial losses), loss (its
    (L, L_Ω, L_∂) at the incoming parameters).
    tol: A1, BL, sym, eig, dir, lb (relative), upd_rtol, upd_atol."""
    assert hyper["init_identity"] and hyper["update"] == "line_search"
    beta, lam, mu = hyper["beta"], hyper["lam"], hyper["momentum"]
    t = len(batches)
    L = len(widths)
    th = [np.asarray(x, dtype=np.float64) for x in obs["theta"]]
    assert len(th) == t + 1 and t >= 2
    fac = obs["factors"]

    # first-layer factors in closed form (the identity part cancels exactly)
    for which, interior in (("A_int", True), ("A_bdy", False)):
        got = fac[(1, which)]
        ref = first_layer_factor_ema(batches, beta, interior)
        base = beta ** t * np.eye(ref.shape[0])
        assert rel(got - base, ref - base) < tol["A1"], (which, rel(got - base, ref - base))

    # last-layer output factors
    for which in ("B_int", "B_bdy"):
        M = fac[(L, which)]
        assert M.shape == (1, 1) and abs(M[0, 0] - 1.0) < tol["BL"], (which, M)

    # symmetric, eigenvalues at least beta^t
    for (l, which), M in fac.items():
        scale = np.abs(M).max()
        assert np.abs(M - M.T).max() <= tol["sym"] * scale, (l, which)
        ev = np.linalg.eigvalsh(0.5 * (M + M.T))
        assert ev[0] >= beta ** t - tol["eig"] * ev[-1], (l, which, ev[0], ev[-1])

    # direction: the damped Kronecker-sum inverse of the step's own factors
    G = ko.unpack_theta(obs["grad"], d, widths)
    ref = [ko.kron_sum_inverse_apply(fac[(l + 1, "A_int")], fac[(l + 1, "B_int")], fac[(l + 1, "A_bdy")],
                                     fac[(l + 1, "B_bdy")], G[l], lam, False) for l in range(L)]
    assert rel(obs["direction"], ko.pack_theta(ref)) < tol["dir"], rel(obs["direction"], ko.pack_theta(ref))
    assert float(np.dot(obs["grad"], obs["direction"])) < 0.0

    # line search: smallest finite trial loss, ties to the larger step
    ls = np.asarray(obs["ls"], dtype=np.float64)
    assert ls.shape == (31, 3)
    fin = np.isfinite(ls[:, 0])
    np.testing.assert_allclose(ls[fin, 0], ls[fin, 1] + ls[fin, 2], rtol=1e-13, atol=0)
    k = int(np.argmin(np.where(fin, ls[:, 0], np.inf)))
    assert fin[k]
    c0, c1 = (float(c) for c in obs["coef"])
    assert c0 == 2.0 ** -k, (c0, k)
    assert math.isclose(c1, c0 * mu, rel_tol=1e-14), (c1, c0, mu)

    # update: theta_t - theta_{t-1} = c0 Delta_t + c1 (theta_{t-1} - theta_{t-2})
    np.testing.assert_allclose(th[t] - th[t - 1], c0 * obs["direction"] + c1 * (th[t - 1] - th[t - 2]),
                               rtol=tol["upd_rtol"], atol=tol["upd_atol"] * np.abs(th[t - 1]).max())

    # losses: L = L_Ω + L_∂; the boundary loss at the incoming and the chosen parameters
    loss = np.asarray(obs["loss"], dtype=np.float64)
    assert math.isclose(loss[0], loss[1] + loss[2], rel_tol=1e-13)
    _, _, X_bdy, g = batches[-1]
    lb_in = boundary_loss(th[t - 1], d, widths, X_bdy, g)
    lb_out = boundary_loss(th[t], d, widths, X_bdy, g)
    assert rel(loss[2], lb_in) < tol["lb"], (loss[2], lb_in)
    assert rel(ls[k, 2], lb_out) < tol["lb"], (ls[k, 2], lb_out)
    return k
