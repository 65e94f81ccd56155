"""The oracle's pins have teeth: each case plants one plausible mistake in the
oracle (on the CPU, by replacing one of its functions for the duration of
the test) and checks that the pin written for that part of the method fails.
A mistake that no pin caught would leave the GPU parity tests comparing
against a wrong reference."""
import numpy as np
import pytest

from oracle import kfac_oracle as ko
from tests import test_oracle as pins
from tests import test_oracle_general_residual as gpins


def _wrap(name, make):
    """(function name, factory of the mutant from the original)."""
    return name, make


def _with(cfg, **kw):
    """A copy of an oracle dataclass (config, residual) with some fields replaced."""
    import dataclasses
    return dataclasses.replace(cfg, **kw)


def _ties_keep_smaller_alpha(cfg, theta, dhat, X_int, f, X_bdy, g):
    losses = [ko.batch_loss(cfg, theta + a * dhat, X_int, f, X_bdy, g) for a in ko.LINE_SEARCH_GRID]
    best = None
    for k, (tot, _, _) in enumerate(losses):
        if np.isfinite(tot) and (best is None or tot <= losses[best][0]):
            best = k
    return (0.0 if best is None else ko.LINE_SEARCH_GRID[best]), np.array(losses)


MUTANTS = {
    # Eq. 6: the second-order column loses σ'' Σ_ij c_ij a_i a_j
    "tanh rule without the second-order term": (
        _wrap("tanh_taylor", lambda o: lambda Z, C: o(Z, 0.0 * C)),
        lambda: pins.test_forward_laplacian_vs_autograd_hessian_trace(2, (5, 4, 1))),
    # Eq. 6 with σ'' of the wrong sign
    "tanh rule with the sign of sigma'' flipped": (
        _wrap("tanh_taylor", lambda o: lambda Z, C: o(Z, -C)),
        pins.test_one_hidden_layer_closed_form),
    # Eq. 1: Δu - f instead of -Δu - f
    "interior residual with the wrong sign of the Laplacian": (
        _wrap("interior_residual", lambda o: lambda fp, f, op, kappa: -o(fp, f, op, kappa) - 2.0 * f),
        lambda: pins.test_loss_gradient_vs_autograd("laplace")),
    # Sec. 3.2: the adjoint of the second-order column drops its cross terms
    "adjoint of the tanh rule without the second-order terms": (
        _wrap("tanh_taylor_adjoint", lambda o: lambda Z, Ybar, C: o(Z, Ybar, 0.0 * C)),
        lambda: pins.test_loss_gradient_vs_autograd("laplace")),
    # Eq. 2: the boundary term of the gradient left out
    "gradient without the boundary term": (
        _wrap("loss_gradient", lambda o: lambda fi, zi, ri, fb, zb, rb: o(fi, zi, ri, fb, zb, 0.0 * rb)),
        lambda: pins.test_loss_gradient_vs_autograd("heat")),
    # Eq. 8: A normalised by N instead of N·S
    "A factor normalised by N instead of N S": (
        _wrap("factors_expand", lambda o: lambda T, G: (o(T, G)[0] * T.shape[2], o(T, G)[1])),
        lambda: pins.test_factor_structure("expand")),
    # Eq. 8: B without the 1/N
    "B factor without 1/N": (
        _wrap("factors_expand", lambda o: lambda T, G: (o(T, G)[0], o(T, G)[1] * T.shape[0])),
        lambda: pins.test_factor_structure("expand")),
    # KFAC-reduce with summed instead of averaged inputs
    "KFAC-reduce A from summed inputs": (
        _wrap("factors_reduce", lambda o: lambda T, G: (o(T, G)[0] * T.shape[2] ** 2, o(T, G)[1])),
        lambda: pins.test_factor_structure("reduce")),
    # Sec. 3.4: the boundary Kronecker term left out of the inverse
    "inverse without the boundary Kronecker term": (
        _wrap("kron_sum_inverse_apply",
              lambda o: lambda Ai, Bi, Ab, Bb, G, lam, damping_sqrt=False:
              o(Ai, Bi, 0.0 * Ab, 0.0 * Bb, G, lam, damping_sqrt)),
        lambda: pins.test_kron_sum_inverse_vs_dense_solve(False)),
    # Sec. 3.4: damping added to every entry instead of the diagonal
    "damping on every entry": (
        _wrap("damp", lambda o: lambda M, lam, damping_sqrt: M + (np.sqrt(lam) if damping_sqrt else lam)),
        lambda: pins.test_kron_sum_inverse_vs_dense_solve(False)),
    # the generalized eigenvectors not normalised to V^T P V = I
    "generalized eigenvectors not P-normalised": (
        _wrap("generalized_eig", lambda o: lambda P, Q: (2.0 * o(P, Q)[0], o(P, Q)[1])),
        lambda: pins.test_kron_sum_inverse_vs_dense_solve(True)),
    # Sec. 3.4 (KFAC*): the Gramian products without the boundary term
    "Gramian products without the boundary term": (
        _wrap("gramian_bilinear",
              lambda o: lambda ja, jb, W=None: o((ja[0], 0.0 * ja[1]), (jb[0], 0.0 * jb[1]), W)),
        pins.test_gramian_products_vs_full_ggn),
    # Sec. 3.4 (KFAC*): the model's damping term left out of the 2 x 2 system
    "KFAC* coefficients without damping": (
        _wrap("kfac_star_coefficients",
              lambda o: lambda cfg, cg, Delta, delta, grad:
              o(_with(cfg, lam=0.0), cg, Delta, delta, grad)),
        pins.test_kfac_star_minimises_quadratic_model),
    # Algorithm 1: identity initialisation of the EMA ignored
    "EMA started from zero instead of the identity": (
        _wrap("init_state", lambda o: lambda cfg: o(_with(cfg, init_identity=False))),
        pins.test_ema_and_identity_init),
    # Sec. 3.3 (Eq. 9): the quadratic term without its factor 1/2
    "general residual with the quadratic term doubled": (
        _wrap("quadratic_residual",
              lambda o: lambda res, z, f: o(_with(res, Q=None if res.Q is None else 2.0 * res.Q), z, f)),
        lambda: gpins.test_residual_and_gradient_vs_autograd(True)),
    # Sec. 3.3: the residual's Jacobian without the quadratic term's part
    "general residual Jacobian without the quadratic term": (
        _wrap("quadratic_residual_jacobian", lambda o: lambda res, z: o(_with(res, Q=None), z)),
        gpins.test_full_ggn_vs_autograd),
    # Sec. 3.3: the criterion's Hessian W left out of the loss
    "general loss without the criterion weight": (
        _wrap("loss_general", lambda o: lambda res, ri, rb: o(_with(res, W=None), ri, rb)),
        lambda: gpins.test_residual_and_gradient_vs_autograd(False)),
    # App. B: ties resolved towards the smaller learning rate
    "line search keeping the smaller alpha on ties": (
        ("line_search", lambda o: _ties_keep_smaller_alpha),
        pins.test_line_search_ties_and_nonfinite),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pin_catches_planted_mistake(name, monkeypatch):
    (fn, make), pin = MUTANTS[name]
    monkeypatch.setattr(ko, fn, make(getattr(ko, fn)))
    # the pin fails: a mismatch, or (damping off the diagonal) a factorisation
    # that is no longer positive definite
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        pin()


def test_pins_pass_without_mistakes():
    # the same pins on the unmodified oracle (guards the mutants' harness)
    for _, pin in MUTANTS.values():
        pin()


def test_shifted_line_search_grid_is_caught(monkeypatch):
    # Sec. 3.4 fixes the grid {2^0, .., 2^-30}
    monkeypatch.setattr(ko, "LINE_SEARCH_GRID", tuple(2.0 ** -(k + 1) for k in range(31)))
    with pytest.raises(AssertionError):
        pins.test_line_search_grid_argmin_closed_form()
