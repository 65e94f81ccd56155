"""The full-size step checks (tests/fullsize_checks.py) on the oracle's own
line-search steps at a small size, where they must hold to rounding, and
with planted mistakes, each of which one of them must catch; and the whole
procedure of tests/test_gpu_fullsize.py run against the oracle in place of
the CUDA path."""
import copy
import dataclasses

import numpy as np
import pytest
import torch

import bench
from oracle import kfac_oracle as ko
from synth import inputs as si
from tests import fullsize_checks as fc
from tests.test_gpu_fullsize import run_full_size

PROB = si.PROBLEMS["poisson5d_cos"]
WIDTHS = (12, 10, 1)
N, NB, STEPS = 40, 12, 3
TIGHT = dict(A1=1e-12, BL=1e-12, sym=1e-14, eig=1e-12, dir=1e-12, lb=1e-12, upd_rtol=1e-12, upd_atol=1e-14)


def _oracle_run():
    hyper = bench.HYPER
    cfg = ko.KfacConfig(d=PROB.d, widths=WIDTHS, lam=hyper["lam"], beta=hyper["beta"],
                        momentum=hyper["momentum"], init_identity=hyper["init_identity"], line_search=True)
    state = ko.init_state(cfg)
    theta = si.xavier_theta(PROB.d, WIDTHS, 7)
    batches = [si.make_batch(PROB, N, NB, seed=8, step=k) for k in range(STEPS)]
    thetas = [theta]
    for b in batches:
        res = ko.kfac_step(cfg, state, thetas[-1], *b)
        thetas.append(res.theta_new)
    alpha = res.extras["alpha"]
    factors = {}
    for l in range(len(WIDTHS)):
        for which, mats in zip(fc.WHICH, (state.A_int, state.B_int, state.A_bdy, state.B_bdy)):
            factors[(l + 1, which)] = mats[l]
    obs = dict(theta=thetas, factors=factors, grad=ko.pack_theta(res.grads),
               direction=ko.pack_theta(res.direction), coef=(alpha, alpha * cfg.momentum),
               ls=res.extras["line_search_losses"], loss=np.array(res.loss))
    return obs, batches


@pytest.fixture(scope="module")
def run():
    return _oracle_run()


def test_checks_hold_on_the_oracle(run):
    obs, batches = run
    k = fc.check_step(obs, PROB.d, WIDTHS, bench.HYPER, batches, TIGHT)
    assert 0 <= k <= 30


def _planted(obs, batches):
    """One copy of obs per plausible mistake of a GPU step."""
    L = len(WIDTHS)
    out = {}
    o = copy.deepcopy(obs)                         # factor EMA missing the first step
    o["factors"][(1, "A_int")] = fc.first_layer_factor_ema(batches[1:], bench.HYPER["beta"], True)
    out["A1 ema"] = o
    o = copy.deepcopy(obs)                         # boundary A from the interior points
    o["factors"][(1, "A_bdy")] = o["factors"][(1, "A_int")]
    out["A1 swapped"] = o
    o = copy.deepcopy(obs)                         # seed of the wrong norm
    o["factors"][(L, "B_int")] = 2.0 * o["factors"][(L, "B_int")]
    out["B_L"] = o
    o = copy.deepcopy(obs)                         # an unsymmetric factor
    M = o["factors"][(2, "B_int")].copy()
    M[0, 1] += 1e-3 * np.abs(M).max()
    o["factors"][(2, "B_int")] = M
    out["symmetry"] = o
    o = copy.deepcopy(obs)                         # an indefinite factor
    o["factors"][(2, "A_bdy")] = o["factors"][(2, "A_bdy")] - 2.0 * np.eye(WIDTHS[0] + 1)
    out["eigenvalues"] = o
    o = copy.deepcopy(obs)                         # direction with undamped factors
    G = ko.unpack_theta(o["grad"], PROB.d, WIDTHS)
    f = o["factors"]
    o["direction"] = ko.pack_theta([ko.kron_sum_inverse_apply(f[(l + 1, "A_int")], f[(l + 1, "B_int")],
                                                              f[(l + 1, "A_bdy")], f[(l + 1, "B_bdy")], G[l],
                                                              1e-1, False) for l in range(L)])
    out["damping"] = o
    o = copy.deepcopy(obs)                         # direction without the boundary factors
    o["direction"] = ko.pack_theta([-np.linalg.solve(
        np.kron(f[(l + 1, "A_int")] + 1e-3 * np.eye(f[(l + 1, "A_int")].shape[0]),
                f[(l + 1, "B_int")] + 1e-3 * np.eye(f[(l + 1, "B_int")].shape[0])),
        G[l].reshape(-1, order="F")).reshape(G[l].shape, order="F") for l in range(L)])
    out["boundary curvature"] = o
    o = copy.deepcopy(obs)                         # the smaller step on a tie / wrong grid point
    o["coef"] = (o["coef"][0] / 2, o["coef"][1] / 2)
    out["alpha"] = o
    o = copy.deepcopy(obs)                         # momentum dropped from the update
    o["theta"][-1] = o["theta"][-2] + o["coef"][0] * o["direction"]
    out["momentum"] = o
    o = copy.deepcopy(obs)                         # loss without the 1/2
    o["loss"] = np.array([o["loss"][1] + 2 * o["loss"][2], o["loss"][1], 2 * o["loss"][2]])
    out["loss scale"] = o
    return out


@pytest.mark.parametrize("mistake", ["A1 ema", "A1 swapped", "B_L", "symmetry", "eigenvalues", "damping",
                                     "boundary curvature", "alpha", "momentum", "loss scale"])
def test_checks_catch_planted_mistakes(run, mistake):
    obs, batches = run
    bad = _planted(obs, batches)[mistake]
    with pytest.raises(AssertionError):
        fc.check_step(bad, PROB.d, WIDTHS, bench.HYPER, batches, TIGHT)


class OracleStandIn:
    """The KfacPinn calls of run_full_size, answered by the oracle on the CPU."""

    def __init__(self, d, widths, n_int, n_bdy):
        h = bench.HYPER
        self.cfg = ko.KfacConfig(d=d, widths=tuple(widths), lam=h["lam"], beta=h["beta"], momentum=h["momentum"],
                                 init_identity=h["init_identity"], line_search=True)
        self.state = ko.init_state(self.cfg)
        self.res = None
        self.tuned = False
        self._loss = torch.zeros(3, dtype=torch.float64)

    def set_graph(self, enable):
        pass

    def set_autotune(self, enable):
        self.tuned = bool(enable)

    def tuning(self):
        return [{"kind": 0}] if self.tuned and self.res is not None else []

    def step(self, theta, X_int, f, X_bdy, g):
        self.res = ko.kfac_step(self.cfg, self.state, theta.numpy().copy(), X_int.numpy(), f.numpy(),
                                X_bdy.numpy(), g.numpy())
        theta.copy_(torch.from_numpy(self.res.theta_new))
        self._loss.copy_(torch.tensor(self.res.loss, dtype=torch.float64))
        return self._loss

    def sync_status(self):
        return "KFAC_OK"

    def get_factor(self, layer, which):
        mats = dict(zip(fc.WHICH, (self.state.A_int, self.state.B_int, self.state.A_bdy, self.state.B_bdy)))
        return torch.from_numpy(mats[which][layer - 1].copy())

    def gradient(self):
        return torch.from_numpy(ko.pack_theta(self.res.grads))

    def direction(self):
        return torch.from_numpy(ko.pack_theta(self.res.direction))

    def update_coefficients(self):
        a = self.res.extras["alpha"]
        return torch.tensor([a, a * self.cfg.momentum], dtype=torch.float64)

    def line_search_losses(self):
        return torch.from_numpy(np.asarray(self.res.extras["line_search_losses"], dtype=np.float64))

    def forward_laplacian(self, theta, X):
        Ws = ko.unpack_theta(theta.numpy(), self.cfg.d, self.cfg.widths)
        return tuple(torch.from_numpy(a) for a in ko.forward_laplacian(Ws, np.asarray(X), "laplace"))

    def close(self):
        pass


def test_full_size_procedure_on_the_oracle():
    wl = dataclasses.replace(bench.WORKLOAD, problem=PROB.name, widths=WIDTHS, n_int=N, n_bdy=NB)
    obs = run_full_size(OracleStandIn, wl, "cpu", lambda: None, TIGHT,
                        dict(u=1e-13, grad_u=1e-13, lap_u=1e-13), n_sample=16)
    assert len(obs["theta"]) == 4 and not np.array_equal(obs["theta"][2], obs["theta"][3])
