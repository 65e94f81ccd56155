"""Per-result relative error of one KFAC step against the FP64 oracle, for
both precisions on the configurations the oracle finishes in seconds (the
2-d, 5-d and heat workloads at their full point counts; the 100-d net on a
small batch).  Run with -s to print the table; the assertions are the
per-result bounds of each precision:

  FP64:  forward outputs, loss, gradient and factors to 1e-10, the
         preconditioned direction and the update to 1e-8;
  mixed_bf16: u and the loss to 1e-3 (split-BF16 value channel), the
         tangents, Laplacian, gradient and factors to 2e-2 (BF16 tangent and
         adjoint channels, 8 significant bits); the update is reported, since
         the damped inverse amplifies factor errors by up to ||dA|| / lambda;
  mixed_split (split-BF16 on every channel, about 16 bits): every forward
         output, the loss, the gradient and the factors to 1e-4, the update
         to 1e-3 on the Poisson problems and 5e-3 on the heat problem, whose
         damped inverse amplifies the factor differences about 330-fold.
"""
import numpy as np
import pytest
import torch

from oracle import kfac_oracle as ko
from synth import inputs as si

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CONFIGS = [
    ("C1 poisson2d 2-32-32-1 900/120", si.PROBLEMS["poisson2d_sin"], (32, 32, 1), 900, 120),
    ("C2 poisson5d 5-64-64-48-48-1 3000/500", si.PROBLEMS["poisson5d_cos"], (64, 64, 48, 48, 1), 3000, 500),
    ("C4 heat4d 5-128-128-64-1 4000/1000", si.PROBLEMS["heat4d_sin"], (128, 128, 64, 1), 4000, 1000),
    ("C3 poisson100d 100-768-768-512-512-1 64/32", si.PROBLEMS["poisson100d_norm"], (768, 768, 512, 512, 1), 64, 32),
]
KEYS = ["u", "grad_u", "lap_u", "loss", "gradient", "A_int", "B_int", "A_bdy", "B_bdy", "direction", "update"]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def errors(prob, widths, N, Nb, precision):
    from paper_2405_15603_gb300.api import KfacPinn
    kw = dict(lam=1e-3, lr=0.1, beta=0.0)
    th0 = si.xavier_theta(prob.d, widths, 0)
    Xi, f, Xb, g = si.make_batch(prob, N, Nb, seed=0)
    opt = KfacPinn(prob.d, widths, device=DEV, precision=precision, op=prob.op, kappa=prob.kappa,
                   max_n_int=N, max_n_bdy=Nb, **kw)
    theta = torch.tensor(th0, device=DEV)
    u, gu, lap = (t.cpu().numpy() for t in opt.forward_laplacian(theta, Xi))
    loss = opt.step(theta, Xi, f, Xb, g).cpu().numpy()
    torch.cuda.synchronize()
    out = {}
    ru, rg, rl = ko.forward_laplacian(ko.unpack_theta(th0, prob.d, widths), Xi, prob.op)
    cfg = ko.KfacConfig(d=prob.d, widths=widths, op=prob.op, kappa=prob.kappa, **kw)
    st = ko.init_state(cfg)
    res = ko.kfac_step(cfg, st, th0, Xi, f, Xb, g)
    out["u"], out["grad_u"], out["lap_u"] = rel(u, ru), rel(gu, rg), rel(lap, rl)
    out["loss"] = rel(loss, np.array(res.loss))
    out["gradient"] = rel(opt.gradient().cpu().numpy(), ko.pack_theta(res.grads))
    for which, refs in (("A_int", st.A_int), ("B_int", st.B_int), ("A_bdy", st.A_bdy), ("B_bdy", st.B_bdy)):
        out[which] = max(rel(opt.get_factor(l, which).cpu(), refs[l - 1]) for l in range(1, len(widths) + 1))
    out["direction"] = rel(opt.direction().cpu().numpy(), ko.pack_theta(res.direction))
    out["update"] = rel(theta.cpu().numpy() - th0, res.theta_new - th0)
    assert opt.sync_status() == "KFAC_OK"
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16", "mixed_split"])
def test_error_report(precision):
    print()
    print(f"relative error per result, {precision}, one step, lambda = 1e-3 (factors: max over the layers)")
    print("config".ljust(46) + "".join(k.rjust(11) for k in KEYS))
    rows = []
    for name, prob, widths, N, Nb in CONFIGS:
        e = errors(prob, widths, N, Nb, precision)
        print(name.ljust(46) + "".join(f"{e[k]:11.2e}" for k in KEYS), flush=True)
        rows.append((name, e))
    for name, e in rows:
        if precision == "fp64":
            for k in KEYS[:9]:
                assert e[k] < 1e-10, (name, k, e[k])
            assert e["direction"] < 1e-8 and e["update"] < 1e-8, (name, e)
        elif precision == "mixed_split":
            for k in KEYS[:9]:
                assert e[k] < 1e-4, (name, k, e[k])
            # the update is the damped Kronecker-sum inverse applied to the
            # gradient: at lambda = 1e-3 it amplifies the ~1e-5 factor
            # differences by up to ~330 on the heat problem (measured: update
            # error / factor error), so 1e-3 holds on the Poisson problems
            # and 5e-3 bounds the heat problem
            assert e["update"] < (5e-3 if name.startswith("C4") else 1e-3), (name, e["update"])
        else:
            assert e["u"] < 1e-3 and e["loss"] < 1e-3, (name, e)
            for k in ("grad_u", "lap_u", "gradient", "A_int", "B_int", "A_bdy", "B_bdy"):
                assert e[k] < 2e-2, (name, k, e[k])
            assert np.isfinite(e["update"])
