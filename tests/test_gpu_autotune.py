"""Gram tile autotuner (kfac_pinn_set_autotune, kfac_pinn_get_tuning,
kfac_pinn_set_tuning).

A measured row-chunk length changes only how a Gram's K rows are split among
CTAs, i.e. the order in which FP32 partial sums are added.  So:
  * an autotuned step still matches the FP64 oracle within the bounds of its
    precision (mixed_bf16: 2e-2 on gradient and factors; mixed_split: 1e-4);
  * the step that measures computes with the length it records, so a second
    handle given the same table reproduces it bit for bit, eagerly and as a
    replayed CUDA graph;
  * malformed tables are rejected, and an entry whose chunk count does not
    fit the partial-sum workspace falls back to the wave model (bit-identical
    to a handle without a table).
"""
import numpy as np
import pytest
import torch

from oracle import kfac_oracle as ko
from synth import inputs as si

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

PROB = si.PROBLEMS["poisson5d_cos"]
WIDTHS = (64, 64, 48, 48, 1)
N, NB = 3000, 500
KW = dict(lam=1e-3, lr=0.1, beta=0.0)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _opt(precision, **kw):
    from paper_2405_15603_gb300.api import KfacPinn
    return KfacPinn(PROB.d, WIDTHS, device=DEV, precision=precision, max_n_int=N, max_n_bdy=NB,
                    **{**KW, **kw})


def _factors(opt):
    return [opt.get_factor(l, w).cpu().numpy() for l in range(1, len(WIDTHS) + 1)
            for w in ("A_int", "B_int", "A_bdy", "B_bdy")]


@pytest.mark.parametrize("precision,tol", [("mixed_bf16", 2e-2), ("mixed_split", 1e-4)])
def test_autotuned_step_matches_oracle(precision, tol):
    th0 = si.xavier_theta(PROB.d, WIDTHS, 0)
    Xi, f, Xb, g = si.make_batch(PROB, N, NB, seed=0)
    opt = _opt(precision)
    opt.set_autotune(True)
    theta = torch.tensor(th0, device=DEV)
    loss = opt.step(theta, Xi, f, Xb, g).cpu().numpy()
    torch.cuda.synchronize()
    assert opt.sync_status() == "KFAC_OK"
    table = opt.tuning()
    assert table, "no Gram shape was measured"
    for e in table:
        top = -(-e["rows"] // 64) * 64
        assert e["row_chunk"] % 64 == 0 and 64 <= e["row_chunk"] <= top, e
        assert e["model_row_chunk"] % 64 == 0 and 64 <= e["model_row_chunk"] <= top, e
        assert 0 < e["us"] <= e["model_us"], e          # the model's length is one of the candidates
        assert e["split"] == (precision == "mixed_split"), e
        assert e["sym"] in (0, 1)
    # symmetric Grams of the factors and the weight-gradient contractions
    assert {e["sym"] for e in table} == {0, 1}

    cfg = ko.KfacConfig(d=PROB.d, widths=WIDTHS, op=PROB.op, kappa=PROB.kappa, **KW)
    st = ko.init_state(cfg)
    res = ko.kfac_step(cfg, st, th0, Xi, f, Xb, g)
    assert rel(loss, np.array(res.loss)) < 1e-3
    assert rel(opt.gradient().cpu().numpy(), ko.pack_theta(res.grads)) < tol
    for which, refs in (("A_int", st.A_int), ("B_int", st.B_int), ("A_bdy", st.A_bdy), ("B_bdy", st.B_bdy)):
        for l in range(1, len(WIDTHS) + 1):
            assert rel(opt.get_factor(l, which).cpu(), refs[l - 1]) < tol, (which, l)


def test_copied_table_reproduces_the_measuring_step():
    th0 = si.xavier_theta(PROB.d, WIDTHS, 1)
    batches = [si.make_batch(PROB, N, NB, seed=1, step=k) for k in range(4)]
    tuned = _opt("mixed_bf16", update="line_search", momentum=0.3)
    tuned.set_autotune(True)
    ta = torch.tensor(th0, device=DEV)
    tuned.step(ta, *batches[0])
    torch.cuda.synchronize()
    table = tuned.tuning()
    assert table
    # eager copy and graph-mode copy of the table
    eager, graph = _opt("mixed_bf16", update="line_search", momentum=0.3), \
        _opt("mixed_bf16", update="line_search", momentum=0.3)
    eager.set_tuning(table)
    graph.set_tuning(table)
    graph.set_graph(True)
    tb, tg = torch.tensor(th0, device=DEV), torch.tensor(th0, device=DEV)
    eager.step(tb, *batches[0])
    graph.step(tg, *(torch.tensor(a, device=DEV) for a in batches[0]))
    torch.cuda.synchronize()
    assert torch.equal(ta, tb) and torch.equal(ta, tg)
    for fa, fb in zip(_factors(tuned), _factors(eager)):
        assert np.array_equal(fa, fb)
    for k in range(1, 4):                 # measured shapes are not measured again
        tuned.step(ta, *batches[k])
        graph.step(tg, *(torch.tensor(a, device=DEV) for a in batches[k]))
        torch.cuda.synchronize()
        assert torch.equal(ta, tg), k
    assert len(tuned.tuning()) == len(table)
    # the copied entries carry no measurements
    assert all(e["us"] == 0 and e["model_us"] == 0 for e in graph.tuning())
    for o in (tuned, eager, graph):
        assert o.sync_status() == "KFAC_OK"


def test_set_tuning_validation_and_workspace_fallback():
    from paper_2405_15603_gb300.api import KfacError
    opt = _opt("mixed_bf16")
    ok = dict(P=64, Q=64, rows=7 * 3072, sym=1, split=0, row_chunk=1024)
    for bad in (dict(row_chunk=100), dict(row_chunk=0), dict(row_chunk=7 * 3072 + 64), dict(sym=2),
                dict(split=-1), dict(P=0), dict(rows=0)):
        with pytest.raises(KfacError) as ei:
            opt.set_tuning([{**ok, **bad}])
        assert ei.value.status == "KFAC_BAD_ARG", bad
    with pytest.raises(KfacError):
        opt.set_tuning([ok] * 129)                       # more than KFAC_TUNE_CAP entries
    assert opt.tuning() == []                            # a rejected table leaves it unchanged
    opt.set_tuning([ok])
    assert len(opt.tuning()) == 1 and opt.tuning()[0]["row_chunk"] == 1024
    opt.set_tuning([])
    assert opt.tuning() == []

    # 64-row chunks of the interior Grams would need hundreds of partial sums
    # (the workspace holds 32): ignored at launch; the boundary Grams keep the
    # model's length
    th0 = si.xavier_theta(PROB.d, WIDTHS, 2)
    Xi, f, Xb, g = si.make_batch(PROB, N, NB, seed=2)
    ref = _opt("mixed_bf16")
    tr = torch.tensor(th0, device=DEV)
    ref.step(tr, Xi, f, Xb, g)
    probe = _opt("mixed_bf16")
    probe.set_autotune(True)
    probe.step(torch.tensor(th0, device=DEV), Xi, f, Xb, g)
    torch.cuda.synchronize()
    huge = [{**e, "row_chunk": 64 if -(-e["rows"] // 64) > 32 else e["model_row_chunk"]}
            for e in probe.tuning()]
    assert sum(e["row_chunk"] == 64 for e in huge) >= 4
    fb = _opt("mixed_bf16")
    fb.set_tuning(huge)
    tf = torch.tensor(th0, device=DEV)
    fb.step(tf, Xi, f, Xb, g)
    torch.cuda.synchronize()
    assert torch.equal(tr, tf)
    for o in (opt, ref, probe, fb):
        assert o.sync_status() == "KFAC_OK"


def test_fp64_handle_has_no_tuned_launches():
    opt = _opt("fp64")
    opt.set_autotune(True)
    Xi, f, Xb, g = si.make_batch(PROB, 200, 50, seed=3)
    opt.step(torch.tensor(si.xavier_theta(PROB.d, WIDTHS, 3), device=DEV), Xi, f, Xb, g)
    torch.cuda.synchronize()
    assert opt.tuning() == []
    assert opt.sync_status() == "KFAC_OK"
