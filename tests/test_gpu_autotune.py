"""Split-K autotuner (kfac_pinn_set_autotune, kfac_pinn_get_tuning,
kfac_pinn_set_tuning) of the Grams (row chunks) and of the tangent GEMMs of
the Taylor pass and its adjoint (tangent-tile chunks).

A measured chunk length changes only how a launch's work is split among
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
    assert {e["kind"] for e in table} == {0, 1, 2}, table
    for e in table:
        assert 0 < e["us"] <= e["model_us"], e          # the model's length is one of the candidates
        assert e["split"] == (precision == "mixed_split"), e
        if e["kind"] == 0:
            top = -(-e["K"] // 64) * 64
            assert e["tiles"] == 0 and e["sym"] in (0, 1), e
            for c in (e["chunk"], e["model_chunk"]):
                assert c % 64 == 0 and 64 <= c <= top, e
        else:
            # S - 1 tangent and Laplacian tiles forward, S - 2 tangent tiles in the adjoint
            assert e["tiles"] == PROB.d + 2 - e["kind"] and e["sym"] == 0, e
            assert e["P"] == -(-N // 128) * 128 and e["Q"] % 64 == 0 and e["K"] % 64 == 0, e
            for c in (e["chunk"], e["model_chunk"]):
                assert 1 <= c <= e["tiles"] and -(-e["tiles"] // c) <= 16, e
    # symmetric Grams of the factors and the weight-gradient contractions
    assert {e["sym"] for e in table if e["kind"] == 0} == {0, 1}
    # one entry per distinct padded (output, input) width pair of the hidden
    # layers 2..L-1, forward and adjoint (layers of equal padded widths share it)
    h = [-(-w // 64) * 64 for w in (PROB.d,) + WIDTHS]
    pairs = {(h[l], h[l - 1]) for l in range(2, len(WIDTHS))}
    assert {(e["Q"], e["K"]) for e in table if e["kind"] == 1} == pairs
    assert {(e["K"], e["Q"]) for e in table if e["kind"] == 2} == pairs

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
    ok = dict(kind=0, P=64, Q=64, K=7 * 3072, tiles=0, sym=1, split=0, chunk=1024)
    tan = dict(kind=1, P=3072, Q=64, K=64, tiles=6, sym=0, split=0, chunk=3)
    for base, bad in ((ok, dict(chunk=100)), (ok, dict(chunk=0)), (ok, dict(chunk=7 * 3072 + 64)),
                      (ok, dict(sym=2)), (ok, dict(split=-1)), (ok, dict(P=0)), (ok, dict(K=0)),
                      (ok, dict(tiles=3)), (ok, dict(kind=3)), (tan, dict(chunk=0)), (tan, dict(chunk=7)),
                      (tan, dict(tiles=0)), (tan, dict(sym=1)), (dict(tan, kind=2), dict(Q=0))):
        with pytest.raises(KfacError) as ei:
            opt.set_tuning([{**base, **bad}])
        assert ei.value.status == "KFAC_BAD_ARG", (base, bad)
    with pytest.raises(KfacError):
        opt.set_tuning([ok] * 129)                       # more than KFAC_TUNE_CAP entries
    assert opt.tuning() == []                            # a rejected table leaves it unchanged
    opt.set_tuning([ok, tan, dict(tan, kind=2)])
    assert [e["chunk"] for e in opt.tuning()] == [1024, 3, 3]
    opt.set_tuning([])
    assert opt.tuning() == []

    # 64-row chunks of the interior Grams would need hundreds of partial sums
    # (the workspace holds 32) and one-tile chunks of the 7-tile tangent
    # GEMMs are within the 16 the workspace holds, so take the interior Grams
    # only: ignored at launch; every other shape keeps the model's length
    th0 = si.xavier_theta(PROB.d, WIDTHS, 2)
    Xi, f, Xb, g = si.make_batch(PROB, N, NB, seed=2)
    ref = _opt("mixed_bf16")
    tr = torch.tensor(th0, device=DEV)
    ref.step(tr, Xi, f, Xb, g)
    probe = _opt("mixed_bf16")
    probe.set_autotune(True)
    probe.step(torch.tensor(th0, device=DEV), Xi, f, Xb, g)
    torch.cuda.synchronize()
    huge = [{**e, "chunk": 64 if e["kind"] == 0 and -(-e["K"] // 64) > 32 else e["model_chunk"]}
            for e in probe.tuning()]
    assert sum(e["chunk"] == 64 for e in huge) >= 4
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
