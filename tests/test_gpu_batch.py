"""Batched stepping of many independent problems (worker streams, CUDA graph
capture and replay) gives the same parameters as stepping each problem on its
own, for every update rule and both precisions."""
import numpy as np
import pytest
import torch

from synth import inputs as si

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _members():
    return [si.BatchMember(2, (32, 32, 1), 300, 60), si.BatchMember(5, (64, 48, 1), 517, 130),
            si.BatchMember(10, (128, 64, 32, 1), 211, 53), si.BatchMember(20, (32, 256, 1), 400, 100),
            si.BatchMember(7, (40, 72, 1), 67, 13)]


def _make(members, precision, update):
    from paper_2405_15603_gb300.api import KfacPinn
    kw = dict(lam=1e-3, beta=0.9, lr=0.05, momentum=0.5, init_identity=True, update=update, eig_sm_budget=30)
    return [KfacPinn(m.d, m.widths, device=DEV, precision=precision, max_n_int=m.n_int, max_n_bdy=m.n_bdy, **kw)
            for m in members]


@pytest.mark.parametrize("precision,update", [("fp64", "fixed"), ("mixed_bf16", "line_search"),
                                              ("fp64", "kfac_star")])
def test_batch_matches_individual_steps(precision, update):
    from paper_2405_15603_gb300.api import KfacBatch
    members = _members()
    solo = _make(members, precision, update)
    batched = _make(members, precision, update)
    th0 = [torch.tensor(si.xavier_theta(m.d, m.widths, i), device=DEV) for i, m in enumerate(members)]
    th_solo = [t.clone() for t in th0]
    th_b = [t.clone() for t in th0]
    # fixed input buffers (the graph replays read from the same addresses)
    bufs = [[torch.empty(m.n_int, m.d, dtype=torch.float64, device=DEV),
             torch.empty(m.n_int, dtype=torch.float64, device=DEV),
             torch.empty(m.n_bdy, m.d, dtype=torch.float64, device=DEV),
             torch.empty(m.n_bdy, dtype=torch.float64, device=DEV)] for m in members]
    losses = [torch.zeros(3, dtype=torch.float64, device=DEV) for _ in members]
    batch = KfacBatch(batched, n_streams=3)
    for step in range(4):                     # eager, capture, replay, replay
        for i, m in enumerate(members):
            arrs = si.make_batch(m.prob, m.n_int, m.n_bdy, seed=i, step=step)
            for b, a in zip(bufs[i], arrs):
                b.copy_(torch.from_numpy(a))
            solo[i].step(th_solo[i], *bufs[i])
        batch.step(th_b, [b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs],
                   [b[3] for b in bufs], losses)
        torch.cuda.synchronize()
        for i in range(len(members)):
            assert torch.equal(th_b[i], th_solo[i]), (step, i)
    for opt in solo + batched:
        assert opt.sync_status() == "KFAC_OK"
    batch.close()


def test_batch_rejects_bad_arguments():
    from paper_2405_15603_gb300.api import KfacBatch, KfacError
    members = _members()[:2]
    opts = _make(members, "fp64", "fixed")
    with pytest.raises(KfacError):
        KfacBatch(opts, n_streams=0)
    batch = KfacBatch(opts, n_streams=2)
    too_many = [torch.zeros(m.n_int + 1, m.d, dtype=torch.float64, device=DEV) for m in members]
    small = [torch.zeros(m.n_int, dtype=torch.float64, device=DEV) for m in members]
    xb = [torch.zeros(m.n_bdy, m.d, dtype=torch.float64, device=DEV) for m in members]
    gb = [torch.zeros(m.n_bdy, dtype=torch.float64, device=DEV) for m in members]
    th = [torch.zeros(o.D, dtype=torch.float64, device=DEV) for o in opts]
    with pytest.raises(KfacError):
        batch.step(th, too_many, small, xb, gb)
    batch.close()


@pytest.mark.parametrize("precision,update", [("mixed_bf16", "line_search"), ("fp64", "kfac_star"),
                                              ("fp64", "fixed")])
def test_single_handle_graph_mode_is_bit_identical(precision, update):
    # kfac_pinn_set_graph: eager first step, captured second, replays after;
    # batches in fresh device tensors every step (staged by the library) and
    # through step_host, against plain eager steps
    from paper_2405_15603_gb300.api import KfacPinn
    prob = si.PROBLEMS["poisson5d_cos"]
    widths = (48, 40, 1)
    kw = dict(device=DEV, precision=precision, update=update, max_n_int=150, max_n_bdy=50, lam=1e-3,
              lr=0.1, momentum=0.3, beta=0.9, init_identity=True)
    eager, graph = KfacPinn(prob.d, widths, **kw), KfacPinn(prob.d, widths, **kw)
    graph.set_graph(True)
    th0 = si.xavier_theta(prob.d, widths, 4)
    te, tg = torch.tensor(th0, device=DEV), torch.tensor(th0, device=DEV)
    for step in range(5):
        Xi, f, Xb, g = si.make_batch(prob, 150 - 10 * (step == 4), 50, seed=2, step=step)
        le = eager.step(te, Xi, f, Xb, g).clone()
        n0 = graph.launch_count()
        if step == 3:
            lh = graph.step_host(tg, Xi, f, Xb, g)
            lg = torch.tensor(lh, device=DEV)
        else:
            lg = graph.step(tg, *(torch.tensor(a, device=DEV) for a in (Xi, f, Xb, g))).clone()
        torch.cuda.synchronize()
        assert graph.launch_count() > n0
        assert torch.equal(te, tg), step
        assert torch.equal(le, lg), step
    assert eager.sync_status() == "KFAC_OK" and graph.sync_status() == "KFAC_OK"


@pytest.mark.parametrize("precision,update", [("mixed_split", "fixed"), ("mixed_split", "line_search"),
                                              ("mixed_bf16", "kfac_star")])
def test_grouped_batch_matches_individual_steps(precision, update):
    # grouped form: every kernel launched once for all members (member tables),
    # one batched eigensolve; bit-identical to each problem stepped on its own
    from paper_2405_15603_gb300.api import KfacBatch
    members = _members()
    solo = _make(members, precision, update)
    batched = _make(members, precision, update)
    th0 = [torch.tensor(si.xavier_theta(m.d, m.widths, i), device=DEV) for i, m in enumerate(members)]
    th_solo = [t.clone() for t in th0]
    th_b = [t.clone() for t in th0]
    bufs = [[torch.empty(m.n_int, m.d, dtype=torch.float64, device=DEV),
             torch.empty(m.n_int, dtype=torch.float64, device=DEV),
             torch.empty(m.n_bdy, m.d, dtype=torch.float64, device=DEV),
             torch.empty(m.n_bdy, dtype=torch.float64, device=DEV)] for m in members]
    losses = [torch.zeros(3, dtype=torch.float64, device=DEV) for _ in members]
    solo_losses = []
    batch = KfacBatch(batched, n_streams=3, grouped=True)
    assert batch.launches_per_step() is None
    for step in range(4):                     # eager, record + capture, replay, replay
        solo_losses = []
        for i, m in enumerate(members):
            arrs = si.make_batch(m.prob, m.n_int, m.n_bdy, seed=i, step=step)
            for b, a in zip(bufs[i], arrs):
                b.copy_(torch.from_numpy(a))
            solo_losses.append(solo[i].step(th_solo[i], *bufs[i]).clone())
        batch.step(th_b, [b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs],
                   [b[3] for b in bufs], losses)
        torch.cuda.synchronize()
        for i in range(len(members)):
            assert torch.equal(th_b[i], th_solo[i]), (step, i)
            assert torch.equal(losses[i], solo_losses[i]), (step, i)
    for opt in solo + batched:
        assert opt.sync_status() == "KFAC_OK"
    grouped_launches = batch.launches_per_step()
    batch.close()
    # the same problems in the stream form launch every handle's kernels
    streams = KfacBatch(batched, n_streams=3)
    for _ in range(2):
        streams.step(th_b, [b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs],
                     [b[3] for b in bufs], losses)
    torch.cuda.synchronize()
    assert 0 < grouped_launches < streams.launches_per_step() / 2
    streams.close()


def test_grouped_batch_launches_do_not_grow_with_the_number_of_problems():
    from paper_2405_15603_gb300.api import KfacBatch, KfacError, KfacPinn
    kw = dict(lam=1e-3, beta=0.95, lr=0.05, momentum=0.0, init_identity=True, update="fixed", eig_sm_budget=19)
    members = si.many_pinns(64, seed=0)
    counts = {}
    for n in (8, 64):
        opts = [KfacPinn(m.d, m.widths, device=DEV, precision="mixed_split", max_n_int=m.n_int,
                         max_n_bdy=m.n_bdy, **kw) for m in members[:n]]
        th = [torch.tensor(si.xavier_theta(m.d, m.widths, i), device=DEV) for i, m in enumerate(members[:n])]
        bufs = [[torch.tensor(a, device=DEV) for a in si.make_batch(m.prob, m.n_int, m.n_bdy, seed=i)]
                for i, m in enumerate(members[:n])]
        batch = KfacBatch(opts, n_streams=8, grouped=True)
        for _ in range(3):
            batch.step(th, *[[b[j] for b in bufs] for j in range(4)])
        torch.cuda.synchronize()
        counts[n] = batch.launches_per_step()
        assert all(o.sync_status() == "KFAC_OK" for o in opts)
        assert all(bool(torch.isfinite(t).all()) for t in th)
        batch.close()
        for o in opts:
            o.close()
    assert counts[64] < 500, counts
    assert counts[64] <= counts[8] + 40, counts
    # the grouped form needs the tensor-core precisions
    fp = [KfacPinn(2, (16, 1), device=DEV, precision="fp64", max_n_int=32, max_n_bdy=8)]
    with pytest.raises(KfacError):
        KfacBatch(fp, n_streams=1, grouped=True)
