"""Failure detection without a GPU fault.

* Device: each bounded wait of the library (the eigensolver's group barrier,
  the tcgen05 engine's mbarrier wait) is run against a condition that nothing
  satisfies with a 50 ms limit; the kernel must give up, latch KFAC_TIMEOUT
  in the handle's status word and return, and the context must stay usable
  (a KFAC step afterwards is clean).
* Host: an injected out-of-memory at every device allocation of
  kfac_pinn_create in turn must return KFAC_OOM and leave the device's free
  memory where it was (nothing leaked).
"""
import time

import numpy as np
import pytest
import torch

from synth import inputs as si

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _opt(precision, **kw):
    from paper_2405_15603_gb300.api import KfacPinn
    return KfacPinn(3, (24, 16, 1), device=DEV, precision=precision, max_n_int=40, max_n_bdy=10, **kw)


@pytest.mark.parametrize("kind", ["group_barrier", "mbarrier"])
def test_bounded_wait_gives_up_and_reports_timeout(kind):
    opt = _opt("mixed_split")
    assert opt.sync_status() == "KFAC_OK"
    t0 = time.perf_counter()
    opt.check_wait_timeout(kind, limit_ms=50)
    dt = time.perf_counter() - t0
    assert 0.05 <= dt < 1.9, dt          # gave up after its own limit, not the 2 s default
    assert opt.sync_status() == "KFAC_TIMEOUT"
    assert opt.sync_status() == "KFAC_OK"   # reading clears the word
    # the context is still usable: a step of the same handle is clean
    prob = si.poisson_cos_problem(3)
    Xi, f, Xb, g = si.make_batch(prob, 40, 10, seed=1)
    th = torch.tensor(si.xavier_theta(3, (24, 16, 1), 1), device=DEV)
    loss = opt.step(th, Xi, f, Xb, g)
    torch.cuda.synchronize()
    assert opt.sync_status() == "KFAC_OK"
    assert torch.isfinite(loss).all() and torch.isfinite(th).all()


@pytest.mark.parametrize("precision", ["fp64", "mixed_split"])
def test_injected_out_of_memory_in_create_leaks_nothing(precision):
    from paper_2405_15603_gb300.api import KfacError, inject_alloc_failure
    warm = _opt(precision, update="kfac_star")      # loads the kernels, creates the streams once
    warm.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    try:
        for n in range(4000):
            inject_alloc_failure(n)
            try:
                opt = _opt(precision, update="kfac_star")
            except KfacError as e:
                assert e.status == "KFAC_OOM", (n, e.status)
                failures += 1
                torch.cuda.synchronize()
                assert abs(torch.cuda.mem_get_info()[0] - free0) <= 2 << 20, n
                continue
            opt.close()       # n is past the last allocation: create succeeded
            break
        else:
            pytest.fail("create never succeeded")
    finally:
        inject_alloc_failure(-1)
    assert failures >= 10                    # every allocation of create was exercised
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 2 << 20
