"""The allocation-free forward Laplacian against the handle-based one.

kfac_pinn_forward_laplacian_noalloc exists for callers that cannot allocate
device memory while they run (code inside another runtime's memory pool or
fixed device-memory budget, or a process that must not grow after start-up):
it evaluates u, grad u and the Laplacian using only a fixed scratch array
compiled into the library.  This test calls it through the C-ABI twice in a
row (the scratch array is shared and reused between calls) and compares each
result with kfac_pinn_forward_laplacian on an FP64 handle, to the FP64 parity
tolerance of the other tests.  It is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import inputs as si

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_forward_laplacian_matches_handle_path_twice():
    from paper_2405_15603_gb300 import build, _lib
    from paper_2405_15603_gb300.api import KfacPinn, make_config
    build.build()
    lib = _lib.load()
    prob = si.PROBLEMS["poisson5d_cos"]
    widths = (64, 48, 1)
    N = 333
    cfg = make_config(prob.d, widths, max_n_int=N, max_n_bdy=4)
    ref = KfacPinn(prob.d, widths, device=DEV, max_n_int=N, max_n_bdy=4)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        theta = torch.tensor(si.xavier_theta(prob.d, widths, 10 + call), device=DEV)
        X = torch.tensor(si.sample_interior(N, prob.d, np.random.default_rng(call)), device=DEV)
        u_ref, g_ref, lap_ref = ref.forward_laplacian(theta, X)
        u = torch.full((N,), np.nan, dtype=torch.float64, device=DEV)
        g = torch.full((N, prob.d), np.nan, dtype=torch.float64, device=DEV)
        lap = torch.full((N,), np.nan, dtype=torch.float64, device=DEV)
        st = lib.kfac_pinn_forward_laplacian_noalloc(C.byref(cfg), stream, theta.data_ptr(), X.data_ptr(), N,
                                                     u.data_ptr(), g.data_ptr(), lap.data_ptr())
        assert st == 0, _lib.STATUS.get(st, st)
        torch.cuda.synchronize()
        assert rel(u.cpu(), u_ref.cpu()) < 1e-10
        assert rel(g.cpu(), g_ref.cpu()) < 1e-10
        assert rel(lap.cpu(), lap_ref.cpu()) < 1e-10
    # A request beyond the fixed scratch capacity is refused without running.
    big = make_config(100, (1023, 1023, 1), max_n_int=1, max_n_bdy=1)
    st = lib.kfac_pinn_forward_laplacian_noalloc(C.byref(big), stream, theta.data_ptr(), X.data_ptr(), 4096,
                                                 u.data_ptr(), None, None)
    assert st == 1   # KFAC_BAD_ARG
    ref.close()
