"""Thin Python binding of the C-ABI: argument marshalling only.

torch supplies device memory and the current CUDA stream; every step of the
KFAC path runs in libkfacpinn.so.  Names follow the C entry points.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from . import _lib
from ._lib import KfacConfig, KfacError

OPS = {"laplace": 0, "heat": 1, "general": 2}
PRECISIONS = {"fp64": 0, "mixed_bf16": 1, "mixed_split": 2, "fp32": 3}
VARIANTS = {"expand": 0, "reduce": 1}
FACTORS = {"A_int": 0, "B_int": 1, "A_bdy": 2, "B_bdy": 3}
UPDATES = {"fixed": 0, "line_search": 1, "kfac_star": 2}


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _check(fn: str, code: int):
    if code != 0:
        raise KfacError(fn, code)


def _dev(x, device) -> torch.Tensor:
    t = torch.as_tensor(x, dtype=torch.float64, device=device)
    return t.contiguous()


def make_config(d: int, widths: Sequence[int], op: str = "laplace", kappa: float = 0.0,
                precision: str = "fp64", variant: str = "expand", beta: float = 0.0,
                lam: float = 1e-3, damping_sqrt: bool = False, init_identity: bool = False,
                lr: float = 0.1, momentum: float = 0.0, max_n_int: int = 1024,
                max_n_bdy: int = 1024, line_search: bool = False, update: str = "fixed",
                eig_sm_budget: int = 0, op_coef=None, residual=None) -> KfacConfig:
    """line_search=True is shorthand for update="line_search".  op="general" takes
    the symmetric d x d coefficient matrix op_coef (kept alive on the config).
    residual: a general interior residual (Sec. 3.3) as a dict with "b" (M x S),
    optional "Q" (M x S x S) and "W" (M x M); see kfac_residual_t."""
    cfg = KfacConfig()
    cfg.d = d
    cfg.L = len(widths)
    for i, w in enumerate(widths):
        cfg.widths[i] = int(w)
    cfg.op = OPS[op]
    cfg.kappa = kappa
    cfg.precision = PRECISIONS[precision]
    cfg.variant = VARIANTS[variant]
    cfg.beta = beta
    cfg.lambda_ = lam
    cfg.damping_sqrt = int(damping_sqrt)
    cfg.factor_init_identity = int(init_identity)
    cfg.lr = lr
    cfg.momentum = momentum
    cfg.max_n_int = max_n_int
    cfg.max_n_bdy = max_n_bdy
    cfg.update = UPDATES["line_search" if line_search else update]
    cfg.eig_sm_budget = eig_sm_budget
    if op_coef is not None:
        arr = np.ascontiguousarray(op_coef, dtype=np.float64)
        cfg._op_coef_keepalive = arr
        cfg.op_coef = arr.ctypes.data
    if residual is not None:
        res = _lib.KfacResidual()
        keep = []
        b = np.ascontiguousarray(residual["b"], dtype=np.float64)
        res.M = b.shape[0]
        res.b = b.ctypes.data
        keep.append(b)
        for key in ("Q", "W"):
            if residual.get(key) is not None:
                arr = np.ascontiguousarray(residual[key], dtype=np.float64)
                setattr(res, key, arr.ctypes.data)
                keep.append(arr)
        cfg._residual_keepalive = (res, keep)
        cfg.residual = C.addressof(res)
    return cfg


def param_count(d: int, widths: Sequence[int]) -> int:
    lib = _lib.load()
    return int(lib.kfac_pinn_param_count(C.byref(make_config(d, widths))))


class KfacPinn:
    """One KFAC optimiser state (factors, inverses, momentum) on one GPU."""

    def __init__(self, d: int, widths: Sequence[int], device: str = "cuda", **kw):
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.d = d
        self.widths = tuple(int(w) for w in widths)
        self.cfg = make_config(d, widths, **kw)
        self.h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check("kfac_pinn_create", self.lib.kfac_pinn_create(C.byref(self.cfg), C.byref(self.h)))
        self.D = int(self.lib.kfac_pinn_param_count(C.byref(self.cfg)))
        self._loss = torch.zeros(3, dtype=torch.float64, device=self.device)

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if self.h:
            self.lib.kfac_pinn_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        _check("kfac_pinn_reset", self.lib.kfac_pinn_reset(self.h, _stream()))

    # -- the hot path -----------------------------------------------------
    def forward_laplacian(self, theta: torch.Tensor, X) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
        X = _dev(X, self.device)
        N = X.shape[0]
        u = torch.empty(N, dtype=torch.float64, device=self.device)
        g = torch.empty(N, self.d, dtype=torch.float64, device=self.device)
        lap = torch.empty(N, dtype=torch.float64, device=self.device)
        _check("kfac_pinn_forward_laplacian", self.lib.kfac_pinn_forward_laplacian(
            self.h, _stream(), _ptr(theta), _ptr(X), N, _ptr(u), _ptr(g), _ptr(lap)))
        return u, g, lap

    def forward_laplacian_backward(self, theta: torch.Tensor, X, du=None, dgrad=None, dlap=None,
                                   need_dX: bool = False):
        """dphi/dtheta (and dphi/dX) for upstream gradients of (u, grad u, lap u)."""
        X = _dev(X, self.device)
        N = X.shape[0]
        ups = [None if t is None else _dev(t, self.device) for t in (du, dgrad, dlap)]
        dtheta = torch.empty(self.D, dtype=torch.float64, device=self.device)
        dX = torch.empty(N, self.d, dtype=torch.float64, device=self.device) if need_dX else None
        _check("kfac_pinn_forward_laplacian_backward", self.lib.kfac_pinn_forward_laplacian_backward(
            self.h, _stream(), _ptr(theta.detach().contiguous()), _ptr(X), N, _ptr(ups[0]), _ptr(ups[1]),
            _ptr(ups[2]), _ptr(dtheta), _ptr(dX)))
        return dtheta, dX

    def set_store_forward(self, enable: bool = True):
        """Reverse mode reuses the last forward pass's activations (same theta, X) instead of recomputing."""
        _check("kfac_pinn_set_store_forward", self.lib.kfac_pinn_set_store_forward(self.h, int(enable)))

    def set_cta_pairs(self, enable: bool = True):
        """Forward layer GEMMs of the tensor-core precisions on CTA pairs
        (kfac_pinn_set_cta_pairs; off by default; the same products in the same order)."""
        _check("kfac_pinn_set_cta_pairs", self.lib.kfac_pinn_set_cta_pairs(self.h, int(enable)))

    def set_graph(self, enable: bool = True):
        """Run step / step_host as a captured CUDA graph (kfac_pinn_set_graph):
        the batch is staged into the handle's buffers, the second step is
        captured and later ones replay it; results are bit-identical."""
        _check("kfac_pinn_set_graph", self.lib.kfac_pinn_set_graph(self.h, int(enable)))

    def set_autotune(self, enable: bool = True):
        """Time candidate split-K chunk lengths of each new Gram and tangent
        GEMM shape on the next eager step and keep the fastest
        (kfac_pinn_set_autotune)."""
        _check("kfac_pinn_set_autotune", self.lib.kfac_pinn_set_autotune(self.h, int(enable)))

    def tuning(self) -> list:
        """The handle's tuning table, one dict per launch shape (kind: 0 Gram,
        1 forward tangent GEMM, 2 adjoint tangent GEMM)."""
        n = C.c_int()
        _check("kfac_pinn_get_tuning", self.lib.kfac_pinn_get_tuning(self.h, None, 0, C.byref(n)))
        arr = (_lib.KfacTuneEntry * max(n.value, 1))()
        _check("kfac_pinn_get_tuning", self.lib.kfac_pinn_get_tuning(self.h, arr, n.value, C.byref(n)))
        return [{k: getattr(e, k) for k, _ in _lib.KfacTuneEntry._fields_} for e in arr[:n.value]]

    def set_tuning(self, table: Sequence[dict]):
        """Replace the tuning table (e.g. by another handle's tuning())."""
        arr = (_lib.KfacTuneEntry * max(len(table), 1))()
        for e, t in zip(arr, table):
            for k, _ in _lib.KfacTuneEntry._fields_:
                setattr(e, k, t.get(k, 0))
        _check("kfac_pinn_set_tuning", self.lib.kfac_pinn_set_tuning(self.h, arr, len(table)))

    def factors(self, theta, X_int, f, X_bdy, g) -> torch.Tensor:
        X_int, f, X_bdy, g = (_dev(a, self.device) for a in (X_int, f, X_bdy, g))
        _check("kfac_pinn_factors", self.lib.kfac_pinn_factors(
            self.h, _stream(), _ptr(theta), _ptr(X_int), X_int.shape[0], _ptr(f),
            _ptr(X_bdy), X_bdy.shape[0], _ptr(g), _ptr(self._loss)))
        return self._loss.clone()

    def invert(self):
        _check("kfac_pinn_invert", self.lib.kfac_pinn_invert(self.h, _stream()))

    def precondition(self, grad: Optional[torch.Tensor] = None) -> torch.Tensor:
        out = torch.empty(self.D, dtype=torch.float64, device=self.device)
        _check("kfac_pinn_precondition", self.lib.kfac_pinn_precondition(
            self.h, _stream(), _ptr(grad), _ptr(out)))
        return out

    def update(self, theta: torch.Tensor):
        _check("kfac_pinn_update", self.lib.kfac_pinn_update(self.h, _stream(), _ptr(theta)))

    def step(self, theta: torch.Tensor, X_int, f, X_bdy, g, loss: Optional[torch.Tensor] = None):
        """One KFAC step in place on theta; inputs must already be device tensors
        for the timed path (no copies are made for contiguous FP64 CUDA tensors)."""
        X_int, f, X_bdy, g = (_dev(a, self.device) for a in (X_int, f, X_bdy, g))
        out = self._loss if loss is None else loss
        _check("kfac_pinn_step", self.lib.kfac_pinn_step(
            self.h, _stream(), _ptr(theta), _ptr(X_int), X_int.shape[0], _ptr(f),
            _ptr(X_bdy), X_bdy.shape[0], _ptr(g), _ptr(out)))
        return out

    def step_host(self, theta: torch.Tensor, X_int: np.ndarray, f: np.ndarray, X_bdy: np.ndarray,
                  g: np.ndarray, loss_host: Optional[np.ndarray] = None) -> np.ndarray:
        """One KFAC step with the batch in host memory (copied in by the library)."""
        bufs = [np.ascontiguousarray(a, dtype=np.float64) if not isinstance(a, torch.Tensor) else a
                for a in (X_int, f, X_bdy, g)]
        ptrs = [b.ctypes.data if isinstance(b, np.ndarray) else b.data_ptr() for b in bufs]
        out = np.zeros(3) if loss_host is None else loss_host
        _check("kfac_pinn_step_host", self.lib.kfac_pinn_step_host(
            self.h, _stream(), _ptr(theta), ptrs[0], bufs[0].shape[0], ptrs[1], ptrs[2],
            bufs[2].shape[0], ptrs[3], out.ctypes.data))
        return out

    # -- inspection -------------------------------------------------------
    def factor_shape(self, layer: int, which: str) -> int:
        dims = [self.d] + list(self.widths)
        return dims[layer - 1] + 1 if which.startswith("A") else dims[layer]

    def get_factor(self, layer: int, which: str) -> torch.Tensor:
        n = self.factor_shape(layer, which)
        out = torch.empty(n, n, dtype=torch.float64, device=self.device)
        _check("kfac_pinn_get_factor", self.lib.kfac_pinn_get_factor(
            self.h, _stream(), layer, FACTORS[which], _ptr(out)))
        return out

    def set_factor(self, layer: int, which: str, M):
        t = _dev(M, self.device)
        _check("kfac_pinn_set_factor", self.lib.kfac_pinn_set_factor(
            self.h, _stream(), layer, FACTORS[which], _ptr(t)))
        torch.cuda.current_stream().synchronize()

    def gradient(self) -> torch.Tensor:
        out = torch.empty(self.D, dtype=torch.float64, device=self.device)
        _check("kfac_pinn_get_gradient", self.lib.kfac_pinn_get_gradient(self.h, _stream(), _ptr(out)))
        return out

    def direction(self) -> torch.Tensor:
        out = torch.empty(self.D, dtype=torch.float64, device=self.device)
        _check("kfac_pinn_get_direction", self.lib.kfac_pinn_get_direction(self.h, _stream(), _ptr(out)))
        return out

    def line_search_losses(self) -> torch.Tensor:
        """Trial losses of the last step's line search: (31, 3), row k at alpha = 2^-k."""
        out = torch.empty(31, 3, dtype=torch.float64, device=self.device)
        _check("kfac_pinn_get_line_search_losses", self.lib.kfac_pinn_get_line_search_losses(
            self.h, _stream(), _ptr(out)))
        return out

    def update_coefficients(self) -> torch.Tensor:
        """(c0, c1) of the last step's update delta = c0 Delta + c1 delta_prev."""
        out = torch.empty(2, dtype=torch.float64, device=self.device)
        _check("kfac_pinn_get_update_coefficients", self.lib.kfac_pinn_get_update_coefficients(
            self.h, _stream(), _ptr(out)))
        return out

    def sync_status(self) -> str:
        v = C.c_int(0)
        _check("kfac_pinn_sync_status", self.lib.kfac_pinn_sync_status(self.h, C.byref(v)))
        return _lib.STATUS.get(v.value, str(v.value))

    def launch_count(self) -> int:
        return int(self.lib.kfac_pinn_launch_count(self.h))

    def check_wait_timeout(self, kind: str = "group_barrier", limit_ms: int = 50):
        """Run a bounded device wait that cannot complete ("group_barrier": the
        eigensolver's; "mbarrier": the tcgen05 engine's) with a short limit; the
        handle's status word then holds KFAC_TIMEOUT (see sync_status)."""
        k = {"group_barrier": 0, "mbarrier": 1}[kind]
        _check("kfac_pinn_check_wait_timeout",
               self.lib.kfac_pinn_check_wait_timeout(self.h, _stream(), k, int(limit_ms)))

    def timing_enable(self, on: bool = True):
        _check("kfac_pinn_timing_enable", self.lib.kfac_pinn_timing_enable(self.h, int(on)))

    def timing_read(self) -> dict:
        """Per kernel class since the last read: device ms, launches, the method's
        work ("work": real sizes, one product per contraction, symmetric Grams
        counted once) and the work as executed ("exec": padded tiles and every
        split-BF16 product)."""
        out = {}
        for cls, name in _lib.KERNEL_CLASSES.items():
            ms, n, w, x = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
            _check("kfac_pinn_timing_read_ex", self.lib.kfac_pinn_timing_read_ex(
                self.h, cls, C.byref(ms), C.byref(n), C.byref(w), C.byref(x)))
            out[name] = {"ms": ms.value, "launches": n.value, "work": w.value, "exec": x.value}
        return out


class ForwardLaplacian(torch.autograd.Function):
    """(u, grad u, lap u) of the MLP with packed parameters theta at the points X
    (Sec. 3.1), differentiable in theta and X through the library's reverse pass.

        u, g, lap = ForwardLaplacian.apply(theta, X, opt)     # opt: an FP64 KfacPinn
    """

    @staticmethod
    def forward(ctx, theta, X, opt):
        th = theta.detach().contiguous()
        u, g, lap = opt.forward_laplacian(th, X.detach())
        ctx.save_for_backward(th, X.detach())
        ctx.opt = opt
        return u, g, lap

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, du, dg, dl):
        theta, X = ctx.saved_tensors
        dtheta, dX = ctx.opt.forward_laplacian_backward(theta, X, du, dg, dl, need_dX=ctx.needs_input_grad[1])
        return (dtheta if ctx.needs_input_grad[0] else None), dX, None


class KfacBatch:
    """Many KfacPinn problems stepped together, replayed as one CUDA graph:
    their steps on worker streams, or (grouped=True) every kernel launched
    once for all problems and one batched eigensolve."""

    def __init__(self, problems: Sequence[KfacPinn], n_streams: int = 8, grouped: bool = False):
        self.lib = _lib.load()
        self.problems = list(problems)
        hs = (C.c_void_p * len(self.problems))(*[p.h.value for p in self.problems])
        self.b = C.c_void_p()
        _check("kfac_pinn_batch_create", self.lib.kfac_pinn_batch_create(hs, len(self.problems), n_streams,
                                                                         C.byref(self.b)))
        if grouped:
            _check("kfac_pinn_batch_set_grouped", self.lib.kfac_pinn_batch_set_grouped(self.b, 1))

    def launches_per_step(self):
        """Kernel launches of one replayed batch step (None before the graph exists)."""
        n = C.c_longlong()
        st = self.lib.kfac_pinn_batch_launches(self.b, C.byref(n))
        if st == 7:      # KFAC_NOT_READY
            return None
        _check("kfac_pinn_batch_launches", st)
        return int(n.value)

    def close(self):
        if self.b:
            self.lib.kfac_pinn_batch_destroy(self.b)
            self.b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, thetas, X_int, f, X_bdy, g, losses=None, use_graph: bool = True):
        """One step of every problem; all arguments are lists of device tensors
        (FP64, contiguous) that stay at the same addresses between calls for the
        graph to be replayed."""
        n = len(self.problems)
        P = C.c_void_p * n
        Ia = C.c_int * n

        def ptrs(ts):
            return P(*[None if t is None else t.data_ptr() for t in ts])

        _check("kfac_pinn_batch_step", self.lib.kfac_pinn_batch_step(
            self.b, _stream(), ptrs(thetas), ptrs(X_int), Ia(*[x.shape[0] for x in X_int]), ptrs(f),
            ptrs(X_bdy), Ia(*[x.shape[0] for x in X_bdy]), ptrs(g), None if losses is None else ptrs(losses),
            int(use_graph)))


def inject_alloc_failure(n: int):
    """Make the device allocation after n more successful ones fail as out of
    memory (n = -1: none); process-wide, for failure-path tests."""
    lib = _lib.load()
    _check("kfac_pinn_inject_alloc_failure", lib.kfac_pinn_inject_alloc_failure(int(n)))
