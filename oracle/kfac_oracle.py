"""Plain FP64 CPU oracle of one KFAC step for a PINN loss.

TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path imports,
calls or links this module; only the tests, the smoke check and the timed CPU
baseline of the benchmark do.  It shares no code with the CUDA path: the only
common inputs are the seeded arrays of the `synth` package.

Every function follows the paper (Dangel, Müller, Zeinhofer, "Kronecker-Factored
Approximate Curvature for Physics-Informed Neural Networks", NeurIPS 2024) step
by step in FP64 numpy; a batched matmul over collocation points, a Cholesky
factorisation, a triangular solve and a symmetric eigendecomposition are the
library primitives it uses.  Notation:

  * layers l = 1..L with widths h_0 = d, h_1, .., h_L = 1;
  * W̃_l = (W_l b_l) in R^{h_l x (h_{l-1}+1)}, theta = (vec W̃_1, .., vec W̃_L)
    with vec = column stacking (Sec. 2);
  * per collocation point n the Taylor matrix has S = d + 2 columns
    [value, ∂_1, .., ∂_d, Laplacian] (Sec. 3.2; App. C.2 Eq. 20);
  * arrays of per-point matrices have shape (N, rows, S).

Readings taken where the paper is silent or inconsistent:
  * The Laplacian column carries the full Laplacian Δz (main text, Eq. 6),
    not the half-Laplacian of the Taylor coefficients of App. C.
  * The loss is Eq. 1 with 1/(2N) on both terms, also for the heat equation.
  * The boundary curvature is A_∂ ⊗ B_∂ (Sec. 3.4 prints A_Ω ⊗ B_Ω there; the
    pseudo-code of App. B uses the boundary factors).
  * The update is θ_{t+1} = θ_t + δ_t with δ_t = α · δ̂_t (Sec. 3.4); the
    pseudo-code of App. B multiplies by the step size twice.  α is either a
    fixed learning rate or the grid line search of Sec. 3.4, whose ties (not
    specified) keep the larger α.
  * KFAC* (Sec. 3.4): the printed 2x2 system's lower-right entry δᵀGΔ is read
    as δᵀGδ (the quadratic model's curvature along δ); on the first step, with
    no previous update, only α is fitted and μ = 0.
  * KFAC-reduce, which the paper cites but does not restate, is read as
    A = (1/N) Σ_n ā_n ā_nᵀ with ā_n the mean of the S input columns and
    B = (1/N) Σ_n ḡ_n ḡ_nᵀ with ḡ_n the sum of the S output gradients.
  * Damping adds λ (or √λ when `damping_sqrt`) times the identity to each
    factor (Sec. 3.4).
  * General residuals (Sec. 3.3) are taken as polynomials of degree two in
    the network's Taylor outputs with a quadratic criterion ½ rᵀ W r, so that
    Λ = W; the PDE map Ψ of Eq. 9 is not otherwise specified.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg as sla

# ---------------------------------------------------------------------------
# Parameter bookkeeping (Sec. 2)
# ---------------------------------------------------------------------------


def layer_dims(d: int, widths: Sequence[int]) -> List[int]:
    return [int(d)] + [int(w) for w in widths]


def unpack_theta(theta: np.ndarray, d: int, widths: Sequence[int]) -> List[np.ndarray]:
    """Split theta into W̃_l = (W_l b_l), each h_l x (h_{l-1}+1) (column stacking)."""
    dims = layer_dims(d, widths)
    out, off = [], 0
    for l in range(1, len(dims)):
        rows, cols = dims[l], dims[l - 1] + 1
        out.append(theta[off:off + rows * cols].reshape(cols, rows).T.copy())
        off += rows * cols
    assert off == theta.size, "theta has the wrong length for these widths"
    return out


def pack_theta(Ws: Sequence[np.ndarray]) -> np.ndarray:
    return np.concatenate([W.reshape(-1, order="F") for W in Ws])


def laplacian_set(d: int, op: str) -> np.ndarray:
    """Input coordinates summed in the Laplacian column: all of them for the
    Poisson operator, the spatial ones (coordinate 0 is time) for the heat
    operator (App. A.6)."""
    if op == "heat":
        return np.arange(1, d)
    return np.arange(d)


def operator_matrix(d: int, op: str, coef: Optional[np.ndarray] = None) -> np.ndarray:
    """Coefficients c_ij of the second-order column Σ_ij c_ij ∂²_ij z (App. C.3):
    the identity for the Laplacian, the spatial identity for the heat operator's
    partial Laplacian, the given symmetric matrix for a general operator."""
    if op == "general":
        C = np.asarray(coef, dtype=np.float64)
        assert C.shape == (d, d) and np.allclose(C, C.T, rtol=0, atol=1e-12 * np.abs(C).max())
        return C
    C = np.zeros((d, d))
    idx = laplacian_set(d, op)
    C[idx, idx] = 1.0
    return C


# ---------------------------------------------------------------------------
# Forward Laplacian (Sec. 3.1 Eq. 5-6; App. C.2 Eq. 19-20)
# ---------------------------------------------------------------------------


@dataclass
class TaylorPass:
    """Intermediates of one forward pass over N points with S shared columns.

    T_in[l] is the augmented input T̂^{(l)} of linear layer l+1, shape
    (N, h_l + 1, S) (bias row last); Z[l] is the output Z^{(l+1)} of linear
    layer l+1, shape (N, h_{l+1}, S).
    """
    T_in: List[np.ndarray]
    Z: List[np.ndarray]
    S: int


def input_taylor_matrix(X: np.ndarray, with_derivatives: bool) -> np.ndarray:
    """T̂^{(0)} per point: columns (x, e_1..e_d, 0) with bias row (1, 0, .., 0)
    (Sec. 3.1: z^(0) = x, ∂_i z^(0) = e_i, second derivatives 0)."""
    N, d = X.shape
    if not with_derivatives:
        T = np.zeros((N, d + 1, 1))
        T[:, :d, 0] = X
        T[:, d, 0] = 1.0
        return T
    S = d + 2
    T = np.zeros((N, d + 1, S))
    T[:, :d, 0] = X
    T[:, d, 0] = 1.0
    T[:, np.arange(d), 1 + np.arange(d)] = 1.0
    return T


def tanh_taylor(Z: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Element-wise tanh through the Taylor columns (Eq. 6; App. C.3).

    value  y_0 = σ(a_0)
    ∂_i    y_i = σ'(a_0) a_i
    second y_C = σ'(a_0) a_C + σ''(a_0) Σ_ij c_ij a_i a_j     (Laplacian: c = I)
    with σ = tanh, σ' = 1 - σ², σ'' = -2 σ σ'.
    """
    a0 = Z[:, :, 0]
    y0 = np.tanh(a0)
    s1 = 1.0 - y0 * y0
    s2 = -2.0 * y0 * s1
    Y = np.empty_like(Z)
    Y[:, :, 0] = y0
    S = Z.shape[2]
    if S > 1:
        a_tan = Z[:, :, 1:S - 1]
        Y[:, :, 1:S - 1] = s1[:, :, None] * a_tan
        quad = np.einsum("nhi,ij,nhj->nh", a_tan, C, a_tan)
        Y[:, :, S - 1] = s1 * Z[:, :, S - 1] + s2 * quad
    return Y


def append_bias_row(T: np.ndarray) -> np.ndarray:
    """Append the row (1, 0, .., 0) that multiplies the bias (App. C.2 Eq. 20)."""
    N, h, S = T.shape
    out = np.zeros((N, h + 1, S))
    out[:, :h, :] = T
    out[:, h, 0] = 1.0
    return out


def taylor_forward(Ws: Sequence[np.ndarray], X: np.ndarray, op: str = "laplace",
                   with_derivatives: bool = True, coef: Optional[np.ndarray] = None) -> TaylorPass:
    """Forward Laplacian with intermediates (App. B; App. C.2).

    Z^{(l)} = W̃_l T̂^{(l-1)}; for l < L the tanh rule gives T^{(l)} and its
    bias row is appended.  With with_derivatives=False this is the plain
    forward pass of the boundary term (S = 1)."""
    d = X.shape[1]
    T = input_taylor_matrix(X, with_derivatives)
    C = operator_matrix(d, op, coef)
    T_in, Zs = [], []
    L = len(Ws)
    for l, W in enumerate(Ws):
        T_in.append(T)
        Z = np.matmul(W[None, :, :], T)
        Zs.append(Z)
        if l < L - 1:
            T = append_bias_row(tanh_taylor(Z, C))
    return TaylorPass(T_in=T_in, Z=Zs, S=T.shape[2])


def forward_laplacian(Ws: Sequence[np.ndarray], X: np.ndarray, op: str = "laplace",
                      coef: Optional[np.ndarray] = None):
    """u, ∇u and the second-order column per point: the Laplacian (partial for
    heat) or Σ_ij c_ij ∂²_ij u for a general operator (App. C.3)."""
    fp = taylor_forward(Ws, X, op, True, coef)
    out = fp.Z[-1][:, 0, :]
    return out[:, 0].copy(), out[:, 1:-1].copy(), out[:, -1].copy()


# ---------------------------------------------------------------------------
# Residuals and loss (Eq. 1; App. A.6 for the heat operator)
# ---------------------------------------------------------------------------


def interior_residual(fp: TaylorPass, f: np.ndarray, op: str, kappa: float) -> np.ndarray:
    out = fp.Z[-1][:, 0, :]
    if op == "general":
        return out[:, -1] - f                          # Σ c_ij ∂²_ij u - f
    if op == "heat":
        return out[:, 1] - kappa * out[:, -1] - f      # ∂_t u - κ Δ_x u - f
    return -out[:, -1] - f                             # -Δu - f


def boundary_residual(fp: TaylorPass, g: np.ndarray) -> np.ndarray:
    return fp.Z[-1][:, 0, 0] - g                       # u - g


def residual_seed(S: int, op: str, kappa: float, interior: bool) -> np.ndarray:
    """c = ∂r_n / ∂Z^{(L)}_n, a row of length S (the output has one row)."""
    c = np.zeros(S)
    if not interior:
        c[0] = 1.0
    elif op == "general":
        c[S - 1] = 1.0
    elif op == "heat":
        c[1] = 1.0
        c[S - 1] = -kappa
    else:
        c[S - 1] = -1.0
    return c


@dataclass
class QuadraticResidual:
    """A PDE residual with M outputs (Sec. 3.3, Eq. 9) that is a polynomial of
    degree two in the network's Taylor outputs z_n = Z^{(L)}_n = (u, ∂_1 u, ..,
    ∂_d u, second-order column) ∈ R^S:

        r_{n,k} = Σ_s b[k,s] z_{n,s} + ½ Σ_{s,t} Q[k,s,t] z_{n,s} z_{n,t} - f_{n,k},

    fed into the criterion ℓ(r) = ½ rᵀ W r, whose Hessian Λ(r) = W is constant
    (W = I: the squared residual of Eq. 1).  First-order terms of a linear
    operator are b on the first-derivative columns; the |∇u|² of a nonlinear
    one is Q on them."""
    b: np.ndarray                     # (M, S)
    Q: Optional[np.ndarray] = None    # (M, S, S), symmetric in its last two indices
    W: Optional[np.ndarray] = None    # (M, M) symmetric positive definite; None: identity

    @property
    def M(self) -> int:
        return self.b.shape[0]

    def weight(self) -> np.ndarray:
        return np.eye(self.M) if self.W is None else np.asarray(self.W, dtype=np.float64)


def quadratic_residual(res: QuadraticResidual, z: np.ndarray, f: np.ndarray) -> np.ndarray:
    """r_{n,k} for outputs z (N, S) and data f (N, M): shape (N, M)."""
    r = z @ res.b.T - np.asarray(f, dtype=np.float64).reshape(z.shape[0], res.M)
    if res.Q is not None:
        r = r + 0.5 * np.einsum("ns,kst,nt->nk", z, res.Q, z)
    return r


def quadratic_residual_jacobian(res: QuadraticResidual, z: np.ndarray) -> np.ndarray:
    """∂r_{n,k}/∂z_{n,s} = b[k,s] + Σ_t Q[k,s,t] z_{n,t}: shape (N, M, S)."""
    J = np.broadcast_to(res.b[None, :, :], (z.shape[0],) + res.b.shape).copy()
    if res.Q is not None:
        J = J + np.einsum("kst,nt->nks", res.Q, z)
    return J


def loss(r_int: np.ndarray, r_bdy: np.ndarray) -> Tuple[float, float, float]:
    li = float((r_int ** 2).sum() / (2.0 * r_int.size))
    lb = float((r_bdy ** 2).sum() / (2.0 * r_bdy.size))
    return li + lb, li, lb


def loss_general(res: QuadraticResidual, r_int: np.ndarray, r_bdy: np.ndarray) -> Tuple[float, float, float]:
    """L_Ω = (1/N) Σ_n ℓ(r_n) with ℓ(r) = ½ rᵀ W r (Sec. 3.3), plus the boundary
    term of Eq. 1."""
    W = res.weight()
    li = float(np.einsum("nk,kj,nj->", r_int, W, r_int) / (2.0 * r_int.shape[0]))
    lb = float((r_bdy ** 2).sum() / (2.0 * r_bdy.size))
    return li + lb, li, lb


# ---------------------------------------------------------------------------
# Backward of the Taylor pass: g^{(l)}_{n,s} = ∂r_n/∂Z^{(l)}_{n,s} (Sec. 3.2)
# ---------------------------------------------------------------------------


def tanh_taylor_adjoint(Z: np.ndarray, Ybar: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Vector-Jacobian product of `tanh_taylor` (derived from Eq. 6; App. C.3).

    ā_C = σ' ȳ_C
    ā_i = σ' ȳ_i + 2 σ'' (C a)_i ȳ_C          (C symmetric)
    ā_0 = σ' ȳ_0 + σ'' Σ_i a_i ȳ_i + (σ'' a_C + σ''' Σ_ij c_ij a_i a_j) ȳ_C
    with σ''' = -2 σ' (1 - 3 σ²).
    """
    a0 = Z[:, :, 0]
    y0 = np.tanh(a0)
    s1 = 1.0 - y0 * y0
    s2 = -2.0 * y0 * s1
    s3 = -2.0 * s1 * (1.0 - 3.0 * y0 * y0)
    S = Z.shape[2]
    Abar = np.empty_like(Z)
    if S == 1:
        Abar[:, :, 0] = s1 * Ybar[:, :, 0]
        return Abar
    yd = Ybar[:, :, S - 1]
    a_tan = Z[:, :, 1:S - 1]
    Abar[:, :, S - 1] = s1 * yd
    Ca = np.einsum("ij,nhj->nhi", C, a_tan)
    Abar[:, :, 1:S - 1] = s1[:, :, None] * Ybar[:, :, 1:S - 1] + 2.0 * (s2 * yd)[:, :, None] * Ca
    quad = (a_tan * Ca).sum(axis=2)
    Abar[:, :, 0] = (s1 * Ybar[:, :, 0]
                     + s2 * (a_tan * Ybar[:, :, 1:S - 1]).sum(axis=2)
                     + (s2 * Z[:, :, S - 1] + s3 * quad) * yd)
    return Abar


def taylor_adjoint(Ws: Sequence[np.ndarray], fp: TaylorPass, seed: np.ndarray,
                   op: str = "laplace", coef: Optional[np.ndarray] = None) -> List[np.ndarray]:
    """Backpropagate the seed c through the Taylor pass (App. B, the backward
    that yields g^{(l)}).  Returns Zbar[l] = g^{(l+1)}, shape (N, h_{l+1}, S).

    seed: c = ∂r_n/∂Z^{(L)}_n, the same row of length S for every point, or
    one row per point, shape (N, S) (a residual that is nonlinear in the
    network's outputs, Sec. 3.3).
    Linear layer Z = W̃ T̂: T̄ = W̃ᵀ Z̄ with the bias row dropped.
    Activation layer: `tanh_taylor_adjoint`."""
    L = len(Ws)
    N = fp.Z[-1].shape[0]
    d = fp.T_in[0].shape[1] - 1
    C = operator_matrix(d, op, coef)
    Zbar: List[Optional[np.ndarray]] = [None] * L
    seed = np.asarray(seed, dtype=np.float64)
    if seed.ndim == 1:
        cur = np.broadcast_to(seed[None, None, :], (N, 1, seed.size)).copy()
    else:
        cur = seed[:, None, :].copy()
    for l in range(L - 1, -1, -1):
        Zbar[l] = cur
        if l == 0:
            break
        W = Ws[l][:, :-1]                       # drop the bias column
        Tbar = np.matmul(W.T[None, :, :], cur)  # (N, h_{l}, S)
        cur = tanh_taylor_adjoint(fp.Z[l - 1], Tbar, C)
    return Zbar  # type: ignore[return-value]


# ---------------------------------------------------------------------------
# Gradient of the loss (App. B)
# ---------------------------------------------------------------------------


def weight_jacobian(Zbar_l: np.ndarray, T_in_l: np.ndarray) -> np.ndarray:
    """J_{W̃_l} r_n = Σ_s g_{n,s} T̂_{n,s}ᵀ per point (Sec. 3.2), (N, h_l, h_{l-1}+1)."""
    return np.matmul(Zbar_l, np.transpose(T_in_l, (0, 2, 1)))


def loss_gradient(fp_i: TaylorPass, zb_i: List[np.ndarray], r_i: np.ndarray,
                  fp_b: TaylorPass, zb_b: List[np.ndarray], r_b: np.ndarray) -> List[np.ndarray]:
    """∇_{W̃_l} L = (1/N_Ω) Σ_n r_n J_n + (1/N_∂) Σ_n r^b_n J^b_n."""
    grads = []
    for l in range(len(zb_i)):
        Ji = weight_jacobian(zb_i[l], fp_i.T_in[l])
        Jb = weight_jacobian(zb_b[l], fp_b.T_in[l])
        grads.append(np.tensordot(r_i, Ji, axes=(0, 0)) / r_i.size
                     + np.tensordot(r_b, Jb, axes=(0, 0)) / r_b.size)
    return grads


# ---------------------------------------------------------------------------
# Kronecker factors (Eq. 3 boundary, Eq. 8 interior; App. B)
# ---------------------------------------------------------------------------


def factors_expand(T_in_l: np.ndarray, Zbar_l: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """KFAC-expand (Eq. 8): A = (1/(NS)) Σ_{n,s} T̂ T̂ᵀ, B = (1/N) Σ_{n,s} g gᵀ.
    For S = 1 this is the classic KFAC of Eq. 3."""
    N, _, S = T_in_l.shape
    Tf = np.transpose(T_in_l, (0, 2, 1)).reshape(N * S, -1)
    Gf = np.transpose(Zbar_l, (0, 2, 1)).reshape(N * S, -1)
    return Tf.T @ Tf / (N * S), Gf.T @ Gf / N


def factors_reduce(T_in_l: np.ndarray, Zbar_l: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """KFAC-reduce (reading of the cited weight-sharing KFAC):
    A = (1/N) Σ_n ā ā ᵀ with ā_n = (1/S) Σ_s T̂_{n,s};
    B = (1/N) Σ_n ḡ ḡᵀ with ḡ_n = Σ_s g_{n,s}."""
    N = T_in_l.shape[0]
    abar = T_in_l.mean(axis=2)
    gbar = Zbar_l.sum(axis=2)
    return abar.T @ abar / N, gbar.T @ gbar / N


# ---------------------------------------------------------------------------
# Damped Kronecker-sum inverse (Sec. 3.4 "Gradient preconditioning")
# ---------------------------------------------------------------------------


def damp(M: np.ndarray, lam: float, damping_sqrt: bool) -> np.ndarray:
    eps = np.sqrt(lam) if damping_sqrt else lam
    return M + eps * np.eye(M.shape[0])


def generalized_eig(P: np.ndarray, Q: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Simultaneous diagonalisation of SPD P and symmetric Q: returns V, w with
    Vᵀ P V = I and Vᵀ Q V = diag(w).  Route: P = L Lᵀ, L⁻¹ Q L⁻ᵀ = U diag(w) Uᵀ,
    V = L⁻ᵀ U (the eigen-decomposition trick of the KFAC paper's App. I)."""
    Lc = np.linalg.cholesky(P)
    M = sla.solve_triangular(Lc, Q, lower=True)
    M = sla.solve_triangular(Lc, M.T, lower=True).T
    M = 0.5 * (M + M.T)
    w, U = np.linalg.eigh(M)
    V = sla.solve_triangular(Lc.T, U, lower=False)
    return V, w


def kron_sum_inverse_apply(A_i, B_i, A_b, B_b, G, lam, damping_sqrt=False):
    """Δ = -(Ã_Ω ⊗ B̃_Ω + Ã_∂ ⊗ B̃_∂)⁻¹ vec G, returned as a matrix (App. B).

    With V_A, a from (Ã_Ω, Ã_∂) and V_B, b from (B̃_Ω, B̃_∂):
    Δ = -V_B [(V_Bᵀ G V_A) ⊘ (1 + b aᵀ)] V_Aᵀ, using vec(BXA) = (Aᵀ ⊗ B) vec X."""
    VA, a = generalized_eig(damp(A_i, lam, damping_sqrt), damp(A_b, lam, damping_sqrt))
    VB, b = generalized_eig(damp(B_i, lam, damping_sqrt), damp(B_b, lam, damping_sqrt))
    Y = VB.T @ G @ VA
    Y = Y / (1.0 + np.outer(b, a))
    return -(VB @ Y @ VA.T)


# ---------------------------------------------------------------------------
# One KFAC step (App. B, Algorithm 1, fixed learning rate)
# ---------------------------------------------------------------------------


@dataclass
class KfacConfig:
    d: int
    widths: Tuple[int, ...]
    op: str = "laplace"
    kappa: float = 0.0
    variant: str = "expand"
    beta: float = 0.0
    lam: float = 1e-3
    damping_sqrt: bool = False
    init_identity: bool = False
    lr: float = 0.1
    momentum: float = 0.0
    line_search: bool = False
    kfac_star: bool = False     # automatic learning rate and momentum (KFAC*, Sec. 3.4)
    op_coef: Optional[np.ndarray] = None   # op == "general": symmetric d x d c_ij (App. C.3)
    residual: Optional[QuadraticResidual] = None   # interior residual of Sec. 3.3 (None: the operator's own)


@dataclass
class KfacState:
    A_int: List[np.ndarray]
    B_int: List[np.ndarray]
    A_bdy: List[np.ndarray]
    B_bdy: List[np.ndarray]
    delta_prev: Optional[List[np.ndarray]] = None
    t: int = 0


def init_state(cfg: KfacConfig) -> KfacState:
    dims = layer_dims(cfg.d, cfg.widths)
    mk = (lambda n: np.eye(n)) if cfg.init_identity else (lambda n: np.zeros((n, n)))
    A = [mk(dims[l - 1] + 1) for l in range(1, len(dims))]
    B = [mk(dims[l]) for l in range(1, len(dims))]
    return KfacState([a.copy() for a in A], [b.copy() for b in B],
                     [a.copy() for a in A], [b.copy() for b in B])


@dataclass
class StepResult:
    loss: Tuple[float, float, float]
    grads: List[np.ndarray]
    factors: Tuple[List[np.ndarray], List[np.ndarray], List[np.ndarray], List[np.ndarray]]
    direction: List[np.ndarray]          # Δ_t (preconditioned, before momentum/lr)
    update: List[np.ndarray]             # δ_t = α (μ δ_{t-1} + Δ_t), α = lr or line search
    theta_new: np.ndarray
    extras: dict = field(default_factory=dict)


def curvature_and_gradient_general(cfg: KfacConfig, Ws, X_int, f, X_bdy, g):
    """The curvature and gradient of a general residual (Sec. 3.3): per residual
    output k an adjoint pass seeded with ∂r_{n,k}/∂Z^{(L)}_n gives
    g^{(l)}_{n,s,k} = (J_{Z^{(l)}_{n,s}} r_{n,k})ᵀ, and with Λ = W

        A_Ω = (1/(N S)) Σ_{n,s} T̂_{n,s} T̂_{n,s}ᵀ,
        B_Ω = (1/N) Σ_{n,s} (J_{Z_{n,s}} r_n)ᵀ Λ (J_{Z_{n,s}} r_n)
            = (1/N) Σ_{n,s} Σ_{k,k'} W_{k,k'} g_{n,s,k} g_{n,s,k'}ᵀ            (Eq. 10),
        ∇_{W̃_l} L_Ω = (1/N) Σ_n Σ_k (W r_n)_k J_{W̃_l} r_{n,k}.

    KFAC-expand; the boundary term is the one of Eq. 1."""
    res = cfg.residual
    assert cfg.variant == "expand", "the general residual is expand-only"
    W = res.weight()
    fp_i = taylor_forward(Ws, X_int, cfg.op, True, cfg.op_coef)
    z = fp_i.Z[-1][:, 0, :]
    r_i = quadratic_residual(res, z, f)
    J = quadratic_residual_jacobian(res, z)
    zb_k = [taylor_adjoint(Ws, fp_i, J[:, k, :], cfg.op, cfg.op_coef) for k in range(res.M)]
    fp_b = taylor_forward(Ws, X_bdy, cfg.op, False, cfg.op_coef)
    r_b = boundary_residual(fp_b, g)
    zb_b = taylor_adjoint(Ws, fp_b, residual_seed(1, cfg.op, cfg.kappa, False), cfg.op, cfg.op_coef)
    N = z.shape[0]
    Wr = r_i @ W                                   # (W r_n)_k, W symmetric
    Ai, Bi, Ab, Bb, grads = [], [], [], [], []
    for l in range(len(Ws)):
        T = fp_i.T_in[l]
        S = T.shape[2]
        Tf = np.transpose(T, (0, 2, 1)).reshape(N * S, -1)
        Ai.append(Tf.T @ Tf / (N * S))
        Gf = [np.transpose(zb[l], (0, 2, 1)).reshape(N * S, -1) for zb in zb_k]
        Bi.append(sum(W[k, kk] * (Gf[k].T @ Gf[kk]) for k in range(res.M) for kk in range(res.M)) / N)
        a, b = factors_expand(fp_b.T_in[l], zb_b[l])
        Ab.append(a); Bb.append(b)
        gi = sum(np.tensordot(Wr[:, k], weight_jacobian(zb_k[k][l], T), axes=(0, 0)) for k in range(res.M)) / N
        gb = np.tensordot(r_b, weight_jacobian(zb_b[l], fp_b.T_in[l]), axes=(0, 0)) / r_b.size
        grads.append(gi + gb)
    return dict(fp_i=fp_i, fp_b=fp_b, r_i=r_i, r_b=r_b, zb_i_k=zb_k, zb_b=zb_b, J=J,
                factors=(Ai, Bi, Ab, Bb), grads=grads, loss=loss_general(res, r_i, r_b))


def curvature_and_gradient(cfg: KfacConfig, Ws, X_int, f, X_bdy, g):
    """App. B (without the preconditioner)."""
    if cfg.residual is not None:
        return curvature_and_gradient_general(cfg, Ws, X_int, f, X_bdy, g)
    fp_i = taylor_forward(Ws, X_int, cfg.op, True, cfg.op_coef)
    r_i = interior_residual(fp_i, f, cfg.op, cfg.kappa)
    zb_i = taylor_adjoint(Ws, fp_i, residual_seed(fp_i.S, cfg.op, cfg.kappa, True), cfg.op, cfg.op_coef)
    fp_b = taylor_forward(Ws, X_bdy, cfg.op, False, cfg.op_coef)
    r_b = boundary_residual(fp_b, g)
    zb_b = taylor_adjoint(Ws, fp_b, residual_seed(1, cfg.op, cfg.kappa, False), cfg.op, cfg.op_coef)
    fac = factors_expand if cfg.variant == "expand" else factors_reduce
    Ai, Bi, Ab, Bb = [], [], [], []
    for l in range(len(Ws)):
        a, b = fac(fp_i.T_in[l], zb_i[l])
        Ai.append(a); Bi.append(b)
        a, b = factors_expand(fp_b.T_in[l], zb_b[l])   # S = 1: classic KFAC
        Ab.append(a); Bb.append(b)
    grads = loss_gradient(fp_i, zb_i, r_i, fp_b, zb_b, r_b)
    return dict(fp_i=fp_i, fp_b=fp_b, r_i=r_i, r_b=r_b, zb_i=zb_i, zb_b=zb_b,
                factors=(Ai, Bi, Ab, Bb), grads=grads, loss=loss(r_i, r_b))


def batch_loss(cfg: KfacConfig, theta: np.ndarray, X_int, f, X_bdy, g) -> Tuple[float, float, float]:
    """Eq. 1 at theta on one batch: forward passes and residuals only."""
    Ws = unpack_theta(theta, cfg.d, cfg.widths)
    fp_i = taylor_forward(Ws, X_int, cfg.op, True, cfg.op_coef)
    r_b = boundary_residual(taylor_forward(Ws, X_bdy, cfg.op, False, cfg.op_coef), g)
    if cfg.residual is not None:
        return loss_general(cfg.residual, quadratic_residual(cfg.residual, fp_i.Z[-1][:, 0, :], f), r_b)
    return loss(interior_residual(fp_i, f, cfg.op, cfg.kappa), r_b)


LINE_SEARCH_GRID = tuple(2.0 ** -k for k in range(31))   # {2^0, 2^-1, .., 2^-30} (Sec. 3.4)


def line_search(cfg: KfacConfig, theta: np.ndarray, dhat: np.ndarray, X_int, f, X_bdy, g):
    """α* = argmin_α L(θ + α δ̂) over the logarithmic grid (Sec. 3.4; App. B).

    Returns (α*, losses) with losses[k] = L(θ + 2^-k δ̂) as (L, L_Ω, L_∂).  Equal
    losses keep the larger α; non-finite losses never win; α* = 0 when no
    trial is finite."""
    losses = [batch_loss(cfg, theta + a * dhat, X_int, f, X_bdy, g) for a in LINE_SEARCH_GRID]
    best = None
    for k, (tot, _, _) in enumerate(losses):
        if np.isfinite(tot) and (best is None or tot < losses[best][0]):
            best = k
    alpha = 0.0 if best is None else LINE_SEARCH_GRID[best]
    return alpha, np.array(losses)


def residual_jvp(cg: dict, V: Sequence[np.ndarray]) -> Tuple[np.ndarray, np.ndarray]:
    """J_θ r · v for the interior and boundary residuals: (J_n v) = Σ_l ⟨J_{W̃_l} r_n, V_l⟩
    with the per-point weight Jacobians of Sec. 3.2 (V_l shaped like W̃_l).  A
    residual with M outputs (Sec. 3.3) gives (N, M) interior products."""
    if "zb_i_k" in cg:
        ji = np.stack([sum(np.einsum("nij,ij->n", weight_jacobian(zb[l], cg["fp_i"].T_in[l]), V[l])
                           for l in range(len(V))) for zb in cg["zb_i_k"]], axis=1)
    else:
        ji = sum(np.einsum("nij,ij->n", weight_jacobian(cg["zb_i"][l], cg["fp_i"].T_in[l]), V[l])
                 for l in range(len(V)))
    jb = sum(np.einsum("nij,ij->n", weight_jacobian(cg["zb_b"][l], cg["fp_b"].T_in[l]), V[l])
             for l in range(len(V)))
    return ji, jb


def gramian_bilinear(ja: Tuple[np.ndarray, np.ndarray], jb: Tuple[np.ndarray, np.ndarray],
                     W: Optional[np.ndarray] = None) -> float:
    """aᵀ G b with G of Eq. 2 (Λ = W for a residual with M outputs, Sec. 3.3),
    from the residual JVPs J a and J b."""
    if ja[0].ndim == 2:
        Wm = np.eye(ja[0].shape[1]) if W is None else W
        inner = float(np.einsum("nk,kj,nj->", ja[0], Wm, jb[0]) / ja[0].shape[0])
    else:
        inner = float(ja[0] @ jb[0] / ja[0].size)
    return inner + float(ja[1] @ jb[1] / ja[1].size)


def kfac_star_coefficients(cfg: KfacConfig, cg: dict, Delta: np.ndarray, delta: Optional[np.ndarray],
                           grad: np.ndarray) -> Tuple[float, float]:
    """(α*, μ*) minimising the quadratic model m(αΔ + μδ) with the exact damped
    Gramian G + λI (Sec. 3.4, after Martens & Grosse 2015, Sec. 7).  On the
    first step (δ = 0) the model is minimised over α alone and μ* = 0."""
    lam = cfg.lam
    W = None if cfg.residual is None else cfg.residual.weight()
    unpack = lambda v: unpack_theta(v, cfg.d, cfg.widths)
    jD = residual_jvp(cg, unpack(Delta))
    a11 = gramian_bilinear(jD, jD, W) + lam * float(Delta @ Delta)
    b1 = float(Delta @ grad)
    if delta is None or not np.any(delta):
        return -b1 / a11, 0.0
    jd = residual_jvp(cg, unpack(delta))
    a12 = gramian_bilinear(jD, jd, W) + lam * float(Delta @ delta)
    a22 = gramian_bilinear(jd, jd, W) + lam * float(delta @ delta)
    b2 = float(delta @ grad)
    alpha, mu = -np.linalg.solve(np.array([[a11, a12], [a12, a22]]), np.array([b1, b2]))
    return float(alpha), float(mu)


def kfac_step(cfg: KfacConfig, state: KfacState, theta: np.ndarray,
              X_int, f, X_bdy, g) -> StepResult:
    Ws = unpack_theta(theta, cfg.d, cfg.widths)
    cg = curvature_and_gradient(cfg, Ws, X_int, f, X_bdy, g)
    Ai, Bi, Ab, Bb = cg["factors"]
    beta = cfg.beta
    for l in range(len(Ws)):    # exponential moving average (Sec. 3.4)
        state.A_int[l] = beta * state.A_int[l] + (1 - beta) * Ai[l]
        state.B_int[l] = beta * state.B_int[l] + (1 - beta) * Bi[l]
        state.A_bdy[l] = beta * state.A_bdy[l] + (1 - beta) * Ab[l]
        state.B_bdy[l] = beta * state.B_bdy[l] + (1 - beta) * Bb[l]
    direction, dhat = [], []
    for l in range(len(Ws)):
        D = kron_sum_inverse_apply(state.A_int[l], state.B_int[l], state.A_bdy[l],
                                   state.B_bdy[l], cg["grads"][l], cfg.lam, cfg.damping_sqrt)
        direction.append(D)
        dhat.append(D if (state.delta_prev is None) else cfg.momentum * state.delta_prev[l] + D)
    extras = dict(cg)
    if cfg.kfac_star:
        # KFAC*: δ_t = α* Δ_t + μ* δ_{t-1} (Sec. 3.4)
        prev = None if state.delta_prev is None else pack_theta(state.delta_prev)
        alpha, mu = kfac_star_coefficients(cfg, cg, pack_theta(direction), prev, pack_theta(cg["grads"]))
        extras["alpha"], extras["mu"] = alpha, mu
        update = [alpha * direction[l] + (0.0 if prev is None else mu * state.delta_prev[l])
                  for l in range(len(Ws))]
        state.delta_prev = update
        state.t += 1
        theta_new = theta + pack_theta(update)
        return StepResult(cg["loss"], cg["grads"], (list(state.A_int), list(state.B_int),
                          list(state.A_bdy), list(state.B_bdy)), direction, update, theta_new,
                          extras=extras)
    if cfg.line_search:
        alpha, extras["line_search_losses"] = line_search(cfg, theta, pack_theta(dhat), X_int, f, X_bdy, g)
        extras["alpha"] = alpha
    else:
        alpha = cfg.lr
    # with no finite trial the line search makes no step (α* = 0, reading of Sec. 3.4)
    update = [alpha * v if alpha != 0.0 else np.zeros_like(v) for v in dhat]
    state.delta_prev = update
    state.t += 1
    theta_new = theta + pack_theta(update)
    return StepResult(cg["loss"], cg["grads"], (list(state.A_int), list(state.B_int),
                      list(state.A_bdy), list(state.B_bdy)), direction, update, theta_new,
                      extras=extras)


# ---------------------------------------------------------------------------
# Brute force (Eq. 2 and Eq. 7) for tiny nets
# ---------------------------------------------------------------------------


def exact_interior_block(T_in_l: np.ndarray, Zbar_l: np.ndarray) -> np.ndarray:
    """Eq. 7: (1/N) Σ_n Σ_{s,s'} T̂_s T̂_{s'}ᵀ ⊗ g_s g_{s'}ᵀ = (1/N) Σ_n vec J_n vec J_nᵀ."""
    J = weight_jacobian(Zbar_l, T_in_l)
    N = J.shape[0]
    v = np.stack([J[n].reshape(-1, order="F") for n in range(N)])
    return v.T @ v / N


def full_ggn(cfg: KfacConfig, Ws, X_int, f, X_bdy, g) -> np.ndarray:
    """Eq. 2: G = (1/N_Ω) Σ J_θ r_nᵀ J_θ r_n + (1/N_∂) Σ J_θ r^bᵀ J_θ r^b (D x D)."""
    cg = curvature_and_gradient(cfg, Ws, X_int, f, X_bdy, g)

    def jac_rows(fp, zb):
        N = zb[0].shape[0]
        rows = []
        for n in range(N):
            rows.append(np.concatenate([
                weight_jacobian(zb[l][n:n + 1], fp.T_in[l][n:n + 1])[0].reshape(-1, order="F")
                for l in range(len(Ws))]))
        return np.stack(rows)

    Jb = jac_rows(cg["fp_b"], cg["zb_b"])
    Gb = Jb.T @ Jb / Jb.shape[0]
    if "zb_i_k" in cg:     # Σ_n J_nᵀ Λ J_n with the rows of J_n per residual output (Sec. 3.3)
        W = cfg.residual.weight()
        Jk = [jac_rows(cg["fp_i"], zb) for zb in cg["zb_i_k"]]
        N = Jk[0].shape[0]
        Gi = sum(W[k, kk] * (Jk[k].T @ Jk[kk]) for k in range(len(Jk)) for kk in range(len(Jk))) / N
        return Gi + Gb
    Ji = jac_rows(cg["fp_i"], cg["zb_i"])
    return Ji.T @ Ji / Ji.shape[0] + Gb


def relative_l2(u: np.ndarray, u_star: np.ndarray) -> float:
    return float(np.linalg.norm(u - u_star) / np.linalg.norm(u_star))
