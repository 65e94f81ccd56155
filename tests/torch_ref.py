"""Independent autograd route used to pin the oracle (CPU, float64).

A tanh MLP written directly in torch; derivatives come from torch.autograd
(Hessian traces, Jacobians), a library route that shares nothing with the
oracle's Taylor-mode arithmetic.  Test helper only.
"""
import numpy as np
import torch


def unpack(theta: np.ndarray, d: int, widths):
    dims = [d] + list(widths)
    t = torch.as_tensor(theta, dtype=torch.float64)
    out, off = [], 0
    for l in range(1, len(dims)):
        rows, cols = dims[l], dims[l - 1] + 1
        out.append(t[off:off + rows * cols].reshape(cols, rows).T)
        off += rows * cols
    return out


def mlp_from_flat(theta_t: torch.Tensor, d: int, widths):
    dims = [d] + list(widths)

    def net(x):  # x: (d,)
        off = 0
        z = x
        for l in range(1, len(dims)):
            rows, cols = dims[l], dims[l - 1] + 1
            Wt = theta_t[off:off + rows * cols].reshape(cols, rows).T
            off += rows * cols
            z = Wt[:, :-1] @ z + Wt[:, -1]
            if l < len(dims) - 1:
                z = torch.tanh(z)
        return z[0]
    return net


def value_grad_lap(theta: np.ndarray, d: int, widths, X: np.ndarray, lap_coords=None):
    th = torch.as_tensor(theta, dtype=torch.float64)
    net = mlp_from_flat(th, d, widths)
    us, gs, ls = [], [], []
    for x in X:
        xt = torch.as_tensor(x, dtype=torch.float64)
        H = torch.autograd.functional.hessian(net, xt)
        xg = xt.clone().requires_grad_(True)
        u = net(xg)
        (g,) = torch.autograd.grad(u, xg)
        idx = range(d) if lap_coords is None else lap_coords
        us.append(float(u.detach()))
        gs.append(g.numpy())
        ls.append(float(sum(H[i, i] for i in idx)))
    return np.array(us), np.stack(gs), np.array(ls)


def residual_fn(d, widths, op, kappa, coef=None):
    """Returns r(theta_t, x, target, interior) as a torch scalar function."""
    def r(theta_t, x, target, interior):
        net = mlp_from_flat(theta_t, d, widths)
        if not interior:
            return net(x) - target
        xg = x.clone().requires_grad_(True)
        u = net(xg)
        (g,) = torch.autograd.grad(u, xg, create_graph=True)
        if op == "general":                       # sum_ij c_ij d2u/dx_i dx_j - f
            C = torch.as_tensor(coef, dtype=torch.float64)
            tot = 0.0
            for i in range(d):
                (gi,) = torch.autograd.grad(g[i], xg, create_graph=True)
                tot = tot + (C[i] * gi).sum()
            return tot - target
        lap = 0.0
        coords = range(1, d) if op == "heat" else range(d)
        for i in coords:
            (gi,) = torch.autograd.grad(g[i], xg, create_graph=True)
            lap = lap + gi[i]
        if op == "heat":
            return g[0] - kappa * lap - target
        return -lap - target
    return r


def residual_jacobians(theta, d, widths, X, targets, op="laplace", kappa=0.0, interior=True, coef=None):
    """Rows J_θ r_n (N x D) by autograd."""
    rf = residual_fn(d, widths, op, kappa, coef)
    rows = []
    for x, t in zip(X, targets):
        th = torch.as_tensor(theta, dtype=torch.float64).clone().requires_grad_(True)
        val = rf(th, torch.as_tensor(x, dtype=torch.float64), float(t), interior)
        (jr,) = torch.autograd.grad(val, th)
        rows.append(jr.numpy())
    return np.stack(rows)


def residuals(theta, d, widths, X, targets, op="laplace", kappa=0.0, interior=True):
    rf = residual_fn(d, widths, op, kappa)
    th = torch.as_tensor(theta, dtype=torch.float64)
    return np.array([float(rf(th, torch.as_tensor(x, dtype=torch.float64), float(t), interior))
                     for x, t in zip(X, targets)])


def operator_value(theta: np.ndarray, d: int, widths, X: np.ndarray, coef: np.ndarray):
    """sum_ij c_ij d2u/dx_i dx_j per point from the autograd Hessian."""
    th = torch.as_tensor(theta, dtype=torch.float64)
    net = mlp_from_flat(th, d, widths)
    C = torch.as_tensor(coef, dtype=torch.float64)
    out = []
    for x in X:
        H = torch.autograd.functional.hessian(net, torch.as_tensor(x, dtype=torch.float64))
        out.append(float((C * H).sum()))
    return np.array(out)


def taylor_outputs_fn(d, widths, op="laplace"):
    """z(theta_t, x) = (u, du/dx_1, .., du/dx_d, second-order column) by autograd:
    the Laplacian, or the spatial Laplacian (coordinates 1..d-1) for the heat
    operator."""
    def z(theta_t, x):
        net = mlp_from_flat(theta_t, d, widths)
        xg = x.clone().requires_grad_(True)
        u = net(xg)
        (g,) = torch.autograd.grad(u, xg, create_graph=True)
        lap = 0.0
        for i in (range(1, d) if op == "heat" else range(d)):
            (gi,) = torch.autograd.grad(g[i], xg, create_graph=True)
            lap = lap + gi[i]
        return torch.cat([u.reshape(1), g, torch.as_tensor(lap, dtype=torch.float64).reshape(1)])
    return z


def quadratic_residual_rows(theta, d, widths, X, F, b, Q=None, op="laplace"):
    """r_{n,k} = b_k . z_n + 1/2 z_n^T Q_k z_n - F_{n,k} and their Jacobians
    J_theta r_{n,k} (N x M x D) by autograd."""
    zf = taylor_outputs_fn(d, widths, op)
    bt = torch.as_tensor(b, dtype=torch.float64)
    Qt = None if Q is None else torch.as_tensor(Q, dtype=torch.float64)
    rs, Js = [], []
    for x, f in zip(X, F):
        th = torch.as_tensor(theta, dtype=torch.float64).clone().requires_grad_(True)
        z = zf(th, torch.as_tensor(x, dtype=torch.float64))
        r = bt @ z - torch.as_tensor(f, dtype=torch.float64)
        if Qt is not None:
            r = r + 0.5 * torch.einsum("s,kst,t->k", z, Qt, z)
        rows = []
        for k in range(r.shape[0]):
            (jr,) = torch.autograd.grad(r[k], th, retain_graph=True)
            rows.append(jr.numpy())
        rs.append(r.detach().numpy())
        Js.append(np.stack(rows))
    return np.stack(rs), np.stack(Js)
