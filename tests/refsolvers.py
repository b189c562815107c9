"""Independent ROF solvers and operators used to pin the oracle.

Nothing here calls the oracle or the CUDA library. The operators are built as explicit
matrices from the textbook definition of forward differences, and the divergence is taken as
the literal negative transpose of that matrix, so a wrong index or boundary case in either
implementation under test shows up as a mismatch.

* ``grad_matrix``   -- the (2N x N) forward-difference matrix with a zero last row/column.
* ``rof_fista``     -- one ROF step  min_u 1/2|u-g|^2 + lam TV(u)  (Eq. ROF) solved on the dual
  by FISTA with adaptive restart (Beck & Teboulle 2009; O'Donoghue & Candes 2015), stopped by
  the duality gap, which bounds |u - u*|^2 <= 2 gap.
* ``rof_1d_bvls``   -- the 1-D ROF step solved exactly: its dual is a bound-constrained least
  squares problem, handed to scipy's active-set BVLS solver.
"""
from __future__ import annotations

import numpy as np


def grad_matrix(H: int, W: int) -> np.ndarray:
    """Rows 0..N-1: (grad u)^1 (along i); rows N..2N-1: (grad u)^2 (along j)."""
    N = H * W
    D = np.zeros((2 * N, N))
    for i in range(H):
        for j in range(W):
            n = i * W + j
            if i < H - 1:
                D[n, n] = -1.0
                D[n, n + W] = 1.0
            if j < W - 1:
                D[N + n, n] = -1.0
                D[N + n, n + 1] = 1.0
    return D


def tv_iso(u: np.ndarray, D: np.ndarray) -> float:
    """Isotropic discrete TV: sum over pixels of the Euclidean norm of the gradient (Eq. TV)."""
    N = u.size
    g = D @ u.ravel()
    return float(np.sum(np.sqrt(g[:N] ** 2 + g[N:] ** 2)))


def rof_gap(g: np.ndarray, lam: float, q: np.ndarray, D: np.ndarray):
    """Primal point u = g - lam D^T q and the gap P(u) - D(q) (q is dual-feasible)."""
    gv = g.ravel()
    u = gv - lam * (D.T @ q)
    primal = 0.5 * np.sum((u - gv) ** 2) + lam * tv_iso(u, D)
    dual = 0.5 * np.sum(gv ** 2) - 0.5 * np.sum(u ** 2)
    return u.reshape(g.shape), float(primal - dual)


def _project(q: np.ndarray, N: int) -> np.ndarray:
    a, b = q[:N], q[N:]
    n = np.maximum(1.0, np.sqrt(a * a + b * b))
    return np.concatenate([a / n, b / n])


def rof_fista(g: np.ndarray, lam: float, gap_tol: float = 1e-24, max_iter: int = 400000):
    """Dual FISTA with gradient restart for  max_{|q_ij|<=1}  (dual of Eq. ROF).

    The dual objective to minimise is  1/2 |g - lam D^T q|^2  over pointwise unit balls; its
    gradient is  -lam D (g - lam D^T q), Lipschitz with constant lam^2 |D|^2.
    Returns (u, gap, iterations).
    """
    H, W = g.shape
    N = H * W
    D = grad_matrix(H, W)
    L = lam * lam * np.linalg.norm(D, 2) ** 2
    gv = g.ravel()
    q = np.zeros(2 * N)
    y = q.copy()
    t = 1.0
    gap = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        r = gv - lam * (D.T @ y)
        q_new = _project(y + (lam / L) * (D @ r), N)
        # restart when the momentum points uphill
        if np.dot(y - q_new, q_new - q) > 0:
            t = 1.0
            y = q_new.copy()
        else:
            t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
            y = q_new + ((t - 1.0) / t_new) * (q_new - q)
            t = t_new
        q = q_new
        if it % 200 == 0:
            _, gap = rof_gap(g, lam, q, D)
            if gap <= gap_tol:
                break
    u, gap = rof_gap(g, lam, q, D)
    return u, gap, it


def rof_1d_bvls(g: np.ndarray, lam: float) -> np.ndarray:
    """Exact 1-D ROF step  min_u 1/2|u-g|^2 + lam sum_i |u_{i+1}-u_i|.

    Dual: u = g + lam D^T q with D the (n-1 x n) forward difference and |q_i| <= 1, where q
    minimises |g + lam D^T q|^2 -- a bounded least-squares problem (Stark & Parker BVLS).
    """
    from scipy.optimize import lsq_linear

    g = np.asarray(g, dtype=np.float64).ravel()
    n = g.size
    if n == 1:
        return g.copy()
    D = np.zeros((n - 1, n))
    for i in range(n - 1):
        D[i, i] = -1.0
        D[i, i + 1] = 1.0
    A = lam * D.T
    res = lsq_linear(A, -g, bounds=(-1.0, 1.0), method="bvls", tol=1e-15,
                     lsq_solver="exact", max_iter=100000)
    return g + A @ res.x
