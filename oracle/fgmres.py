"""Right-preconditioned flexible GMRES (oracle; test infrastructure only).

Section 3.2 runs GMRES with a relative-residual tolerance and restart 40 around
the preconditioner.  The readings taken here: right preconditioning in its
flexible form (the preconditioned vectors z_j = M^-1 v_j are stored, so the
GMRES residual is the true residual of A x = f), zero initial guess, modified
Gram-Schmidt, complex Givens rotations, stop when the residual estimate
|g_{j+1}| / ||f|| <= tol, restart with the true residual.

The iteration count is the number of preconditioner applications.
"""
from __future__ import annotations

import numpy as np


def givens(a: complex, b: complex):
    """(c, s) with c real such that [[c, s], [-conj(s), c]] @ [a, b] = [r, 0]."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    rho = np.hypot(abs(a), abs(b))
    c = abs(a) / rho
    s = (a / abs(a)) * np.conj(b) / rho
    return c, s


def fgmres(matvec, precond, f: np.ndarray, tol: float = 1e-6, restart: int = 40,
           maxit: int = 400, fixed_iters: int | None = None):
    """Solve A x = f for one right-hand side (a flat complex vector).

    ``fixed_iters``: run exactly that many iterations (tol ignored), used to
    compare two implementations at the same Krylov dimension.
    Returns (x, iterations, history) with history[k] = residual estimate / ||f||
    after k iterations (history[0] = 1).
    """
    f = np.asarray(f, dtype=np.complex128).ravel()
    N = f.size
    x = np.zeros(N, dtype=np.complex128)
    fnorm = np.linalg.norm(f)
    hist = [1.0]
    if fnorm == 0.0:
        return x, 0, hist
    limit = fixed_iters if fixed_iters is not None else maxit
    its = 0
    while its < limit:
        r = f - matvec(x)
        beta = np.linalg.norm(r)
        if fixed_iters is None and beta / fnorm <= tol:
            break
        k_max = min(restart, limit - its)
        V = np.zeros((k_max + 1, N), dtype=np.complex128)
        Z = np.zeros((k_max, N), dtype=np.complex128)
        H = np.zeros((k_max + 1, k_max), dtype=np.complex128)
        cs = np.zeros(k_max)
        sn = np.zeros(k_max, dtype=np.complex128)
        g = np.zeros(k_max + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k = 0
        done = False
        for j in range(k_max):
            Z[j] = precond(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):  # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            hjj = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            hj1 = H[j + 1, j]
            H[j, j] = hjj
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / fnorm)
            if fixed_iters is None and abs(g[j + 1]) / fnorm <= tol:
                done = True
                break
            if hj1 == 0.0:  # happy breakdown: exact solution in the space
                done = True
                break
            V[j + 1] = w / hj1
        # y = H[:k,:k]^-1 g[:k] (upper triangular), x += Z y
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + y @ Z[:k]
        if done:
            break
    return x, its, hist


def solve(precond_obj, A, f: np.ndarray, tol: float = 1e-6, restart: int = 40,
          maxit: int = 400, fixed_iters: int | None = None):
    """FGMRES for each right-hand side in ``f`` (shape (n,)*dim + (R,)).

    Returns (u, iterations[R], true relative residuals[R]).
    """
    R = f.shape[-1]
    shape = f.shape[:-1]
    u = np.zeros(f.shape, dtype=np.complex128)
    its, res = [], []
    for r in range(R):
        fr = f[..., r].reshape(-1)
        x, k, _ = fgmres(lambda v: A @ v,
                         lambda v: precond_obj.apply(v.reshape(shape)).reshape(-1),
                         fr, tol, restart, maxit, fixed_iters)
        u[..., r] = x.reshape(shape)
        its.append(k)
        res.append(np.linalg.norm(fr - A @ x) / np.linalg.norm(fr))
    return u, np.array(its), np.array(res)
