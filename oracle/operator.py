"""Discrete Helmholtz operator with PML (oracle; test infrastructure only).

Eq. (2) (1D) discretizes ((s d/dx)^2 + omega^2/c^2) u = f with central
differences and step h = 1/(n+1):

    (s_i/h) [ (s_{i+1/2}/h)(u_{i+1} - u_i) - (s_{i-1/2}/h)(u_i - u_{i-1}) ]
        + omega^2/c_i^2 u_i = f_i,

where a subscript i means "evaluated at x = i h" and u_0 = u_{n+1} = 0.
Eq. (4) (2D) and Eq. (5) (3D) add one such term per axis.  The experiments put
the PML on every side (Sections 3.2 and 4.2), so every axis carries its own
s-profile; the grid ordering is the paper's column-major one (x1 fastest).

Arrays are numpy arrays indexed ``u[i_d-1, ..., i1-1]`` (sweep axis x_d first).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .pml import Profile, global_profile


def second_difference(lo: int, hi: int, n: int, prof: Profile, omega: float) -> sp.csr_matrix:
    """The 1D PML second difference of Eq. (2) restricted to grid nodes lo..hi
    (global 1-based indices), Dirichlet zero at nodes lo-1 and hi+1.

    Row i: coefficient s_i s_{i+1/2}/h^2 on u_{i+1}, s_i s_{i-1/2}/h^2 on
    u_{i-1} and -s_i (s_{i+1/2} + s_{i-1/2})/h^2 on u_i.
    """
    h = 1.0 / (n + 1)
    idx = np.arange(lo, hi + 1, dtype=np.float64)
    s = prof.s(idx * h, omega)
    sp_ = prof.s((idx + 0.5) * h, omega)
    sm_ = prof.s((idx - 0.5) * h, omega)
    up = s * sp_ / h**2
    dn = s * sm_ / h**2
    main = -(up + dn)
    w = hi - lo + 1
    return sp.diags([dn[1:], main, up[:-1]], [-1, 0, 1], shape=(w, w), format="csr",
                    dtype=np.complex128)


def transverse_operator(dim: int, n: int, gamma: int, C: float, omega: float) -> sp.csr_matrix:
    """Sum of the PML second differences along the non-sweep axes x1 (and x2
    in 3D), on the flattened transverse index t (x1 fastest).  Identity-sized
    1x1 zero for dim = 1."""
    if dim == 1:
        return sp.csr_matrix((1, 1), dtype=np.complex128)
    g = global_profile(n, gamma, C)
    D = second_difference(1, n, n, g, omega)
    if dim == 2:
        return D.tocsr()
    I = sp.identity(n, dtype=np.complex128, format="csr")
    # t = i2*n + i1: kron(D_x2, I) acts on i2, kron(I, D_x1) on i1.
    return (sp.kron(D, I) + sp.kron(I, D)).tocsr()


def helmholtz_matrix(dim: int, n: int, omega: float, c: np.ndarray, gamma: int,
                     C: float) -> sp.csr_matrix:
    """A of Eq. (2)/(4)/(5) with PML of width gamma*h on every side, in the
    paper's column-major ordering (x1 fastest, the sweep axis x_d slowest)."""
    T = n ** (dim - 1)
    g = global_profile(n, gamma, C)
    Ds = second_difference(1, n, n, g, omega)
    Dt = transverse_operator(dim, n, gamma, C, omega)
    k2 = (omega**2 / np.asarray(c, dtype=np.float64) ** 2).reshape(-1)
    A = sp.kron(Ds, sp.identity(T, format="csr")) + sp.diags(k2.astype(np.complex128))
    if dim > 1:
        A = A + sp.kron(sp.identity(n, format="csr"), Dt)
    return A.tocsr()


def apply_A(dim: int, n: int, omega: float, c: np.ndarray, gamma: int, C: float,
            u: np.ndarray) -> np.ndarray:
    """y = A u for one grid function ``u`` (shape (n,)*dim) or a batch with a
    trailing right-hand-side axis."""
    A = helmholtz_matrix(dim, n, omega, c, gamma, C)
    N = n**dim
    if u.ndim == dim:
        return (A @ u.reshape(N)).reshape(u.shape)
    R = u.shape[-1]
    return (A @ u.reshape(N, R)).reshape(u.shape)
