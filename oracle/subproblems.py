"""Auxiliary problems H_q^M, H_p^R, H_p^L and operators G~ (oracle; test
infrastructure only).

Section 3.1 ("Auxiliary problems") defines each H as the discretization of the
Helmholtz operator on a padded grid X^M / X^R / X^L, with the boundary PML kept
on the transverse axes and the sweep-axis s replaced by the auxiliary profile,
and Dirichlet conditions on the padded grid's boundary.  "Auxiliary Green's
operators" then defines

* G~_q^M y: put y on X_q, zero elsewhere on X_q^M; solve H_q^M v = g; restrict v to X_q;
* G~_p^R w: g = (-1/h^2) [w, 0, ..., 0] (w on the first sweep column);
  solve H_p^R v = g; restrict v to X_p;
* G~_p^L w: g = (-1/h^2) [0, ..., 0, w] (w on the last sweep column);
  solve H_p^L v = g; restrict v to X_p.

The quasi-1D remark after "Putting together" (Section 3.1) orders each
subproblem with the sweep axis fastest, which gives a banded matrix of
half-bandwidth w * n^(d-2) (w = padded width); Algorithm 1 factors every
subproblem once.  This module does exactly that with LAPACK's banded LU with
partial pivoting (``zgbtrf``) and solves with ``zgbtrs``.

Array conventions: a grid function on a sweep range [lo, hi] is an array of
shape (hi-lo+1, T) -- sweep index first, transverse index t (x1 fastest)
second, T = n^(d-1).  A batch adds a trailing right-hand-side axis.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg.lapack as lapack
import scipy.sparse as sp

from .operator import second_difference, transverse_operator
from .partition import Partition, sweep_profile


def subproblem_matrix(dim: int, n: int, omega: float, c: np.ndarray, gamma: int, C: float,
                      part: Partition, p: int, kind: str, order: str = "natural") -> sp.csr_matrix:
    """H_p^kind on its padded sweep range.

    ``order='natural'`` returns it in the paper's ordering (x1 fastest, sweep
    axis slowest); ``order='banded'`` in the quasi-1D ordering (sweep axis
    fastest) whose half-bandwidth is w * n^(d-2)."""
    L = part.layers[p - 1]
    lo, hi = {"M": (L.m_lo, L.m_hi), "R": (L.r_lo, L.r_hi), "L": (L.l_lo, L.l_hi)}[kind]
    w = hi - lo + 1
    T = n ** (dim - 1)
    prof = sweep_profile(part, p, kind, C)
    Ds = second_difference(lo, hi, n, prof, omega)
    Dt = transverse_operator(dim, n, gamma, C, omega)
    cc = np.asarray(c, dtype=np.float64).reshape(n, T)[lo - 1:hi, :]  # (w, T)
    k2 = omega**2 / cc**2
    It = sp.identity(T, format="csr", dtype=np.complex128)
    Iw = sp.identity(w, format="csr", dtype=np.complex128)
    if order == "natural":
        H = sp.kron(Ds, It) + sp.diags(k2.reshape(-1).astype(np.complex128))
        if dim > 1:
            H = H + sp.kron(Iw, Dt)
    elif order == "banded":
        H = sp.kron(It, Ds) + sp.diags(k2.T.reshape(-1).astype(np.complex128))
        if dim > 1:
            H = H + sp.kron(Dt, Iw)
    else:
        raise ValueError(order)
    return H.tocsr()


def to_lapack_band(H: sp.spmatrix, kl: int, ku: int) -> np.ndarray:
    """Band storage for ?gbtrf: ab[kl + ku + i - j, j] = H[i, j], with kl extra
    rows on top for the fill of partial pivoting."""
    Hc = H.tocoo()
    Hc.eliminate_zeros()  # explicit zeros from sparse sums carry no coupling
    N = H.shape[0]
    ab = np.zeros((2 * kl + ku + 1, N), dtype=np.complex128)
    if np.any(Hc.row - Hc.col > kl) or np.any(Hc.col - Hc.row > ku):
        raise ValueError("matrix exceeds the stated bandwidth")
    ab[kl + ku + Hc.row - Hc.col, Hc.col] = Hc.data
    return ab


@dataclasses.dataclass
class Factored:
    """One factored subproblem: banded LU of H_p^kind in the quasi-1D order."""

    kind: str
    p: int
    lo: int  # padded sweep range [lo, hi]
    hi: int
    x_lo: int  # X_p inside it
    x_hi: int
    T: int
    kl: int
    lu: np.ndarray
    ipiv: np.ndarray

    @property
    def w(self) -> int:
        return self.hi - self.lo + 1

    def solve(self, g: np.ndarray) -> np.ndarray:
        """v = H^-1 g for g of shape (w, T) or (w, T, R)."""
        batch = g.ndim == 3
        G = g if batch else g[..., None]
        R = G.shape[-1]
        # natural (sweep, t) -> banded index t*w + j
        gb = np.ascontiguousarray(np.transpose(G, (1, 0, 2)).reshape(self.T * self.w, R))
        x, info = lapack.zgbtrs(self.lu, self.kl, self.kl, gb, self.ipiv)
        if info != 0:
            raise RuntimeError(f"zgbtrs info={info}")
        v = np.transpose(x.reshape(self.T, self.w, R), (1, 0, 2))
        return v if batch else v[..., 0]


def factor_subproblem(dim: int, n: int, omega: float, c: np.ndarray, gamma: int, C: float,
                      part: Partition, p: int, kind: str) -> Factored:
    """Algorithm 1, one subproblem: banded LU of H_p^kind (partial pivoting)."""
    L = part.layers[p - 1]
    lo, hi = {"M": (L.m_lo, L.m_hi), "R": (L.r_lo, L.r_hi), "L": (L.l_lo, L.l_hi)}[kind]
    w = hi - lo + 1
    T = n ** (dim - 1)
    kl = 1 if dim == 1 else w * n ** (dim - 2)
    H = subproblem_matrix(dim, n, omega, c, gamma, C, part, p, kind, order="banded")
    ab = to_lapack_band(H, kl, kl)
    lu, ipiv, info = lapack.zgbtrf(ab, kl, kl)
    if info != 0:
        raise RuntimeError(f"zgbtrf info={info} for {kind}{p}")
    return Factored(kind, p, lo, hi, L.x_lo, L.x_hi, T, kl, lu, ipiv)


def G_M(F: Factored, y: np.ndarray) -> np.ndarray:
    """G~_q^M y: embed y (on X_q) in X_q^M, solve, restrict to X_q."""
    g = np.zeros((F.w,) + y.shape[1:], dtype=np.complex128)
    a = F.x_lo - F.lo
    g[a:a + y.shape[0]] = y
    v = F.solve(g)
    return v[a:a + (F.x_hi - F.x_lo + 1)]


def G_R(F: Factored, w: np.ndarray, h: float) -> np.ndarray:
    """G~_p^R w: g = (-1/h^2)[w, 0, ..., 0]; solve H_p^R v = g; restrict to X_p."""
    g = np.zeros((F.w,) + w.shape, dtype=np.complex128)
    g[0] = -w / h**2
    v = F.solve(g)
    a = F.x_lo - F.lo
    return v[a:a + (F.x_hi - F.x_lo + 1)]


def G_L(F: Factored, w: np.ndarray, h: float) -> np.ndarray:
    """G~_p^L w: g = (-1/h^2)[0, ..., 0, w]; solve H_p^L v = g; restrict to X_p."""
    g = np.zeros((F.w,) + w.shape, dtype=np.complex128)
    g[-1] = -w / h**2
    v = F.solve(g)
    a = F.x_lo - F.lo
    return v[a:a + (F.x_hi - F.x_lo + 1)]
