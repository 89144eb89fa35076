"""The additive sweeping preconditioner (oracle; test infrastructure only).

:class:`Preconditioner` follows Algorithm 1 (setup: factor H_q^M for q=1..m,
H_p^R for p=2..m, H_p^L for p=1..m-1) and Algorithm 2 (apply) of Section 3.1,
which is the same for 1D (Section 2.2) and 3D (Algorithms 3/4 with the banded
LU standing in for nested dissection):

    u~_{q,q}     = G~_q^M f_q                                     q = 1..m
    u~_{p,1:p-1} = G~_p^R (u~_{p-1,1:p-1})^R,
    (u~_{p,1:p})^R = (u~_{p,1:p-1})^R + (u~_{p,p})^R             p = 2..m
    u~_{p,p+1:m} = G~_p^L (u~_{p+1,p+1:m})^L,
    (u~_{p,p:m})^L = (u~_{p,p})^L + (u~_{p,p+1:m})^L             p = m-1..1
    u~_1 = u~_{1,1} + u~_{1,2:m},  u~_p = u~_{p,1:p-1} + u~_{p,p} + u~_{p,p+1:m},
    u~_m = u~_{m,1:m-1} + u~_{m,m},

where g^R (g^L) is the last (first) sweep column of a layer array.
:meth:`Preconditioner.apply_naive` is the O(m^2) definition of Section 2.1
(u~_{p,q} for every pair, then u~_p = sum_q u~_{p,q}), used only to pin the
accumulation above.
"""
from __future__ import annotations

import numpy as np

from .partition import Partition, make_partition
from .subproblems import G_L, G_M, G_R, Factored, factor_subproblem


class Preconditioner:
    """Algorithm 1 at construction, Algorithm 2 in :meth:`apply`."""

    def __init__(self, dim: int, n: int, omega: float, c: np.ndarray, gamma: int, b: int,
                 C: float = 20.0, gamma_a: int | None = None, layers=None, widths=None):
        self.dim, self.n, self.omega, self.gamma, self.b, self.C = dim, n, omega, gamma, b, C
        self.c = np.asarray(c, dtype=np.float64)
        # widths: physical layer widths b_1..b_m (Section 3.1, practical remark 3);
        # None = b columns per layer, the last absorbing the remainder
        self.part: Partition = make_partition(n, gamma, b, gamma_a, widths)
        self.T = n ** (dim - 1)
        m = self.part.m
        args = (dim, n, omega, self.c, gamma, C, self.part)
        # Algorithm 1 (optionally restricted to a subset of layers, for sampling)
        want = set(range(1, m + 1)) if layers is None else set(layers)
        self.FM: dict[int, Factored] = {q: factor_subproblem(*args, q, "M") for q in want}
        self.FR: dict[int, Factored] = {p: factor_subproblem(*args, p, "R")
                                        for p in want if p >= 2}
        self.FL: dict[int, Factored] = {p: factor_subproblem(*args, p, "L")
                                        for p in want if p <= m - 1}

    @property
    def m(self) -> int:
        return self.part.m

    @property
    def h(self) -> float:
        return 1.0 / (self.n + 1)

    def _split(self, f: np.ndarray) -> list:
        """f (shape (n, T[, R])) -> [f_1, ..., f_m] restricted to X_p."""
        return [f[L.x_lo - 1:L.x_hi] for L in self.part.layers]

    def _join(self, parts: list, like: np.ndarray) -> np.ndarray:
        out = np.zeros_like(like, dtype=np.complex128)
        for L, u in zip(self.part.layers, parts):
            out[L.x_lo - 1:L.x_hi] = u
        return out

    def _as_layers(self, r: np.ndarray):
        """Accept (n,)*dim or (n,)*dim + (R,) arrays; return (n, T[, R])."""
        batch = r.ndim == self.dim + 1
        shape = (self.n, self.T) + ((r.shape[-1],) if batch else ())
        return r.reshape(shape)

    def apply(self, r: np.ndarray) -> np.ndarray:
        """z = M^-1 r by Algorithm 2 (accumulated boundary values)."""
        f = self._as_layers(np.asarray(r, dtype=np.complex128))
        m, h = self.m, self.h
        fp = self._split(f)
        uqq = [G_M(self.FM[q], fp[q - 1]) for q in range(1, m + 1)]
        # right-going sweep: uR[p] = u~_{p,1:p-1}
        uR = [None] * (m + 1)
        acc = uqq[0][-1]  # (u~_{1,1})^R
        for p in range(2, m + 1):
            uR[p] = G_R(self.FR[p], acc, h)
            acc = uR[p][-1] + uqq[p - 1][-1]
        # left-going sweep: uL[p] = u~_{p,p+1:m}
        uL = [None] * (m + 1)
        acc = uqq[m - 1][0]  # (u~_{m,m})^L
        for p in range(m - 1, 0, -1):
            uL[p] = G_L(self.FL[p], acc, h)
            acc = uqq[p - 1][0] + uL[p][0]
        out = []
        for p in range(1, m + 1):
            u = uqq[p - 1].copy()
            if p >= 2:
                u = u + uR[p]
            if p <= m - 1:
                u = u + uL[p]
            out.append(u)
        return self._join(out, f).reshape(np.shape(r))

    def apply_naive(self, r: np.ndarray) -> np.ndarray:
        """u~_p = sum_q u~_{p,q} with every u~_{p,q} computed separately
        (Section 2.1.3: u~_{q,q} = G~_q^M f_q, u~_{p,q} = G~_p^R u~_{p-1,q}^R for
        p > q and G~_p^L u~_{p+1,q}^L for p < q).  O(m^2) subproblem solves."""
        f = self._as_layers(np.asarray(r, dtype=np.complex128))
        m, h = self.m, self.h
        fp = self._split(f)
        tot = [np.zeros_like(x) for x in fp]
        for q in range(1, m + 1):
            u = G_M(self.FM[q], fp[q - 1])
            tot[q - 1] = tot[q - 1] + u
            cur = u
            for p in range(q + 1, m + 1):
                cur = G_R(self.FR[p], cur[-1], h)
                tot[p - 1] = tot[p - 1] + cur
            cur = u
            for p in range(q - 1, 0, -1):
                cur = G_L(self.FL[p], cur[0], h)
                tot[p - 1] = tot[p - 1] + cur
        return self._join(tot, f).reshape(np.shape(r))
