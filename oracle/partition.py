"""Layers and padded grids along the sweep axis (oracle; test infrastructure only).

Section 2 (1D) and Section 3.1 (2D) partition the sweep axis into m layers

    X_1 = [1, gamma+b-1],  X_p = [gamma+(p-1)b, gamma+pb-1],  X_m = [gamma+(m-1)b, n]

with n = 2 gamma + m b - 2, and pad them with auxiliary PMLs:

    X_q^M = [(q-1)b+1, 2gamma+qb-2],  X_p^R = [gamma+(p-1)b, 2gamma+pb-2],
    X_p^L = [(p-1)b+1, gamma+pb-1].

Readings taken here (each also listed in the design notes):

* The upper end of X_q^M is 2gamma+qb-2 as in the 1D definition; the 2D/3D
  text prints 2gamma+qb-1, which is the Dirichlet node of D_q^M itself.
* Layer widths may be arbitrary (Section 3.1, practical remark 3): with
  P = n+2-2gamma physical nodes, m = floor(P/b) and the last layer absorbs the
  remainder r = P - m b.
* The auxiliary PML width gamma_a may differ from gamma (practical remark 2);
  the boundary PML of X_1 (left) and X_m (right) stays gamma wide.
* The layers' widths b_1, ..., b_m may differ (practical remark 3: widths are
  arbitrary, larger where the velocity varies heavily).  With physical widths
  b_p summing to P, alpha_p = gamma + b_1 + ... + b_{p-1} and
  beta_p = alpha_p + b_p - 1, and the printed ranges above hold with (p-1)b
  replaced by b_1 + ... + b_{p-1}; equal widths b with the remainder on the
  last layer give the formulas as printed.
"""
from __future__ import annotations

import dataclasses

from .pml import Profile


@dataclasses.dataclass(frozen=True)
class Layer:
    p: int  # 1-based layer index
    x_lo: int  # X_p = [x_lo, x_hi] (global 1-based sweep indices)
    x_hi: int
    phys_lo: int  # alpha_p: first node with sigma = 0 in the layer
    phys_hi: int  # beta_p:  last node with sigma = 0 in the layer
    m_lo: int  # X_p^M
    m_hi: int
    r_lo: int  # X_p^R
    r_hi: int
    l_lo: int  # X_p^L
    l_hi: int


@dataclasses.dataclass(frozen=True)
class Partition:
    n: int
    gamma: int
    gamma_a: int
    b: int
    m: int
    layers: tuple

    @property
    def h(self) -> float:
        return 1.0 / (self.n + 1)


def uniform_widths(n: int, gamma: int, b: int) -> list:
    """m = floor(P/b) layers of b physical columns, the last one absorbing the
    remainder P - m b (P = n + 2 - 2 gamma)."""
    P = n + 2 - 2 * gamma
    m = P // b
    if m < 1:
        raise ValueError(f"n={n} too small for gamma={gamma}, b={b}")
    return [b] * (m - 1) + [b + P - m * b]


def make_partition(n: int, gamma: int, b: int, gamma_a: int | None = None, widths=None) -> Partition:
    """Layers of b physical columns (the last absorbing the remainder), or of
    the given physical widths b_1..b_m (summing to P = n + 2 - 2 gamma)."""
    if gamma_a is None:
        gamma_a = gamma
    if gamma < 2 or b < 1 or gamma_a < 1:
        raise ValueError("need gamma >= 2, gamma_a >= 1, b >= 1")
    P = n + 2 - 2 * gamma
    if widths is None:
        widths = uniform_widths(n, gamma, b)
    widths = [int(x) for x in widths]
    if min(widths) < 1 or sum(widths) != P:
        raise ValueError(f"layer widths must be positive and sum to P = {P}")
    m = len(widths)
    layers = []
    alpha = gamma
    for p in range(1, m + 1):
        beta = alpha + widths[p - 1] - 1
        assert p < m or beta == n + 1 - gamma
        x_lo = 1 if p == 1 else alpha
        x_hi = n if p == m else beta
        m_lo = 1 if p == 1 else alpha - gamma_a + 1
        m_hi = n if p == m else beta + gamma_a - 1
        layers.append(Layer(p, x_lo, x_hi, alpha, beta, m_lo, m_hi,
                            alpha, m_hi, m_lo, beta))
        alpha = beta + 1
    return Partition(n, gamma, gamma_a, b, m, tuple(layers))


def sweep_profile(part: Partition, p: int, kind: str, C: float) -> Profile:
    """The sweep-axis PML profile of H_p^M (``kind='M'``), H_p^R (``'R'``) or
    H_p^L (``'L'``), written as zero on [alpha_p h, beta_p h] with a quadratic
    PML past each padded side (sigma_q^M, sigma_p^R, sigma_p^L of Sections
    2.1.1-2.1.3).  The first layer's left side and the last layer's right side
    keep the boundary PML of width gamma."""
    h = part.h
    L = part.layers[p - 1]
    eta = part.gamma * h
    eta_a = part.gamma_a * h
    lo_edge, eta_lo = (L.phys_lo * h, eta if p == 1 else eta_a)
    hi_edge, eta_hi = (L.phys_hi * h, eta if p == part.m else eta_a)
    if kind == "M":
        return Profile(lo_edge, hi_edge, eta_lo, eta_hi, C)
    if kind == "R":
        return Profile(None, hi_edge, eta_lo, eta_hi, C)
    if kind == "L":
        return Profile(lo_edge, None, eta_lo, eta_hi, C)
    raise ValueError(kind)
