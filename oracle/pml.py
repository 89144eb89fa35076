"""PML profiles (oracle; test infrastructure only).

Section 2 defines, on [0, 1] with PML width eta = gamma*h,

    sigma(x) = (C/eta) * ((x - eta)/eta)^2        for x in [0, eta),
             = 0                                  for x in [eta, 1 - eta],
             = (C/eta) * ((x - 1 + eta)/eta)^2    for x in (1 - eta, 1],
    s(x)     = (1 + i sigma(x)/omega)^-1.

Every auxiliary profile of Sections 2.1.1-2.1.3 and 3.1 (sigma_q^M, sigma_p^R,
sigma_p^L) has the same shape: zero on a closed interval [lo_edge, hi_edge]
and (C/eta)(d/eta)^2 at distance d outside it, on the sides that carry a PML.
:class:`Profile` states a profile by those two edges and the width used on
each side (``None`` = no PML on that side).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Profile:
    """sigma(x) = 0 on [lo_edge, hi_edge]; quadratic PML of width eta_lo / eta_hi
    outside it.  ``lo_edge=None`` (``hi_edge=None``) means no PML on that side."""

    lo_edge: float | None
    hi_edge: float | None
    eta_lo: float
    eta_hi: float
    C: float

    def sigma(self, x):
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros_like(x)
        if self.lo_edge is not None:
            d = self.lo_edge - x
            msk = d > 0
            out = np.where(msk, (self.C / self.eta_lo) * (d / self.eta_lo) ** 2, out)
        if self.hi_edge is not None:
            d = x - self.hi_edge
            msk = d > 0
            out = np.where(msk, (self.C / self.eta_hi) * (d / self.eta_hi) ** 2, out)
        return out

    def s(self, x, omega: float):
        """s(x) = (1 + i sigma(x)/omega)^-1."""
        return 1.0 / (1.0 + 1j * self.sigma(x) / omega)


def global_profile(n: int, gamma: int, C: float) -> Profile:
    """The boundary PML of the unit interval (Section 2): eta = gamma*h on both
    ends, zero on [eta, 1 - eta] = [gamma*h, (n+1-gamma)*h]."""
    h = 1.0 / (n + 1)
    eta = gamma * h
    return Profile(gamma * h, (n + 1 - gamma) * h, eta, eta, C)
