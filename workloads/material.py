"""Material and time-step mapping (Sec. 2.1, Eq. stab_cond).

Input generation only.  With density 1 and Lame constants (lam, mu), the law of
Eq. cauchy gives cK^2 = lam + mu and cmu^2 = mu (plane strain: cK^2 = (3K+mu)/3
with K = lam + 2 mu / 3).  The plane-strain Poisson ratio nu = lam / (2 (lam+mu))
fixes cK^2 / cmu^2 = 1 / (1 - 2 nu).
"""
from __future__ import annotations

import math


def lame_to_speeds(lam: float, mu: float):
    """(cK^2, cmu^2) for density 1."""
    return lam + mu, mu


def poisson_to_speeds(nu: float, total: float = 2.0):
    """(cK^2, cmu^2) with cK^2 + cmu^2 = total and plane-strain Poisson ratio nu."""
    ratio = 1.0 / (1.0 - 2.0 * nu)          # cK^2 / cmu^2
    cmu2 = total / (1.0 + ratio)
    return total - cmu2, cmu2


def lattice_speed(cK2: float, cmu2: float, cfl_fraction: float) -> float:
    """c = dx/dt such that 2 sqrt(cK^2 + cmu^2) / c = cfl_fraction (Eq. stab_cond)."""
    return 2.0 * math.sqrt(cK2 + cmu2) / cfl_fraction


def cfl_ratio(cK2: float, cmu2: float, c: float) -> float:
    return 2.0 * math.sqrt(cK2 + cmu2) / c
