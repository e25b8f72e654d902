"""Post-processing and error norms (Sec. 3.5 and Sec. 6.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import numpy as np

OUTPUT_NAMES = ["v_x", "v_y", "j_s", "j_d", "j_xy", "u_x", "u_y", "sigma_xx", "sigma_yy", "sigma_xy"]


def outputs_from_moments(U, ustar, dt, cK, cmu):
    """[v (2), j (3), u (2), sigma (3)] from U^num and u* (V = 1).

    v^num = first two rows of U^num; u^num = u* + dt/2 v^num (step 1(b));
    sigma^num = -[cK j_s + cmu j_d, cK j_s - cmu j_d, cmu j_xy] (Eq. sigma_num).
    """
    v = U[0:2]
    u = ustar + 0.5 * dt * v
    sxx = -(cK * U[2] + cmu * U[3])
    syy = -(cK * U[2] - cmu * U[3])
    sxy = -(cmu * U[4])
    return np.concatenate([U, u, sxx[None], syy[None], sxy[None]], axis=0)


class SpaceTimeNorms:
    """Accumulates the space-time L2 and Linf norms of Sec. 6.1 over t in T.

    L2(e) = (dx^2 dt sum_{x,t} |e|^2)^(1/2), |.| Euclidean over the field's components;
    Linf(e) = max_{x,t} |e|_inf.  ``relative`` divides both by L2 of the exact field.
    """

    def __init__(self, dx, dt):
        self.dx, self.dt = dx, dt
        self.sq_err = 0.0
        self.sq_ref = 0.0
        self.max_err = 0.0

    def add(self, num, exact):
        e = np.asarray(num) - np.asarray(exact)
        self.sq_err += float(np.sum(e * e))
        self.sq_ref += float(np.sum(np.asarray(exact) ** 2))
        self.max_err = max(self.max_err, float(np.max(np.abs(e))))

    @property
    def L2(self):
        return float(np.sqrt(self.dx ** 2 * self.dt * self.sq_err))

    @property
    def L2_exact(self):
        return float(np.sqrt(self.dx ** 2 * self.dt * self.sq_ref))

    @property
    def Linf(self):
        return self.max_err

    @property
    def L2rel(self):
        return self.L2 / self.L2_exact

    @property
    def Linfrel(self):
        return self.Linf / self.L2_exact


def rel_l2(a, b):
    """Relative L2 difference ||a - b|| / ||b|| of one field (plain, no weights)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.sqrt(np.sum(b * b)))
    return float(np.sqrt(np.sum((a - b) ** 2))) / nb if nb > 0 else float(np.sqrt(np.sum(a * a)))
