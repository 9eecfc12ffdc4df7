"""Oracle of the built-in matrix-free operators (test infrastructure: only tests/,
__graft_entry__.smoke() and bench.py's CPU baseline use it).

Sec. 3.5 lets A be given as a function computing A x; the oracle's Operator accepts
any object with apply(x), n, and the two scalars the method needs from A (R24):
norm_inf, an upper bound of ||A||_inf (Eq. tau_0 and the breakdown threshold), and
nnz, the cost N_A of one product in the units of Eq. (4).  This module writes the
library's built-in function PHIPM_FN_VARCOEF_CONVDIFF out from its definition
(include/phipm.h), in FP64 numpy, for an input object of
paper_0907_4631_gb300.workloads.VarCoefConvDiff (data only):

    (A x)_i = sum_{d<ndim} ( s_d [ kp (x_{i+e_d} - x_i) - km (x_i - x_{i-e_d}) ]
                             - c_d v_{d,i} (x_{i+e_d} - x_{i-e_d}) ),

kp, km the face diffusivities (kappa_i + kappa_neighbour) / 2, kappa_i alone at the
boundary where the neighbour value is 0, s_d = 1/h^2, c_d = 1/(2h).

Pins (tests/test_oracle_matrix_free.py): constant coefficients reproduce the pinned
constant-coefficient stencils (the Dirichlet Laplacian and the convection-diffusion
operator of R14); without convection the product is symmetric and negative definite;
norm_inf equals the largest absolute row sum of the assembled matrix; the full method
with constant kappa meets the sine expansion.
"""
from __future__ import annotations

import numpy as np


class VarCoefConvDiffOperator:
    """The matrix-free operator as the oracle's Operator kind "function"."""

    def __init__(self, data):
        self.ndim = int(data.ndim)
        self.shape = (int(data.nz), int(data.ny), int(data.nx))        # x fastest
        self.n = int(data.nx * data.ny * data.nz)
        self.kappa = np.asarray(data.kappa, dtype=np.float64).reshape(self.shape)
        self.vel = [None if v is None else np.asarray(v, dtype=np.float64).reshape(self.shape)
                    for v in list(data.vel)[: self.ndim]]
        self.vel += [None] * (self.ndim - len(self.vel))
        self.s = 1.0 / (data.h * data.h)
        self.c = 1.0 / (2.0 * data.h)
        dims = (data.nx, data.ny, data.nz)[: self.ndim]
        self.nnz = self.n + sum(2 * (self.n // nd) * (nd - 1) for nd in dims)
        self.norm_inf = self._norm_inf()

    def _faces(self, d):
        """Face diffusivities km, kp along dimension d and the masks of inner neighbours."""
        ax = 2 - d
        k = self.kappa
        km = k.copy()
        kp = k.copy()
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        kp[tuple(lo)] = 0.5 * (k[tuple(lo)] + k[tuple(hi)])      # i and i + e_d
        km[tuple(hi)] = 0.5 * (k[tuple(hi)] + k[tuple(lo)])      # i and i - e_d
        has_p = np.zeros(self.shape, dtype=bool)
        has_m = np.zeros(self.shape, dtype=bool)
        has_p[tuple(lo)] = True
        has_m[tuple(hi)] = True
        return km, kp, has_m, has_p, tuple(lo), tuple(hi)

    def apply(self, x: np.ndarray) -> np.ndarray:
        X = np.asarray(x, dtype=np.float64).reshape(self.shape)
        Y = np.zeros(self.shape)
        for d in range(self.ndim):
            km, kp, _, _, lo, hi = self._faces(d)
            xp = np.zeros(self.shape)
            xm = np.zeros(self.shape)
            xp[lo] = X[hi]                          # x_{i+e_d}, 0 outside the grid
            xm[hi] = X[lo]                          # x_{i-e_d}
            Y += self.s * (kp * (xp - X) - km * (X - xm))
            if self.vel[d] is not None:
                Y -= self.c * self.vel[d] * (xp - xm)
        return Y.reshape(-1)

    def _norm_inf(self) -> float:
        rows = np.zeros(self.shape)
        for d in range(self.ndim):
            km, kp, has_m, has_p, _, _ = self._faces(d)
            v = self.vel[d] if self.vel[d] is not None else 0.0
            rows += self.s * (kp + km)
            rows += np.where(has_p, np.abs(self.s * kp - self.c * v), 0.0)
            rows += np.where(has_m, np.abs(self.s * km + self.c * v), 0.0)
        return float(rows.max())
