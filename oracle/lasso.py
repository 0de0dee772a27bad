"""Masked operators, the LASSO objective and its duality-gap certificate.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed
-----------------------
* Sec. 3, Eq. (MMperp): M = A_M (rows of missing samples) and
  M_perp = A_{[n] minus M} (rows of observed samples).
* Sec. 3, Eq. (realopt): beta* = argmin 1/2 ||b - M_perp beta||^2 + lambda ||beta||_1.
* Sec. 3.1: M_perp beta = (IDFT(v))_{observed} with v = B^H beta, and
  M_perp^T b = A^T b_hat = B DFT(b_hat) with b_hat the zero-filled signal (Eq. (xi)).

The duality-gap certificate is not in the paper (it stops on a primal-dual
residual).  Our reading: the standard LASSO dual
    max_theta  b^T theta - 1/2 ||theta||^2   s.t.  ||M_perp^T theta||_inf <= lambda,
evaluated at the residual theta = b - M_perp beta scaled into the feasible set,
theta_s = theta * min(1, lambda / ||M_perp^T theta||_inf).  Weak duality makes
P(beta) - D(theta_s) >= P(beta) - P(beta*) >= 0, so it certifies suboptimality.
The reported gap is (P - D) / max(1, |P|).
"""

import numpy as np

from .dft import dft, idft
from .mapping import beta_to_v, v_to_beta


class Problem:
    """One masked, noisy real signal on a d-dimensional grid (any extents >= 2).

    mask[j] = True where sample j is observed (the complement of the paper's
    missing set M); y holds the signal, its values at missing samples are
    ignored (the zero-filled b_hat of Sec. 3.1 is built here).
    """

    def __init__(self, dims, mask, y, lam):
        self.dims = tuple(int(d) for d in dims)
        self.n = int(np.prod(self.dims))
        self.mask = np.asarray(mask, dtype=bool).reshape(self.dims)
        self.b_hat = np.where(self.mask, np.asarray(y, dtype=np.float64).reshape(self.dims), 0.0)
        self.b = self.b_hat[self.mask]
        self.c = self.At(self.b_hat)           # M_perp^T b, computed once
        self.lam = float(lam)

    # ---- A and its transpose (Sec. 3, Eq. (map); A real orthogonal) -------------
    def A(self, beta):
        """A beta = IDFT(B^H beta), a real grid (its imaginary part is rounding)."""
        return idft(beta_to_v(beta, self.dims)).real

    def At(self, x):
        """A^T x = B DFT(x) for a real grid x."""
        return v_to_beta(dft(x), self.dims)

    # ---- masked operators (Sec. 3.1) ----------------------------------------
    def Mperp(self, beta):
        return self.A(beta)[self.mask]

    def MperpT(self, b):
        b_hat = np.zeros(self.dims)
        b_hat[self.mask] = b
        return self.At(b_hat)

    def G(self, beta):
        """M_perp^T M_perp beta = A^T diag(mask) A beta."""
        return self.At(np.where(self.mask, self.A(beta), 0.0))

    # ---- objective and certificate -------------------------------------------
    def objective(self, beta):
        """1/2 ||b - M_perp beta||^2 + lambda ||beta||_1 (Eq. (realopt))."""
        r = self.b - self.Mperp(beta)
        return 0.5 * r @ r + self.lam * np.abs(beta).sum()

    def lambda_max(self):
        """||M_perp^T b||_inf: for lambda >= this value beta* = 0."""
        return float(np.abs(self.c).max())

    def certificate(self, beta):
        """(primal P, dual D, relative gap) at beta; see the module docstring."""
        theta = self.b - self.Mperp(beta)
        P = 0.5 * theta @ theta + self.lam * np.abs(beta).sum()
        corr = np.abs(self.MperpT(theta)).max()
        scale = 1.0 if corr <= self.lam else self.lam / corr
        ts = scale * theta
        D = self.b @ ts - 0.5 * ts @ ts
        return P, D, (P - D) / max(1.0, abs(P))
