"""Independent LASSO solvers for tiny instances, used only to pin the IPM oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``soft_threshold``: with no missing samples M_perp = A is orthogonal, so
  1/2 ||b - A beta||^2 = 1/2 ||A^T b - beta||^2 (Sec. 3, A real orthogonal) and
  Eq. (realopt) separates into scalar problems solved by soft-thresholding.
* ``enumerate_active_sets``: for every sign pattern sigma in {-1, 0, +1}^n
  solve the restricted normal equations N_A^T N_A beta_A = N_A^T b - lambda sigma_A
  and keep the pattern whose solution has those signs and satisfies the
  subgradient bound |N_i^T (b - N beta)| <= lambda on the zero set (the KKT
  conditions of Eq. (realopt)).  Exact for tiny n, independent of the IPM.
* ``proximal_gradient``: ISTA on the dense matrix with step 1 (||M_perp|| <= 1).
"""

import itertools

import numpy as np


def soft_threshold(c, lam):
    return np.sign(c) * np.maximum(np.abs(c) - lam, 0.0)


def enumerate_active_sets(N, b, lam, tol=1e-10):
    """Exact LASSO minimiser of 1/2||b - N beta||^2 + lam ||beta||_1 for tiny n."""
    m, n = N.shape
    NtN, Ntb = N.T @ N, N.T @ b
    found = []
    for sigma in itertools.product((-1, 0, 1), repeat=n):
        sigma = np.asarray(sigma, dtype=np.float64)
        act = np.flatnonzero(sigma)
        beta = np.zeros(n)
        if act.size:
            sub = NtN[np.ix_(act, act)]
            if np.linalg.matrix_rank(sub) < act.size:
                continue
            beta[act] = np.linalg.solve(sub, Ntb[act] - lam * sigma[act])
            if np.any(sigma[act] * beta[act] <= 0):
                continue
        grad = Ntb - NtN @ beta                    # N^T (b - N beta)
        zero = np.flatnonzero(sigma == 0)
        if np.all(np.abs(grad[zero]) <= lam * (1 + tol)):
            found.append(beta)
    return found


def proximal_gradient(N, b, lam, iters=200000, tol=1e-15):
    """ISTA with unit step on 1/2||b - N beta||^2 + lam ||beta||_1."""
    beta = np.zeros(N.shape[1])
    for _ in range(iters):
        new = soft_threshold(beta + N.T @ (b - N @ beta), lam)
        if np.max(np.abs(new - beta)) <= tol:
            return new
        beta = new
    return beta
