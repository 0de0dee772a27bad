"""Pins for the oracle's masked operators, KKT algebra and Newton step (no GPU).

The references are dense matrices and numpy.linalg routines on tiny grids, the
identities the paper proves (Prop. exprbd, Eq. (invprecond1), Eq. (precond1)),
and a finite-difference Jacobian of the barrier system Eq. (kktmu), which pins
the residuals, the condensed right-hand side and the back-substitution.
"""

import numpy as np
import pytest

from oracle import ipm
from oracle.lasso import Problem

SMALL = [(8,), (12,), (4, 6), (4, 4, 4), (2, 4, 6), (9,), (3, 5), (3, 4, 5)]


def _problem(dims, seed=0, missing=0.3, lam=0.1):
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    mask = np.ones(n, bool)
    mask[rng.choice(n, size=max(1, int(missing * n)), replace=False)] = False
    return Problem(dims, mask.reshape(dims), rng.standard_normal(dims), lam)


def _dense(op, n):
    return np.stack([np.ravel(op(e)) for e in np.eye(n)], axis=1)


def _interior_point(n, rng):
    s1, s2 = rng.uniform(0.1, 2.0, n), rng.uniform(0.1, 2.0, n)
    nu1, nu2 = rng.uniform(0.1, 2.0, n), rng.uniform(0.1, 2.0, n)
    return s1, nu1, s2, nu2


@pytest.mark.parametrize("dims", SMALL)
def test_masked_operators_against_dense_rows(dims):
    prob = _problem(dims)
    n = prob.n
    A = _dense(prob.A, n)
    Mp = A[prob.mask.reshape(-1)]                     # M_perp = A_{observed rows}, Eq. (MMperp)
    rng = np.random.default_rng(5)
    beta = rng.standard_normal(n)
    b = rng.standard_normal(Mp.shape[0])
    assert np.abs(prob.Mperp(beta) - Mp @ beta).max() < 1e-13
    assert np.abs(prob.MperpT(b) - Mp.T @ b).max() < 1e-13
    assert np.abs(prob.c - Mp.T @ prob.b).max() < 1e-13   # Eq. (xi): M_perp^T b = A^T b_hat


@pytest.mark.parametrize("dims", SMALL)
def test_G_is_orthogonal_projector(dims):
    prob = _problem(dims)
    G = _dense(prob.G, prob.n)
    assert np.abs(G - G.T).max() < 1e-13
    assert np.abs(G @ G - G).max() < 1e-13
    assert abs(np.trace(G) - prob.mask.sum()) < 1e-10


def test_objective_and_certificate_against_dense():
    prob = _problem((4, 6), lam=0.3)
    Mp = _dense(prob.A, prob.n)[prob.mask.reshape(-1)]
    beta = np.random.default_rng(6).standard_normal(prob.n)
    r = prob.b - Mp @ beta
    assert abs(prob.objective(beta) - (0.5 * r @ r + 0.3 * np.abs(beta).sum())) < 1e-12
    P, D, gap = prob.certificate(beta)
    assert abs(P - prob.objective(beta)) < 1e-12 and gap >= 0
    # the scaled dual point is feasible: ||M_perp^T theta_s||_inf <= lambda
    corr = np.abs(Mp.T @ r).max()
    ts = r * min(1.0, 0.3 / corr)
    assert np.abs(Mp.T @ ts).max() <= 0.3 * (1 + 1e-12)
    assert abs(D - (prob.b @ ts - 0.5 * ts @ ts)) < 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_preconditioner_closed_form(seed):
    rng = np.random.default_rng(seed)
    n = 7
    s1, nu1, s2, nu2 = _interior_point(n, rng)
    S1, S2 = ipm.sigmas(s1, nu1, s2, nu2)
    L1, L2 = S1 + S2, S1 - S2
    P = np.block([[np.diag(1 + L1), np.diag(L2)], [np.diag(L2), np.diag(L1)]])
    Pinv = _dense(lambda e: np.concatenate(ipm.Pinv_apply(S1, S2, e[:n], e[n:])), 2 * n)
    assert np.abs(Pinv - np.linalg.inv(P)).max() < 1e-12 * np.abs(np.linalg.inv(P)).max()
    Pd = _dense(lambda e: np.concatenate(ipm.P_apply(S1, S2, e[:n], e[n:])), 2 * n)
    assert np.abs(Pd - P).max() < 1e-14
    # Prop. exprbd: D = Lambda1 (I + Lambda1) - Lambda2^2 = Sigma1 + Sigma2 + 4 Sigma1 Sigma2 > 0
    D = L1 * (1 + L1) - L2 ** 2
    assert np.abs(D - (S1 + S2 + 4 * S1 * S2)).max() < 1e-12 * D.max()
    # Eq. (11block): Lambda1 D^{-1} lies in (0, 1)
    assert np.all((L1 / D > 0) & (L1 / D < 1))


@pytest.mark.parametrize("dims", [(8,), (4, 6), (2, 2, 4)])
def test_K_structure_and_preconditioned_blocks(dims):
    prob = _problem(dims)
    n = prob.n
    rng = np.random.default_rng(7)
    s1, nu1, s2, nu2 = _interior_point(n, rng)
    S1, S2 = ipm.sigmas(s1, nu1, s2, nu2)
    L1, L2 = S1 + S2, S1 - S2
    D = S1 + S2 + 4 * S1 * S2
    G = _dense(prob.G, n)
    K = _dense(lambda e: np.concatenate(ipm.K_apply(prob.G, S1, S2, e[:n], e[n:])), 2 * n)
    P = _dense(lambda e: np.concatenate(ipm.P_apply(S1, S2, e[:n], e[n:])), 2 * n)
    I = np.eye(n)
    # K = P + [[G - I, 0], [0, 0]]  (Eq. (condensedkkt) against the definition of P)
    E = np.zeros((2 * n, 2 * n))
    E[:n, :n] = G - I
    assert np.abs(K - (P + E)).max() < 1e-12 * np.abs(K).max()
    # Eq. (precond1): blocks of P^{-1} K
    PiK = _dense(lambda e: np.concatenate(ipm.Pinv_apply(S1, S2, *np.split(K @ e, 2))), 2 * n)
    assert np.abs(PiK[:n, n:]).max() < 1e-12
    assert np.abs(PiK[n:, n:] - I).max() < 1e-12
    assert np.abs(PiK[:n, :n] - (I + np.diag(L1 / D) @ (G - I))).max() < 1e-12
    assert np.abs(PiK[n:, :n] - (-np.diag(L2 / D) @ (G - I))).max() < 1e-12


def _F(prob, w, sigma, mu_fixed):
    """Barrier residual of Eq. (kktmu) with y = nu and target sigma*mu held fixed."""
    beta, z, s1, s2, nu1, nu2 = np.split(w, 6)
    Mp = prob._Mp
    return np.concatenate([
        Mp.T @ (Mp @ beta - prob.b) - nu1 + nu2,
        prob.lam - nu1 - nu2,
        z + beta - s1,
        z - beta - s2,
        s1 * nu1 - sigma * mu_fixed,
        s2 * nu2 - sigma * mu_fixed,
    ])


@pytest.mark.parametrize("dims", [(8,), (4, 4), (2, 2, 4)])
def test_condensed_newton_step_equals_full_newton_step(dims):
    prob = _problem(dims, lam=0.2)
    n = prob.n
    prob._Mp = _dense(prob.A, n)[prob.mask.reshape(-1)]
    rng = np.random.default_rng(8)
    beta = rng.standard_normal(n) * 0.3
    z = np.abs(beta) + rng.uniform(0.2, 1.0, n)
    s1 = z + beta + rng.uniform(-0.05, 0.05, n)       # deliberately infeasible rows 5, 6
    s2 = z - beta + rng.uniform(-0.05, 0.05, n)
    nu1, nu2 = rng.uniform(0.05, 0.2, n), rng.uniform(0.05, 0.2, n)
    w = [beta, z, s1, s2, nu1, nu2]
    sigma = 0.1
    mu = (nu1 @ s1 + nu2 @ s2) / (2 * n)
    # Jacobian by central differences (exact for this linear + bilinear map)
    W = np.concatenate(w)
    h = 1e-3
    J = np.stack([(_F(prob, W + h * e, sigma, mu) - _F(prob, W - h * e, sigma, mu)) / (2 * h)
                  for e in np.eye(6 * n)], axis=1)
    dW = np.linalg.solve(J, -_F(prob, W, sigma, mu))
    # the oracle's condensed path
    res, mu2 = ipm.residuals(prob, prob.G(beta), w, sigma)
    assert abs(mu2 - mu) < 1e-15
    S1, S2 = ipm.sigmas(s1, nu1, s2, nu2)
    rhs = ipm.condensed_rhs(res, w)
    (db, dz), it, _ = ipm.pcg(lambda a, b: ipm.K_apply(prob.G, S1, S2, a, b),
                              lambda a, b: ipm.Pinv_apply(S1, S2, a, b), rhs, 1e-14, 500)
    ds1, ds2, dnu1, dnu2 = ipm.back_substitute(res, w, db, dz)
    mine = np.concatenate([db, dz, ds1, ds2, dnu1, dnu2])
    assert np.abs(mine - dW).max() < 1e-8 * max(1.0, np.abs(dW).max())


def test_pcg_one_iteration_without_mask():
    """No missing samples: G = I, so P^{-1} K = I (Sec. 3.5) and PCG stops after one step."""
    dims = (4, 6)
    prob = Problem(dims, np.ones(dims, bool), np.random.default_rng(9).standard_normal(dims), 0.1)
    n = prob.n
    rng = np.random.default_rng(10)
    s1, nu1, s2, nu2 = _interior_point(n, rng)
    S1, S2 = ipm.sigmas(s1, nu1, s2, nu2)
    rhs = (rng.standard_normal(n), rng.standard_normal(n))
    x, it, _ = ipm.pcg(lambda a, b: ipm.K_apply(prob.G, S1, S2, a, b),
                       lambda a, b: ipm.Pinv_apply(S1, S2, a, b), rhs, 1e-12, 50)
    assert it == 1
    Kx = np.concatenate(ipm.K_apply(prob.G, S1, S2, *x))
    assert np.abs(Kx - np.concatenate(rhs)).max() < 1e-12


def test_pcg_solves_masked_system():
    prob = _problem((6, 4), missing=0.4)
    n = prob.n
    rng = np.random.default_rng(11)
    s1, nu1, s2, nu2 = _interior_point(n, rng)
    S1, S2 = ipm.sigmas(s1, nu1, s2, nu2)
    K = _dense(lambda e: np.concatenate(ipm.K_apply(prob.G, S1, S2, e[:n], e[n:])), 2 * n)
    rhs = rng.standard_normal(2 * n)
    x, it, _ = ipm.pcg(lambda a, b: ipm.K_apply(prob.G, S1, S2, a, b),
                       lambda a, b: ipm.Pinv_apply(S1, S2, a, b), tuple(np.split(rhs, 2)), 1e-13, 500)
    assert np.abs(np.concatenate(x) - np.linalg.solve(K, rhs)).max() < 1e-10


@pytest.mark.parametrize("rho", [0.5, 1.25, 4.0])
def test_scaled_identity_preconditioner_closed_form(rho):
    """P_rho = [rho I + Lambda1, Lambda2; Lambda2, Lambda1] (the scaled identity the paper
    compares with, Sec. 3.5): closed-form inverse against a dense inverse, and
    D_rho = Lambda1 (rho + Lambda1) - Lambda2^2 = rho (Sigma1 + Sigma2) + 4 Sigma1 Sigma2."""
    rng = np.random.default_rng(40)
    n = 7
    s1, nu1, s2, nu2 = _interior_point(n, rng)
    S1, S2 = ipm.sigmas(s1, nu1, s2, nu2)
    L1, L2 = S1 + S2, S1 - S2
    P = np.block([[np.diag(rho + L1), np.diag(L2)], [np.diag(L2), np.diag(L1)]])
    Pd = _dense(lambda e: np.concatenate(ipm.P_apply(S1, S2, e[:n], e[n:], rho)), 2 * n)
    assert np.abs(Pd - P).max() < 1e-14 * np.abs(P).max()
    Pinv = _dense(lambda e: np.concatenate(ipm.Pinv_apply(S1, S2, e[:n], e[n:], rho)), 2 * n)
    assert np.abs(Pinv - np.linalg.inv(P)).max() < 1e-12 * np.abs(np.linalg.inv(P)).max()
    D = L1 * (rho + L1) - L2 ** 2
    assert np.abs(D - (rho * (S1 + S2) + 4 * S1 * S2)).max() < 1e-12 * D.max()


@pytest.mark.parametrize("dims", [(8,), (4, 6)])
def test_preconditioned_conjugate_residuals_solve_the_newton_system(dims):
    """CR (Sec. 3.5 lists it beside CG): the condensed system K x = rhs solved by PCR equals
    the dense solve, and PCR reaches it in no more iterations than the system's size."""
    prob = _problem(dims)
    n = prob.n
    rng = np.random.default_rng(41)
    s1, nu1, s2, nu2 = _interior_point(n, rng)
    S1, S2 = ipm.sigmas(s1, nu1, s2, nu2)
    K = _dense(lambda e: np.concatenate(ipm.K_apply(prob.G, S1, S2, e[:n], e[n:])), 2 * n)
    rhs = rng.standard_normal(2 * n)
    (xb, xz), it, res = ipm.pcr(lambda a, b: ipm.K_apply(prob.G, S1, S2, a, b),
                                lambda a, b: ipm.Pinv_apply(S1, S2, a, b), tuple(np.split(rhs, 2)), 1e-13, 500)
    ref = np.linalg.solve(K, rhs)
    assert np.abs(np.concatenate([xb, xz]) - ref).max() < 1e-9 * np.abs(ref).max()
    assert it <= 2 * n + 2


@pytest.mark.parametrize("dims", [(8,), (4, 6), (9,)])
def test_conjugate_a_residuals_solve_the_newton_system(dims):
    """CAr (Sec. 3.5 names it beside CG and CR): the condensed system solved by PCAR
    equals the dense solve."""
    prob = _problem(dims)
    n = prob.n
    rng = np.random.default_rng(43)
    s1, nu1, s2, nu2 = _interior_point(n, rng)
    S1, S2 = ipm.sigmas(s1, nu1, s2, nu2)
    K = _dense(lambda e: np.concatenate(ipm.K_apply(prob.G, S1, S2, e[:n], e[n:])), 2 * n)
    rhs = rng.standard_normal(2 * n)
    (xb, xz), it, res = ipm.pcar(lambda a, b: ipm.K_apply(prob.G, S1, S2, a, b),
                                 lambda a, b: ipm.Pinv_apply(S1, S2, a, b), tuple(np.split(rhs, 2)), 1e-13, 500)
    ref = np.linalg.solve(K, rhs)
    assert np.abs(np.concatenate([xb, xz]) - ref).max() < 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_krylov_iterates_minimise_their_norms(k):
    """After k iterations from x0 = 0 each method's iterate is the minimiser, over the
    Krylov space span{M r0, (MK) M r0, ..., (MK)^{k-1} M r0} (M = P^{-1}), of its own
    norm, found here by dense least squares on an orthonormal basis:
    CG the K-norm of the error, CR r^T M r, CAr (K M r)^T M (K M r)."""
    prob = _problem((4, 6))
    n = prob.n
    rng = np.random.default_rng(47)
    s1, nu1, s2, nu2 = _interior_point(n, rng)
    S1, S2 = ipm.sigmas(s1, nu1, s2, nu2)
    K = _dense(lambda e: np.concatenate(ipm.K_apply(prob.G, S1, S2, e[:n], e[n:])), 2 * n)
    M = _dense(lambda e: np.concatenate(ipm.Pinv_apply(S1, S2, e[:n], e[n:])), 2 * n)
    M = (M + M.T) / 2
    Lc = np.linalg.cholesky(M)                     # M = Lc Lc^T
    b = rng.standard_normal(2 * n)
    V = [M @ b]
    for _ in range(k - 1):
        V.append(M @ (K @ V[-1]))
    Qb, _ = np.linalg.qr(np.stack(V, axis=1))
    xs = np.linalg.solve(K, b)
    Kh = np.linalg.cholesky(K)                     # K = Kh Kh^T
    # each norm is || W (b - K Qb c) || for a fixed W; minimise over c
    W = {"cg": Kh.T @ np.linalg.inv(K),            # ||e||_K = ||Kh^T K^{-1} r||
         "cr": Lc.T,                               # r^T M r
         "car": Lc.T @ K @ M}                      # (K M r)^T M (K M r)
    split = lambda v: tuple(np.split(v, 2))
    Kop = lambda a, c: ipm.K_apply(prob.G, S1, S2, a, c)
    Mop = lambda a, c: ipm.Pinv_apply(S1, S2, a, c)
    for name, fn in (("cg", ipm.pcg), ("cr", ipm.pcr), ("car", ipm.pcar)):
        A = W[name] @ K @ Qb
        c, *_ = np.linalg.lstsq(A, W[name] @ b, rcond=None)
        x_ref = Qb @ c
        (xb, xz), it, _ = fn(Kop, Mop, split(b), 0.0, k)
        assert it == k
        x = np.concatenate([xb, xz])
        assert np.abs(x - x_ref).max() < 1e-8 * np.abs(xs).max(), name


def _pc_point(n, rng):
    beta = rng.standard_normal(n) * 0.3
    z = np.abs(beta) + rng.uniform(0.2, 1.0, n)
    s1 = z + beta + rng.uniform(-0.05, 0.05, n)       # infeasible rows 5, 6 as well
    s2 = z - beta + rng.uniform(-0.05, 0.05, n)
    nu1, nu2 = rng.uniform(0.05, 0.2, n), rng.uniform(0.05, 0.2, n)
    return [beta, z, s1, s2, nu1, nu2]


def _full_newton_rows(prob, w, d, r_c):
    """The six linearised rows of Eq. (kktmu) at w for the direction d, with the
    complementarity residuals r_c = (r_c1, r_c2) given: returns each row's value."""
    beta, z, s1, s2, nu1, nu2 = w
    db, dz, ds1, ds2, dn1, dn2 = d
    r_d = prob.G(beta) - prob.c - nu1 + nu2
    return [prob.G(db) - dn1 + dn2 + r_d,                  # row 1: G dbeta - dnu1 + dnu2 = -r_d
            -dn1 - dn2 + (prob.lam - nu1 - nu2),           # row 2
            dz + db - ds1 + (z + beta - s1),               # row 5
            dz - db - ds2 + (z - beta - s2),               # row 6
            s1 * dn1 + nu1 * ds1 + r_c[0],                 # complementarity 1
            s2 * dn2 + nu2 * ds2 + r_c[1]]                 # complementarity 2


@pytest.mark.parametrize("dims", [(8,), (4, 4), (2, 2, 4), (9,)])
def test_affine_predictor_without_missing_samples_is_the_newton_direction(dims):
    """No missing samples: G = I, so P = K and the predictor P^{-1} rhs_aff is the exact
    affine-scaling direction: it satisfies all six linearised rows of Eq. (kktmu) with
    sigma = 0 (r_c = s o nu)."""
    prob = _problem(dims, missing=0.0, lam=0.2)
    prob.mask[:] = True
    prob.b_hat = np.asarray(prob.b_hat)
    rng = np.random.default_rng(11)
    w = _pc_point(prob.n, rng)
    S1, S2 = ipm.sigmas(w[2], w[4], w[3], w[5])
    res_aff, mu = ipm.residuals(prob, prob.G(w[0]), w, 0.0)
    d = ipm.affine_predictor(prob, w, res_aff, S1, S2)[:6]
    for row in _full_newton_rows(prob, w, d, (w[2] * w[4], w[3] * w[5])):
        assert np.abs(row).max() < 1e-12


@pytest.mark.parametrize("dims", [(8,), (4, 4), (2, 2, 4), (3, 5)])
def test_predictor_corrector_direction_solves_the_second_order_system(dims):
    """The single-step predictor-corrector's direction (the PCG solve of the corrector
    system, solved here to 1e-14) satisfies the linearised rows of Eq. (kktmu) with the
    complementarity target sigma mu e - ds_aff o dnu_aff:
        S dnu + V ds = -(s o nu - sigma mu e + ds_aff o dnu_aff),
    the predictor being P^{-1} rhs_aff (masked problem: an estimate); and sigma is
    (mu_aff / mu)^3 with alpha_aff the largest step along the predictor keeping s, nu >= 0,
    found here by bisection on positivity."""
    prob = _problem(dims, lam=0.2)
    rng = np.random.default_rng(12)
    w = _pc_point(prob.n, rng)
    S1, S2 = ipm.sigmas(w[2], w[4], w[3], w[5])
    Gb = prob.G(w[0])
    res, sigma, its = ipm.predictor_corrector(prob, w, Gb, S1, S2, 0.0, 1.0)
    assert its == 0
    # the predictor, independently
    res_aff, mu = ipm.residuals(prob, Gb, w, 0.0)
    rhs_aff = ipm.condensed_rhs(res_aff, w)
    Pd = _dense(lambda v: np.concatenate(ipm.P_apply(S1, S2, v[:prob.n], v[prob.n:])), 2 * prob.n)
    daff = np.linalg.solve(Pd, np.concatenate(rhs_aff))
    ds1, ds2, dn1, dn2 = ipm.back_substitute(res_aff, w, daff[:prob.n], daff[prob.n:])
    lo, hi = 0.0, 1.0
    pos = lambda a: all(np.all(v + a * dv >= 0) for v, dv in zip(w[2:], (ds1, ds2, dn1, dn2)))
    if not pos(1.0):
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if pos(mid) else (lo, mid)
    a = 1.0 if pos(1.0) else lo
    mu_aff = ((w[2] + a * ds1) @ (w[4] + a * dn1) + (w[3] + a * ds2) @ (w[5] + a * dn2)) / (2 * prob.n)
    assert abs(sigma - min(1.0, (mu_aff / mu) ** 3)) < 1e-9 * max(sigma, 1e-12) + 1e-15
    # the corrector's residuals and direction
    r_c1 = w[2] * w[4] - sigma * mu + ds1 * dn1
    r_c2 = w[3] * w[5] - sigma * mu + ds2 * dn2
    assert np.abs(res[4] - r_c1).max() < 1e-13 and np.abs(res[5] - r_c2).max() < 1e-13
    rhs = ipm.condensed_rhs(res, w)
    (db, dz), it, _ = ipm.pcg(lambda u, v: ipm.K_apply(prob.G, S1, S2, u, v),
                              lambda u, v: ipm.Pinv_apply(S1, S2, u, v), rhs, 1e-14, 500)
    d = (db, dz) + ipm.back_substitute(res, w, db, dz)
    for row in _full_newton_rows(prob, w, d, (r_c1, r_c2)):
        assert np.abs(row).max() < 1e-9
