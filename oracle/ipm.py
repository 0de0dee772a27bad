"""Primal-dual interior-point method with PCG on the condensed KKT system.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation follows the paper: variables (beta, z, s1, s2, y1, y2, nu1, nu2) of the
slack QP Eq. (slackproblem); at every iterate we keep y = nu (the KKT rows
y_i - nu_i = 0 of Eq. (kkt) are linear, so a Newton step keeps them).

Paper passages followed, in the order the method applies them
-------------------------------------------------------------
* Sec. 3.3, duality measure mu = (nu1^T s1 + nu2^T s2) / 2n.
* Sec. 3.3, barrier system Eq. (kktmu): S_i V_i e = mu e replaces the
  complementarity rows; we target sigma * mu (path following).
* Sec. 3.4, Eq. (defsigma): Sigma_i = S_i^{-1} V_i.
* Sec. 3.4, Eq. (condensedkkt): K = [[G + Lambda1, Lambda2], [Lambda2, Lambda1]],
  Lambda1 = Sigma1 + Sigma2, Lambda2 = Sigma1 - Sigma2, G = M_perp^T M_perp.
* Sec. 3.5: P = [[I + Lambda1, Lambda2], [Lambda2, Lambda1]], Eq. (defBD),
  Prop. exprbd (D = Sigma1 + Sigma2 + 4 Sigma1 Sigma2) and Eq. (invprecond1):
  P^{-1} = [[Lambda1 D^{-1}, -Lambda2 D^{-1}], [-D^{-1} Lambda2, B^{-1}]],
  B^{-1} = D^{-1} (I + Lambda1).
* Sec. 3.5 / Sec. 5: conjugate gradients on K with preconditioner P.
* Sec. 3.5 (the comparison with Fountoulakis et al.): their preconditioner
  multiplies the identity by a scalar rho = n/m set by the fraction of observed
  data, P_rho = [[rho I + Lambda1, Lambda2], [Lambda2, Lambda1]]; then
  D_rho = Lambda1 (rho I + Lambda1) - Lambda2^2 = rho (Sigma1 + Sigma2) + 4 Sigma1 Sigma2
  and P_rho^{-1} = [[Lambda1, -Lambda2], [-Lambda2, rho I + Lambda1]] D_rho^{-1}
  (``precond_rho``; rho = 1 is the paper's P).

Our readings (the paper leaves them to MadNLP or prints them with typos)
----------------------------------------------------------------------
* Right-hand side.  The Newton system is derived from minus the residual
  F(w) of Eq. (kktmu) with y = nu:
      r_d  = G beta - c - nu1 + nu2        (c = M_perp^T b; row 1 of Eq. (kkt))
      r_z  = lambda e - nu1 - nu2          (row 2)
      r_p1 = z + beta - s1,  r_p2 = z - beta - s2     (rows 5, 6)
      r_c1 = s1 nu1 - sigma mu,  r_c2 = s2 nu2 - sigma mu
  Eliminating ds and dnu gives K [dbeta; dz] = [rho_b; rho_c] with
      rho_b = -r_d - r_c1/s1 - Sigma1 r_p1 + r_c2/s2 + Sigma2 r_p2
      rho_c = -r_z - r_c1/s1 - Sigma1 r_p1 - r_c2/s2 - Sigma2 r_p2
  and back-substitution ds1 = dz + dbeta + r_p1, ds2 = dz - dbeta + r_p2,
  dnu_i = -r_ci/s_i - Sigma_i ds_i.  The matrix is exactly the paper's K;
  the paper's printed r_1 and r_6 carry sign typos, which we do not follow.
* Start: beta = 0, z = zeta e with zeta = max(1, ||c||_inf), s1 = s2 = z,
  nu1 = nu2 = lambda/2 e (feasible in every linear row except row 1).
* Step: one common step alpha = min(1, tau * alpha_max) for all variables,
  alpha_max the largest step keeping (s, nu) >= 0; tau = 0.995.  sigma = 0.1,
  raised to 0.5 for the next iteration after a step alpha < 0.1.
* Optional adaptive centring (``sigma_rule="adaptive"``), in the direction of the
  single-step predictor-corrector the paper suggests (Sec. 5): Mehrotra's
  centring heuristic sigma = (mu_aff / mu)^3 needs the affine-scaling predictor,
  a second Newton system per iteration; here the previous step stands in for it,
  sigma = clamp((1 - alpha)^3, sigma_min, sigma_slow) for the next direction
  (the first direction uses sigma0), and each iteration solves one system.
  After a PCG solve that stopped at max_cg (an inexact direction) the fixed rule
  applies instead: with the aggressive centring, mu then ran to 0 while the gap
  stalled.
* Single-step predictor-corrector (``sigma_rule="single"``), the adaptation of
  Mehrotra's method to one Krylov solve per iteration that Sec. 5 proposes (its form
  is ours).  Mehrotra's method solves two systems with the same K per iteration:
  the affine-scaling predictor (sigma = 0), then the corrector whose complementarity
  rows target sigma mu e - ds_aff o dnu_aff with sigma = (mu_aff / mu)^3.  Here the
  predictor costs no Krylov solve: it is P^{-1} rhs_aff with the closed-form P^{-1}
  of Eq. (invprecond1).  P differs from K by [G - I, 0; 0, 0] = -[M^T M, 0; 0, 0]
  (M the rows of missing samples), so the estimate is exact on the complement of
  the span of the missing samples and wholly exact when none is missing (the
  asymptotic spectrum result Prop. limitprecond is the same statement for P^{-1} K).
  alpha_aff = min(1, largest step keeping (s, nu) >= 0 along the predictor),
  mu_aff = (s + alpha_aff ds)^T (nu + alpha_aff dnu) / 2n, sigma = (mu_aff / mu)^3
  clamped to [sigma_min, sigma_max], and the one Krylov solve is the corrector's.
  ``sigma_rule="mehrotra"`` is the two-solve method (exact predictor), kept for
  comparison.  After a PCG solve that stopped at max_cg the next direction takes
  the fixed rule and no second-order term.
* Stop when the relative duality gap (``Problem.certificate``) is <= gap_tol.
* PCG: x0 = 0, stop when sqrt(r^T z) <= cg_tol * sqrt(r0^T z0) (relative,
  the default) or sqrt(r^T z) <= cg_tol (absolute, as the paper's 1e-12 rule),
  or after max_cg iterations.  ``krylov="cr"`` uses preconditioned conjugate
  residuals and ``krylov="car"`` the conjugate A-residual method instead (Sec. 3.5
  lists CR and CAr beside CG), with the same stop rule.
"""

import numpy as np


# ---- the barrier diagonals and the preconditioner (Sec. 3.4-3.5) -------------------

def sigmas(s1, nu1, s2, nu2):
    """Sigma_1 = S_1^{-1} V_1 and Sigma_2 = S_2^{-1} V_2 (Eq. (defsigma))."""
    return nu1 / s1, nu2 / s2


def K_apply(G, Sig1, Sig2, p_beta, p_z):
    """[G + Lambda1, Lambda2; Lambda2, Lambda1] [p_beta; p_z] (Eq. (condensedkkt))."""
    L1, L2 = Sig1 + Sig2, Sig1 - Sig2
    return G(p_beta) + L1 * p_beta + L2 * p_z, L2 * p_beta + L1 * p_z


def P_apply(Sig1, Sig2, p_beta, p_z, rho=1.0):
    """P [p_beta; p_z] with P = [rho I + Lambda1, Lambda2; Lambda2, Lambda1] (rho = 1: the paper's P)."""
    L1, L2 = Sig1 + Sig2, Sig1 - Sig2
    return rho * p_beta + L1 * p_beta + L2 * p_z, L2 * p_beta + L1 * p_z


def Pinv_apply(Sig1, Sig2, r_beta, r_z, rho=1.0):
    """P^{-1} [r_beta; r_z] by the closed form Eq. (invprecond1) with Prop. exprbd
    (D = Sigma1 + Sigma2 + 4 Sigma1 Sigma2; for P_rho, D = rho (Sigma1 + Sigma2) + 4 Sigma1 Sigma2)."""
    L1, L2 = Sig1 + Sig2, Sig1 - Sig2
    D = rho * (Sig1 + Sig2) + 4.0 * Sig1 * Sig2
    Binv = (rho + L1) / D
    return (L1 / D) * r_beta - (L2 / D) * r_z, -(L2 / D) * r_beta + Binv * r_z


# ---- preconditioned conjugate gradients (Sec. 3.5) --------------------------------

def pcg(apply_K, apply_Pinv, rhs, tol, max_iter, relative=True):
    """Solve K x = rhs; vectors are pairs (beta-part, z-part).

    Returns (x, iterations, final sqrt(r^T z)).
    """
    def dot(a, b):
        return a[0] @ b[0] + a[1] @ b[1]

    x = (np.zeros_like(rhs[0]), np.zeros_like(rhs[1]))
    r = (rhs[0].copy(), rhs[1].copy())
    zv = apply_Pinv(*r)
    p = (zv[0].copy(), zv[1].copy())
    rho = dot(r, zv)
    stop = tol * np.sqrt(max(rho, 0.0)) if relative else tol
    it = 0
    while it < max_iter and np.sqrt(max(rho, 0.0)) > stop:
        q = apply_K(*p)
        alpha = rho / dot(p, q)
        x = (x[0] + alpha * p[0], x[1] + alpha * p[1])
        r = (r[0] - alpha * q[0], r[1] - alpha * q[1])
        zv = apply_Pinv(*r)
        rho_new = dot(r, zv)
        p = (zv[0] + (rho_new / rho) * p[0], zv[1] + (rho_new / rho) * p[1])
        rho = rho_new
        it += 1
    return x, it, np.sqrt(max(rho, 0.0))


def pcr(apply_K, apply_Pinv, rhs, tol, max_iter, relative=True):
    """Preconditioned conjugate residuals (the CR the paper lists beside CG for these
    SPD systems, Sec. 3.5): one product K z per iteration, the residual minimised in
    the P^{-1} norm; same stop rule as ``pcg``.  Returns (x, iterations, sqrt(r^T z))."""
    def dot(a, b):
        return a[0] @ b[0] + a[1] @ b[1]

    x = (np.zeros_like(rhs[0]), np.zeros_like(rhs[1]))
    r = (rhs[0].copy(), rhs[1].copy())
    z = apply_Pinv(*r)
    rho = dot(r, z)
    stop = tol * np.sqrt(max(rho, 0.0)) if relative else tol
    p = q = None
    zw_old = 0.0
    it = 0
    while it < max_iter and np.sqrt(max(rho, 0.0)) > stop:
        w = apply_K(*z)                                     # K z
        zw = dot(z, w)
        beta = zw / zw_old if p is not None else 0.0
        p = z if p is None else (z[0] + beta * p[0], z[1] + beta * p[1])
        q = w if q is None else (w[0] + beta * q[0], w[1] + beta * q[1])   # q = K p
        u = apply_Pinv(*q)
        alpha = zw / dot(q, u)
        x = (x[0] + alpha * p[0], x[1] + alpha * p[1])
        r = (r[0] - alpha * q[0], r[1] - alpha * q[1])
        z = (z[0] - alpha * u[0], z[1] - alpha * u[1])
        rho = dot(r, z)
        zw_old = zw
        it += 1
    return x, it, np.sqrt(max(rho, 0.0))


def pcar(apply_K, apply_Pinv, rhs, tol, max_iter, relative=True):
    """Preconditioned conjugate A-residuals (CAr, named in Sec. 3.5 beside CG and CR for
    these SPD systems; Montoison, Orban and Saunders 2023).  With M = P^{-1} = L L^T and
    the split system L^T K L, CG minimises the K-norm of the error, CR the norm of
    the residual, and CAr the norm of (L^T K L) times the residual, i.e.
    w^T M w with w = K M r, over the same Krylov space.  It is CG in the inner product
    of the cube of the split operator.  Written on the unsplit vectors:
        z = M r, w = K z, y = M w       (w, y kept by recurrence after the start)
        v = K y                          (the one product per iteration)
        rho = y^T v, beta = rho / rho_prev,
        p = z + beta p, Q = w + beta Q (= K p), U = v + beta U (= K M K p),
        alpha = rho / (U^T M U),
        x += alpha p, r -= alpha Q, w -= alpha U, y -= alpha M U, z = M r.
    Starting costs one more product (w = K z).  Same stop rule as ``pcg``.
    In floating point the recurred w and y drift from K M r once rho has fallen
    by the unit round-off against the rho of the cycle's start (rho weighs the
    residual by the cube of the operator), and r^T z then stalls above the stop
    threshold: the method restarts there (w = K z, y = M w from the current
    residual, beta = 0; one more product), as it does when rho or U^T M U is not
    positive.  Returns (x, iterations, sqrt(r^T z))."""
    def dot(a, b):
        return a[0] @ b[0] + a[1] @ b[1]

    def axpy(a, x, y):
        return (y[0] + a * x[0], y[1] + a * x[1])

    x = (np.zeros_like(rhs[0]), np.zeros_like(rhs[1]))
    r = (rhs[0].copy(), rhs[1].copy())
    z = apply_Pinv(*r)
    rho_rz = dot(r, z)
    stop = tol * np.sqrt(max(rho_rz, 0.0)) if relative else tol
    eps = np.finfo(np.float64).eps
    w = y = p = Q = U = None
    rho_prev = rho_start = 0.0
    it = 0
    while it < max_iter and np.sqrt(max(rho_rz, 0.0)) > stop:
        if w is None:                                   # (re)start: w and y from r
            w = apply_K(*z)
            y = apply_Pinv(*w)
            p = None
        v = apply_K(*y)
        rho = dot(y, v)
        if p is None:
            rho_start = rho
            p, Q, U = z, w, v
        else:
            if not (rho > eps * rho_start):
                w = None                                # recurrences exhausted: restart
                continue
            beta = rho / rho_prev
            p, Q, U = axpy(beta, p, z), axpy(beta, Q, w), axpy(beta, U, v)
        MU = apply_Pinv(*U)
        um = dot(U, MU)
        if not (rho > 0.0 and um > 0.0):
            break                                       # breakdown right after a (re)start
        alpha = rho / um
        x = axpy(alpha, p, x)
        r = axpy(-alpha, Q, r)
        w = axpy(-alpha, U, w)
        y = axpy(-alpha, MU, y)
        z = apply_Pinv(*r)
        rho_rz = dot(r, z)
        rho_prev = rho
        it += 1
    return x, it, np.sqrt(max(rho_rz, 0.0))


# ---- Newton system ------------------------------------------------------------------

def residuals(prob, Gbeta, w, sigma):
    """r_d, r_z, r_p1, r_p2, r_c1, r_c2 and mu at w = (beta, z, s1, s2, nu1, nu2)."""
    beta, z, s1, s2, nu1, nu2 = w
    mu = (nu1 @ s1 + nu2 @ s2) / (2 * prob.n)
    r_d = Gbeta - prob.c - nu1 + nu2
    r_z = prob.lam - nu1 - nu2
    r_p1 = z + beta - s1
    r_p2 = z - beta - s2
    r_c1 = s1 * nu1 - sigma * mu
    r_c2 = s2 * nu2 - sigma * mu
    return (r_d, r_z, r_p1, r_p2, r_c1, r_c2), mu


def condensed_rhs(res, w):
    """[rho_b; rho_c] of the condensed system (module docstring)."""
    r_d, r_z, r_p1, r_p2, r_c1, r_c2 = res
    _, _, s1, s2, nu1, nu2 = w
    Sig1, Sig2 = sigmas(s1, nu1, s2, nu2)
    rho_b = -r_d - r_c1 / s1 - Sig1 * r_p1 + r_c2 / s2 + Sig2 * r_p2
    rho_c = -r_z - r_c1 / s1 - Sig1 * r_p1 - r_c2 / s2 - Sig2 * r_p2
    return rho_b, rho_c


def back_substitute(res, w, dbeta, dz):
    """ds1, ds2, dnu1, dnu2 from the eliminated rows."""
    _, _, r_p1, r_p2, r_c1, r_c2 = res
    _, _, s1, s2, nu1, nu2 = w
    Sig1, Sig2 = sigmas(s1, nu1, s2, nu2)
    ds1 = dz + dbeta + r_p1
    ds2 = dz - dbeta + r_p2
    dnu1 = -r_c1 / s1 - Sig1 * ds1
    dnu2 = -r_c2 / s2 - Sig2 * ds2
    return ds1, ds2, dnu1, dnu2


def max_step(vals, dirs):
    """Largest alpha in (0, inf] with vals + alpha * dirs >= 0 (inf if none binds)."""
    amax = np.inf
    for v, d in zip(vals, dirs):
        neg = d < 0
        if np.any(neg):
            amax = min(amax, float(np.min(-v[neg] / d[neg])))
    return amax


def starting_point(prob):
    """beta = 0, z = s1 = s2 = zeta e, nu1 = nu2 = lambda/2 e."""
    n = prob.n
    zeta = max(1.0, float(np.abs(prob.c).max()))
    beta = np.zeros(n)
    z = np.full(n, zeta)
    nu = np.full(n, 0.5 * prob.lam)
    return [beta, z, z.copy(), z.copy(), nu, nu.copy()]


def affine_predictor(prob, w, res_aff, Sig1, Sig2, solve_K=None, rho=1.0):
    """Affine-scaling predictor of Mehrotra's method: the Newton direction for sigma = 0.
    With solve_K (a Krylov solve of K d = rhs) it is the exact direction; without it,
    P^{-1} rhs (Sec. 3.5): P differs from K only by [G - I, 0; 0, 0], minus the projector
    onto the missing samples, so the estimate is exact on the complement of that subspace
    (and wholly exact without missing samples).  Returns (dbeta, dz, ds1, ds2, dnu1, dnu2,
    Krylov iterations)."""
    rhs = condensed_rhs(res_aff, w)
    if solve_K is not None:
        (db, dz), its = solve_K(rhs)
    else:
        db, dz = Pinv_apply(Sig1, Sig2, rhs[0], rhs[1], rho)
        its = 0
    return (db, dz) + back_substitute(res_aff, w, db, dz) + (its,)


def predictor_corrector(prob, w, Gbeta, Sig1, Sig2, sigma_min, sigma_max, solve_K=None, rho=1.0):
    """Mehrotra's centring and second-order correction from an affine predictor.

    alpha_aff = min(1, largest step keeping (s, nu) >= 0 along the predictor),
    mu_aff = ((s + alpha_aff ds)^T (nu + alpha_aff dnu)) / 2n, sigma = (mu_aff / mu)^3
    clamped to [sigma_min, sigma_max], and the complementarity rows of the corrector
    system target sigma mu e - ds_aff o dnu_aff:
        r_ci = s_i o nu_i - sigma mu e + ds_i,aff o dnu_i,aff.
    Returns (residuals of the corrector system, sigma, predictor's Krylov iterations)."""
    res_aff, mu = residuals(prob, Gbeta, w, 0.0)
    _, _, ds1, ds2, dn1, dn2, its = affine_predictor(prob, w, res_aff, Sig1, Sig2, solve_K, rho)
    s1, s2, nu1, nu2 = w[2], w[3], w[4], w[5]
    a_aff = min(1.0, max_step((s1, s2, nu1, nu2), (ds1, ds2, dn1, dn2)))
    mu_aff = ((s1 + a_aff * ds1) @ (nu1 + a_aff * dn1) + (s2 + a_aff * ds2) @ (nu2 + a_aff * dn2)) / (2 * prob.n)
    sigma = min(sigma_max, max(sigma_min, (mu_aff / mu) ** 3))
    (r_d, r_z, r_p1, r_p2, r_c1, r_c2), _ = residuals(prob, Gbeta, w, sigma)
    return (r_d, r_z, r_p1, r_p2, r_c1 + ds1 * dn1, r_c2 + ds2 * dn2), sigma, its


def next_sigma(alpha, rule, sigma0, sigma_slow, sigma_min):
    """Centring parameter for the next direction after a step of length alpha."""
    if rule == "adaptive":
        return min(sigma_slow, max(sigma_min, (1.0 - alpha) ** 3))
    return sigma_slow if alpha < 0.1 else sigma0


def solve(prob, gap_tol=1e-6, cg_tol=1e-10, max_ipm=200, max_cg=500, cg_relative=True,
          sigma0=0.1, sigma_slow=0.5, tau=0.995, w0=None, log=None, sigma_rule="fixed", sigma_min=None,
          precond_rho=1.0, krylov="cg", sigma_max=1.0):
    """Run the IPM; returns a dict with the point, counts and the certificate.

    sigma_min (the lower clamp of the adaptive and predictor-corrector rules) defaults to
    the value the library documents for the rule: 0.03 for "adaptive", 0.01 for
    "single" and "mehrotra"."""
    if sigma_min is None:
        sigma_min = 0.03 if sigma_rule == "adaptive" else 0.01
    w = [np.array(v, dtype=np.float64, copy=True) for v in (w0 or starting_point(prob))]
    sigma = sigma0
    cg_counts, pred_counts, sigmas_used = [], [], []
    after_cap = False
    status = "maxiter"
    for it in range(max_ipm + 1):
        beta = w[0]
        Gbeta = prob.G(beta)
        P, D, gap = prob.certificate(beta)
        if log is not None:
            log.append(dict(it=it, primal=P, dual=D, gap=gap))
        if gap <= gap_tol:
            status = "converged"
            break
        if it == max_ipm:
            break
        Sig1, Sig2 = sigmas(w[2], w[4], w[3], w[5])
        solver = {"cg": pcg, "cr": pcr, "car": pcar}[krylov]
        apply_K = lambda a, b: K_apply(prob.G, Sig1, Sig2, a, b)
        apply_Pinv = lambda a, b: Pinv_apply(Sig1, Sig2, a, b, precond_rho)
        n_pred = 0
        if sigma_rule in ("mehrotra", "single") and not after_cap:
            exact = None
            if sigma_rule == "mehrotra":
                def exact(rhs):
                    x, k, _ = solver(apply_K, apply_Pinv, rhs, cg_tol, max_cg, cg_relative)
                    return x, k
            res, sigma, n_pred = predictor_corrector(prob, w, Gbeta, Sig1, Sig2, sigma_min, sigma_max, exact,
                                                     precond_rho)
        else:
            res, mu = residuals(prob, Gbeta, w, sigma)
        rhs = condensed_rhs(res, w)
        (dbeta, dz), ncg, _ = solver(apply_K, apply_Pinv, rhs, cg_tol, max_cg, cg_relative)
        cg_counts.append(ncg)
        pred_counts.append(n_pred)
        sigmas_used.append(sigma)
        ds1, ds2, dnu1, dnu2 = back_substitute(res, w, dbeta, dz)
        amax = max_step(w[2:], (ds1, ds2, dnu1, dnu2))
        alpha = min(1.0, tau * amax)
        for v, d in zip(w, (dbeta, dz, ds1, ds2, dnu1, dnu2)):
            v += alpha * d
        after_cap = ncg >= max_cg
        rule = "fixed" if (after_cap or sigma_rule not in ("fixed", "adaptive")) else sigma_rule
        sigma = next_sigma(alpha, rule, sigma0, sigma_slow, sigma_min)
    P, D, gap = prob.certificate(w[0])
    return dict(status=status, point=w, beta=w[0], primal=P, dual=D, gap=gap,
                ipm_iters=len(cg_counts), cg_counts=cg_counts, predictor_counts=pred_counts, sigmas=sigmas_used)
