"""Pins for the oracle's whole IPM solve (no GPU).

References: the soft-thresholding closed form of the unmasked problem, the
lambda >= lambda_max zero solution, exhaustive active-set enumeration and
proximal gradient on tiny masked instances, the KKT conditions of
Eq. (realopt), a hand-derived worked example, and the asymptotic spectrum of
P^{-1} K (Prop. limitprecond / boundskappa).
"""

import os

import numpy as np
import pytest

from oracle import brute, ipm
from oracle.lasso import Problem
from paper_2502_04217_gb300.synth import make_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense(op, n):
    return np.stack([np.ravel(op(e)) for e in np.eye(n)], axis=1)


def _masked(dims, seed, missing=0.25, lam_rel=0.1):
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    mask = np.ones(n, bool)
    mask[rng.choice(n, size=max(1, int(round(missing * n))), replace=False)] = False
    prob = Problem(dims, mask.reshape(dims), rng.standard_normal(dims), 1.0)
    prob.lam = lam_rel * prob.lambda_max()
    return prob


def test_golden_unmasked_n2():
    vals = {}
    with open(os.path.join(GOLDEN, "lasso_n2_unmasked.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                vals[k] = np.array([float(x) for x in v])
    prob = Problem((2,), np.ones(2, bool), vals["Y"], vals["LAMBDA"][0])
    res = ipm.solve(prob, gap_tol=1e-13)
    assert np.abs(res["beta"] - vals["BETA_STAR"]).max() < 1e-10
    assert abs(res["primal"] - vals["OBJECTIVE"][0]) < 1e-11


@pytest.mark.parametrize("dims", [(16,), (8, 6), (4, 4, 4), (256,), (15,), (5, 6), (3, 4, 5)])
def test_unmasked_equals_soft_threshold(dims):
    rng = np.random.default_rng(12)
    prob = Problem(dims, np.ones(dims, bool), rng.standard_normal(dims), 1.0)
    prob.lam = 0.3 * prob.lambda_max()
    res = ipm.solve(prob, gap_tol=1e-12)
    assert res["status"] == "converged"
    ref = brute.soft_threshold(prob.c, prob.lam)
    assert np.abs(res["beta"] - ref).max() < 1e-8


@pytest.mark.parametrize("dims", [(8,), (4, 4), (2, 2, 4)])
def test_lambda_above_lambda_max_gives_zero(dims):
    prob = _masked(dims, 13)
    prob.lam = 1.01 * prob.lambda_max()
    res = ipm.solve(prob, gap_tol=1e-12)
    assert np.abs(res["beta"]).max() < 1e-8


@pytest.mark.parametrize("dims,seed", [((8,), 14), ((8,), 16), ((10,), 16), ((2, 4), 14), ((4, 2), 15),
                                       ((2, 2, 2), 15), ((7,), 14), ((3, 3), 15), ((2, 3), 16)])
def test_masked_tiny_against_enumeration(dims, seed):
    prob = _masked(dims, seed, missing=0.25, lam_rel=0.3)
    Mp = _dense(prob.A, prob.n)[prob.mask.reshape(-1)]
    sols = brute.enumerate_active_sets(Mp, prob.b, prob.lam)
    assert len(sols) >= 1
    # unique minimiser (N_A has full column rank): every valid pattern gives the same point
    for s in sols[1:]:
        assert np.abs(s - sols[0]).max() < 1e-9
    res = ipm.solve(prob, gap_tol=1e-13)
    assert res["status"] == "converged"
    assert np.abs(res["beta"] - sols[0]).max() < 1e-7
    assert abs(res["primal"] - prob.objective(sols[0])) < 1e-10 * max(1, abs(res["primal"]))


@pytest.mark.parametrize("dims,seed", [((32,), 19), ((8, 8), 20), ((4, 4, 4), 21), ((6, 10), 22),
                                       ((27,), 19), ((5, 7), 20), ((3, 5, 4), 21)])
def test_masked_small_against_proximal_gradient(dims, seed):
    prob = _masked(dims, seed, missing=0.2, lam_rel=0.2)
    Mp = _dense(prob.A, prob.n)[prob.mask.reshape(-1)]
    ref = brute.proximal_gradient(Mp, prob.b, prob.lam)
    res = ipm.solve(prob, gap_tol=1e-13)
    assert res["status"] == "converged"
    assert np.abs(res["beta"] - ref).max() < 1e-6
    assert abs(res["primal"] - prob.objective(ref)) < 1e-9 * max(1, abs(res["primal"]))


def test_kkt_conditions_at_solution():
    prob = _masked((8, 8), 23, missing=0.2, lam_rel=0.1)
    res = ipm.solve(prob, gap_tol=1e-13)
    beta = res["beta"]
    g = prob.c - prob.G(beta)               # M_perp^T (b - M_perp beta)
    act = np.abs(beta) > 1e-7
    assert act.any()
    assert np.abs(g[act] - prob.lam * np.sign(beta[act])).max() < 1e-6
    assert np.abs(g[~act]).max() <= prob.lam * (1 + 1e-6)
    # slack-form KKT rows (Eq. (kkt)) hold at the returned point
    b, z, s1, s2, nu1, nu2 = res["point"]
    assert np.abs(z + b - s1).max() < 1e-8 and np.abs(z - b - s2).max() < 1e-8
    assert np.abs(prob.lam - nu1 - nu2).max() < 1e-8
    assert np.all(s1 > 0) and np.all(s2 > 0) and np.all(nu1 > 0) and np.all(nu2 > 0)


def test_asymptotic_spectrum_of_preconditioned_K():
    """Prop. limitprecond / boundskappa: as mu -> 0 the spectrum of P^{-1}K tends to
    {1} union spec(Q*), Q* = G restricted to the support of beta*; eigenvalue 1
    has multiplicity 2n - l."""
    prob = _masked((16,), 24, missing=0.25, lam_rel=0.3)
    res = ipm.solve(prob, gap_tol=1e-13)
    b, z, s1, s2, nu1, nu2 = res["point"]
    n = prob.n
    S1, S2 = ipm.sigmas(s1, nu1, s2, nu2)
    M = _dense(lambda e: np.concatenate(ipm.Pinv_apply(S1, S2, *ipm.K_apply(prob.G, S1, S2, e[:n], e[n:]))), 2 * n)
    ev = np.sort(np.linalg.eigvals(M).real)
    act = np.flatnonzero(np.abs(b) > 1e-6)
    ell = act.size
    G = _dense(prob.G, n)
    q = np.sort(np.linalg.eigvalsh(G[np.ix_(act, act)]))
    ref = np.sort(np.concatenate([np.ones(2 * n - ell), q]))
    assert 0 < ell < n
    # asymptotic statement: the match is O(sqrt(mu)) and the dense product of
    # Lambda ~ 1/mu entries loses digits, so a loose tolerance still pins the structure
    assert np.abs(ev - ref).max() < 1e-2
    assert np.sum(np.abs(ev - 1) < 1e-2) >= 2 * n - ell


def test_config_1d_workload_converges():
    w = make_problem("1d")
    prob = Problem(w.dims, w.mask.astype(bool), w.y, 1.0)
    prob.lam = w.lam_rel * prob.lambda_max()
    res = ipm.solve(prob, gap_tol=1e-10)
    assert res["status"] == "converged" and res["gap"] <= 1e-10
    # planted frequencies clearly above the threshold are recovered
    from oracle.mapping import frequency_classes
    _, rep, _ = frequency_classes(w.dims)
    pos = {int(k): i for i, k in enumerate(rep)}
    nsc, nrep = 2, rep.size
    strong = 0
    for f, a in zip(w.freqs, w.amps):
        if np.sqrt(2) * max(abs(a.real), abs(a.imag)) > 3 * prob.lam:
            i = pos[int(f)]
            assert abs(res["beta"][nsc + i]) + abs(res["beta"][nsc + nrep + i]) > prob.lam
            strong += 1
    assert strong >= 4


@pytest.mark.parametrize("dims", [(16,), (4, 4, 4)])
def test_adaptive_centring_unmasked_equals_soft_threshold(dims):
    """The adaptive centring rule changes the path, not the solution."""
    rng = np.random.default_rng(31)
    prob = Problem(dims, np.ones(dims, bool), rng.standard_normal(dims), 1.0)
    prob.lam = 0.3 * prob.lambda_max()
    res = ipm.solve(prob, gap_tol=1e-12, sigma_rule="adaptive")
    assert res["status"] == "converged"
    assert np.abs(res["beta"] - brute.soft_threshold(prob.c, prob.lam)).max() < 1e-8


@pytest.mark.parametrize("dims,seed", [((32,), 19), ((8, 8), 20), ((4, 4, 4), 21)])
def test_adaptive_centring_masked_against_proximal_gradient(dims, seed):
    prob = _masked(dims, seed, missing=0.2, lam_rel=0.2)
    Mp = _dense(prob.A, prob.n)[prob.mask.reshape(-1)]
    ref = brute.proximal_gradient(Mp, prob.b, prob.lam)
    # at gaps far below 1e-10 the aggressive centring (sigma down to 0.01) drives
    # PCG into breakdown on such tiny problems; the rule is for practical tolerances
    res = ipm.solve(prob, gap_tol=1e-10, sigma_rule="adaptive")
    assert res["status"] == "converged"
    assert np.abs(res["beta"] - ref).max() < 1e-5
    assert abs(res["primal"] - prob.objective(ref)) < 2e-9 * max(1, abs(res["primal"]))


def test_adaptive_centring_rule():
    """sigma = clamp((1 - alpha)^3, sigma_min, sigma_slow); the fixed rule switches at alpha = 0.1."""
    assert ipm.next_sigma(0.0, "adaptive", 0.1, 0.5, 0.01) == 0.5
    assert ipm.next_sigma(1.0, "adaptive", 0.1, 0.5, 0.01) == 0.01
    assert abs(ipm.next_sigma(0.5, "adaptive", 0.1, 0.5, 0.01) - 0.125) < 1e-15
    assert abs(ipm.next_sigma(0.9, "adaptive", 0.1, 0.5, 0.01) - 0.01) < 1e-15      # 0.001 clamped
    assert ipm.next_sigma(0.05, "fixed", 0.1, 0.5, 0.01) == 0.5
    assert ipm.next_sigma(0.5, "fixed", 0.1, 0.5, 0.01) == 0.1


def test_scaled_identity_preconditioner_same_solution():
    """The preconditioner changes the PCG path only: P_rho with rho = n/m reaches the
    same optimum as the paper's P."""
    prob = _masked((8, 8), 20, missing=0.2, lam_rel=0.2)
    m = int(prob.mask.sum())
    a = ipm.solve(prob, gap_tol=1e-12)
    b = ipm.solve(prob, gap_tol=1e-12, precond_rho=prob.n / m)
    assert b["status"] == "converged"
    assert np.abs(a["beta"] - b["beta"]).max() < 1e-7


def test_conjugate_residual_ipm_same_solution():
    prob = _masked((8, 8), 20, missing=0.2, lam_rel=0.2)
    a = ipm.solve(prob, gap_tol=1e-12)
    b = ipm.solve(prob, gap_tol=1e-12, krylov="cr")
    assert b["status"] == "converged"
    assert np.abs(a["beta"] - b["beta"]).max() < 1e-7


def test_conjugate_a_residual_ipm_same_solution():
    prob = _masked((8, 8), 20, missing=0.2, lam_rel=0.2)
    a = ipm.solve(prob, gap_tol=1e-12)
    b = ipm.solve(prob, gap_tol=1e-12, krylov="car")
    assert b["status"] == "converged"
    assert np.abs(a["beta"] - b["beta"]).max() < 1e-7


@pytest.mark.parametrize("dims", [(16,), (4, 4, 4), (9, 5)])
def test_predictor_corrector_unmasked_equals_soft_threshold(dims):
    """The single-step predictor-corrector (and the two-solve Mehrotra method) change
    the path, not the solution."""
    rng = np.random.default_rng(33)
    prob = Problem(dims, np.ones(dims, bool), rng.standard_normal(dims), 1.0)
    prob.lam = 0.3 * prob.lambda_max()
    for rule in ("single", "mehrotra"):
        res = ipm.solve(prob, gap_tol=1e-12, sigma_rule=rule, sigma_min=0.01)
        assert res["status"] == "converged"
        assert np.abs(res["beta"] - brute.soft_threshold(prob.c, prob.lam)).max() < 1e-8


@pytest.mark.parametrize("dims,seed", [((8,), 14), ((10,), 16), ((2, 4), 14), ((2, 2, 2), 15), ((7,), 14),
                                       ((3, 3), 15)])
def test_predictor_corrector_masked_tiny_against_enumeration(dims, seed):
    prob = _masked(dims, seed, missing=0.25, lam_rel=0.3)
    Mp = _dense(prob.A, prob.n)[prob.mask.reshape(-1)]
    sols = brute.enumerate_active_sets(Mp, prob.b, prob.lam)
    res = ipm.solve(prob, gap_tol=1e-12, sigma_rule="single", sigma_min=0.01)
    assert res["status"] == "converged"
    assert np.abs(res["beta"] - sols[0]).max() < 1e-7


@pytest.mark.parametrize("dims,seed", [((32,), 19), ((8, 8), 20), ((4, 4, 4), 21)])
def test_predictor_corrector_masked_against_proximal_gradient(dims, seed):
    prob = _masked(dims, seed, missing=0.2, lam_rel=0.2)
    Mp = _dense(prob.A, prob.n)[prob.mask.reshape(-1)]
    ref = brute.proximal_gradient(Mp, prob.b, prob.lam)
    res = ipm.solve(prob, gap_tol=1e-10, sigma_rule="single", sigma_min=0.01)
    assert res["status"] == "converged"
    assert np.abs(res["beta"] - ref).max() < 1e-5
    assert abs(res["primal"] - prob.objective(ref)) < 2e-9 * max(1, abs(res["primal"]))
    # one Krylov solve per iteration and no predictor solves; fewer iterations than the
    # adaptive rule on these problems
    assert sum(res["predictor_counts"]) == 0
    ad = ipm.solve(prob, gap_tol=1e-10, sigma_rule="adaptive")
    assert res["ipm_iters"] <= ad["ipm_iters"]
