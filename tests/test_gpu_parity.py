"""CUDA path against the CPU oracle, element by element (needs a GB300).

Tolerances (derived from the arithmetic).  Products with G = M_perp^T M_perp are
held to the norm-wise and element-wise FFT error bounds of ``bounds.py``
(c u (log2 n + 2) with c = 12, Higham's bound for two transforms; u the unit
round-off of the products' precision).  The diagonal terms of K and P^{-1} are
FP64 in every mode: Sigma = nu / s is formed with a Newton reciprocal (relative
error below 1.4e-14), so those terms are compared to 1e-13 relative to
(Sigma1 + Sigma2)(|p_beta| + |p_z|) per element.  Vectors are compared on the
canonical half spectrum, whose norm is at most that of beta (the bounds are
therefore conservative by at most sqrt 2).

Solves: lambda is the oracle's (lambda_rel ||M_perp^T b||_inf computed by the
oracle) and is passed to the library as an absolute value, so no input of the
oracle comes from the GPU.
"""

import numpy as np
import pytest
import torch

from oracle import ipm as oipm
from oracle.lasso import Problem
from paper_2502_04217_gb300 import binding
from paper_2502_04217_gb300.synth import make_problem

from bounds import assert_g_close, fft_bound
from layout import ghost_mask, half_to_beta, lib_to_half, oracle_to_half, oracle_to_lib, to_device

pytestmark = pytest.mark.gpu

SIZES = [(8,), (12,), (96,), (256,), (512,),
         (8, 6), (16, 12), (48, 64), (64, 48), (96, 32), (512, 16),
         (4, 6, 8), (8, 8, 8), (16, 12, 8), (12, 16, 24), (32, 24, 16), (128, 256, 16), (16, 128, 256)]


def _workload(dims, seed=0, missing=0.15):
    w = make_problem("custom", dims=dims, missing=missing, seed=seed)
    return w


def _handle(w, precision=binding.IPM_FP64, lam_rel=0.1, prob=None, **opt):
    """A handle on workload w; with prob, lambda is the oracle's (absolute)."""
    if prob is not None:
        o = binding.default_options(precision=precision, lambda_relative=0, **opt)
        lam = prob.lam
    else:
        o = binding.default_options(precision=precision, lambda_relative=1, **opt)
        lam = lam_rel
    return binding.ipm_create(w.dims, np.ascontiguousarray(w.mask), np.ascontiguousarray(w.y), lam, o)


def _oracle(w, lam):
    return Problem(w.dims, w.mask.astype(bool), w.y, lam)


def _oracle_rel(w, lam_rel):
    """The oracle's problem with lambda = lam_rel * its own lambda_max."""
    prob = _oracle(w, 1.0)
    prob.lam = lam_rel * prob.lambda_max()
    return prob


def _check_kkt(h, prob, dims, precision, S1, S2, pb, pz, qk):
    """q = K p from the library against the oracle: G part by assert_g_close with the FP64
    diagonal terms' allowance, z block (FP64 only) to 1e-13 per element."""
    H2 = qk.numel() // 2
    qb, qz = oipm.K_apply(prob.G, S1, S2, pb, pz)
    gref = oracle_to_half(prob.G(pb), dims)
    dsz = oracle_to_half((S1 + S2) * (np.abs(pb) + np.abs(pz)), dims)
    got_b = lib_to_half(h, qk[:H2])
    ref_b = oracle_to_half(qb, dims)
    b = fft_bound(dims, precision)
    err = np.abs(got_b - ref_b)
    assert np.linalg.norm(err) <= b * np.linalg.norm(pb) + 1e-13 * np.linalg.norm(dsz), \
        ("K beta block norm-wise", np.linalg.norm(err) / np.linalg.norm(pb), b)
    elem = b * np.abs(gref).max() + 1e-13 * np.abs(dsz)
    assert np.all(err <= elem), ("K beta block element-wise", float((err / elem).max()))
    errz = np.abs(lib_to_half(h, qk[H2:]) - oracle_to_half(qz, dims))
    assert np.all(errz <= 1e-13 * np.abs(dsz) + 1e-300), ("K z block", float(errz.max()))
    return H2


def _interior(n, rng):
    return (rng.uniform(0.05, 3.0, n), rng.uniform(0.05, 3.0, n), rng.uniform(0.05, 3.0, n),
            rng.uniform(0.05, 3.0, n))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    binding.load()


@pytest.mark.parametrize("dims", SIZES)
def test_pack_unpack_roundtrip(dims):
    w = _workload(dims)
    h = _handle(w)
    try:
        n = int(np.prod(dims))
        beta = np.random.default_rng(1).standard_normal(n)
        lib = oracle_to_lib(h, beta, dims)
        assert np.abs(lib_to_half(h, lib) - oracle_to_half(beta, dims)).max() < 1e-15 * 8
        assert np.count_nonzero(~ghost_mask(h, dims)) == n       # exactly n LASSO coordinates
    finally:
        binding.ipm_destroy(h)


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
@pytest.mark.parametrize("dims", SIZES)
def test_gapply_matches_oracle(dims, precision):
    w = _workload(dims, seed=2)
    h = _handle(w, precision)
    try:
        n = int(np.prod(dims))
        prob = _oracle(w, 1.0)
        beta = np.random.default_rng(3).standard_normal(n)
        p = oracle_to_lib(h, beta, dims)
        q = torch.empty_like(p)
        binding.gapply(h, p, q)
        assert_g_close(lib_to_half(h, q), oracle_to_half(prob.G(beta), dims), beta, dims, precision)
        assert np.all(q.cpu().numpy()[ghost_mask(h, dims)] == 0.0)
    finally:
        binding.ipm_destroy(h)


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
@pytest.mark.parametrize("dims", [(256,), (48, 64), (16, 12, 8), (32, 24, 16)])
def test_kkt_and_precond_match_oracle(dims, precision):
    w = _workload(dims, seed=4)
    h = _handle(w, precision)
    try:
        n = int(np.prod(dims))
        prob = _oracle(w, 1.0)
        rng = np.random.default_rng(5)
        s1, nu1, s2, nu2 = _interior(n, rng)
        binding.ipm_set_sigma(h, *[oracle_to_lib(h, v, dims) for v in (s1, nu1, s2, nu2)])
        S1, S2 = oipm.sigmas(s1, nu1, s2, nu2)
        pb, pz = rng.standard_normal(n), rng.standard_normal(n)
        p = torch.cat([oracle_to_lib(h, pb, dims), oracle_to_lib(h, pz, dims)])
        q = torch.empty_like(p)
        binding.kkt_apply(h, p, q)
        H2 = _check_kkt(h, prob, dims, precision, S1, S2, pb, pz, q)
        # preconditioner: always FP64
        z = torch.empty_like(p)
        binding.precond_apply(h, p, z)
        zb, zz = oipm.Pinv_apply(S1, S2, pb, pz)
        zs = np.abs(np.concatenate([zb, zz])).max()
        assert np.abs(lib_to_half(h, z[:H2]) - oracle_to_half(zb, dims)).max() < 1e-14 * max(1, zs)
        assert np.abs(lib_to_half(h, z[H2:]) - oracle_to_half(zz, dims)).max() < 1e-14 * max(1, zs)
        # Eq. (precond1): P^{-1} K [0; u] = [0; u]
        u = torch.cat([torch.zeros_like(p[:H2]), oracle_to_lib(h, rng.standard_normal(n), dims)])
        Ku = torch.empty_like(u)
        binding.kkt_apply(h, u, Ku)
        PKu = torch.empty_like(u)
        binding.precond_apply(h, Ku, PKu)
        assert torch.abs(PKu - u).max().item() < 1e-10 * (1 + (S1 + S2).max())
    finally:
        binding.ipm_destroy(h)


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
@pytest.mark.parametrize("dims", [(256,), (48, 64), (16, 12, 8), (32, 24, 16)])
def test_kkt_diagonal_terms_over_wide_ranges(dims, precision):
    """The K epilogue's FP64 diagonal terms beside an FP64 or FP32 G part, with Sigma spread
    over 1e-8 .. 1e8 and p over 1e-6 .. 1e6 with random signs: every element within the
    1e-13 relative allowance of the diagonal terms against the oracle's FP64 K, the G part
    within its FFT bound."""
    w = _workload(dims, seed=12)
    n = int(np.prod(dims))
    prob = _oracle(w, 1.0)
    rng = np.random.default_rng(13)
    s1, s2 = 10.0 ** rng.uniform(-4, 4, n), 10.0 ** rng.uniform(-4, 4, n)
    nu1, nu2 = 10.0 ** rng.uniform(-4, 4, n), 10.0 ** rng.uniform(-4, 4, n)
    S1, S2 = oipm.sigmas(s1, nu1, s2, nu2)
    pb = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-6, 6, n)
    pz = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-6, 6, n)
    h = _handle(w, precision)
    try:
        binding.ipm_set_sigma(h, *[oracle_to_lib(h, v, dims) for v in (s1, nu1, s2, nu2)])
        p = torch.cat([oracle_to_lib(h, pb, dims), oracle_to_lib(h, pz, dims)])
        q = torch.full_like(p, float("nan"))
        binding.kkt_apply(h, p, q)
        _check_kkt(h, prob, dims, precision, S1, S2, pb, pz, q)
    finally:
        binding.ipm_destroy(h)


# Operand staging of the last pass (tile_kstage 1: per-slot loads, 2: L2 bulk prefetch,
# 3: bulk copies into shared memory on an mbarrier) only changes where the epilogue reads
# its operands: products and solves are bit-identical.  Forced tiles make every handle
# launch the same shapes; (48, 64) has 33 rows of 48 and (15, 16, 10) 90 rows of 16, so a
# tile of 4 rows leaves a ragged last tile; (32, 24, 16) runs its tuned tile.
KSTAGE_CASES = [((48, 64), {"tile_e": 8, "tile_p": 4}), ((15, 16, 10), {"tile_e": 8, "tile_p": 4}),
                ((32, 24, 16), {})]


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
@pytest.mark.parametrize("dims,tile", KSTAGE_CASES)
def test_staged_k_operands_give_identical_products(dims, tile, precision):
    w = _workload(dims, seed=6)
    n = int(np.prod(dims))
    prob = _oracle(w, 1.0)
    rng = np.random.default_rng(7)
    s1, nu1, s2, nu2 = _interior(n, rng)
    S1, S2 = oipm.sigmas(s1, nu1, s2, nu2)
    pb, pz = rng.standard_normal(n), rng.standard_normal(n)
    qs = []
    for ks in (1, 2, 3):
        h = _handle(w, precision, tile_kstage=ks, **tile)
        try:
            desc = binding.ipm_describe(h)
            pre = "fp32_" if precision == binding.IPM_MIXED else "fp64_"
            for name in ("row", "row_k"):       # the PCG product's last pass and kkt_apply's
                assert desc[pre + name]["kstage"] == ks - 1, (name, desc[pre + name])
            binding.ipm_set_sigma(h, *[oracle_to_lib(h, v, dims) for v in (s1, nu1, s2, nu2)])
            p = torch.cat([oracle_to_lib(h, pb, dims), oracle_to_lib(h, pz, dims)])
            q = torch.full_like(p, float("nan"))
            binding.kkt_apply(h, p, q)
            if ks == 3:
                _check_kkt(h, prob, dims, precision, S1, S2, pb, pz, q)
            qs.append(q)
        finally:
            binding.ipm_destroy(h)
    assert torch.equal(qs[0], qs[1]) and torch.equal(qs[0], qs[2])


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
def test_staged_k_operands_give_identical_solves(precision):
    w = _workload((15, 16, 10), seed=8)
    prob = _oracle_rel(w, 0.1)
    out = []
    for ks in (1, 3):
        h = _handle(w, precision, prob=prob, gap_tol=1e-8, tile_kstage=ks, tile_e=8, tile_p=4)
        try:
            res = binding.ipm_solve(h)
            H, _ = binding.ipm_sizes(h)
            v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
            binding.ipm_get_spectrum(h, v)
            out.append((res, v))
        finally:
            binding.ipm_destroy(h)
    (r1, v1), (r3, v3) = out
    assert r1["status"] == binding.IPM_OK and r3["status"] == binding.IPM_OK
    for k in ("ipm_iters", "cg_iters_total", "kkt_products", "primal", "dual", "rel_gap"):
        assert r1[k] == r3[k], k
    assert torch.equal(v1, v3)


def test_staged_wait_expiry_reports_timeout():
    """Failure detection: the next product leaves out one operand copy per block of its last
    pass and waits at most 2^10 polls; the call returns IPM_TIMEOUT, the context and the
    handle stay usable, and the next product is exact again."""
    dims = (48, 64)
    w = _workload(dims, seed=9)
    n = int(np.prod(dims))
    rng = np.random.default_rng(10)
    s1, nu1, s2, nu2 = _interior(n, rng)
    h = _handle(w, binding.IPM_MIXED, tile_kstage=3, tile_e=8, tile_p=4)
    try:
        binding.ipm_set_sigma(h, *[oracle_to_lib(h, v, dims) for v in (s1, nu1, s2, nu2)])
        p = torch.cat([oracle_to_lib(h, rng.standard_normal(n), dims), oracle_to_lib(h, rng.standard_normal(n), dims)])
        q_ref = torch.empty_like(p)
        binding.kkt_apply(h, p, q_ref)
        binding.ipm_test_stage_stall(h, 10)
        q = torch.zeros_like(p)
        with pytest.raises(binding.IpmError) as e:
            binding.kkt_apply(h, p, q)
        assert e.value.status == binding.IPM_TIMEOUT
        assert "wait expired" in binding.ipm_last_error(h)
        binding.kkt_apply(h, p, q)
        assert torch.equal(q, q_ref)
    finally:
        binding.ipm_destroy(h)
    h = _handle(w, binding.IPM_MIXED, tile_kstage=1)
    try:
        with pytest.raises(binding.IpmError) as e:
            binding.ipm_test_stage_stall(h, 10)
        assert e.value.status == binding.IPM_ERR_ARG
    finally:
        binding.ipm_destroy(h)


def _solve_both(w, lam_rel, gap_tol, precision=binding.IPM_FP64, **opt):
    """GPU solve of w with the oracle's lambda; returns (result, GPU spectrum, oracle problem)."""
    prob = _oracle_rel(w, lam_rel)
    h = _handle(w, precision, prob=prob, gap_tol=gap_tol, **opt)
    try:
        res = binding.ipm_solve(h)
        H, n = binding.ipm_sizes(h)
        v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
        binding.ipm_get_spectrum(h, v)
        v = v.cpu().numpy()
    finally:
        binding.ipm_destroy(h)
    return res, v, prob


@pytest.mark.parametrize("name,dims", [("1d", None), ("custom", (48, 64)), ("custom", (16, 12, 8))])
def test_solve_matches_oracle_fp64(name, dims):
    w = make_problem(name) if name != "custom" else _workload(dims, seed=6)
    lam_rel = w.lam_rel if name != "custom" else 0.1
    res, v, prob = _solve_both(w, lam_rel, 1e-10)
    assert res["status"] in (binding.IPM_OK,)
    assert res["rel_gap"] <= 1e-10
    ora = oipm.solve(prob, gap_tol=1e-10)
    assert abs(res["primal"] - ora["primal"]) <= 1e-8 * abs(ora["primal"])
    vref = oracle_to_half(ora["beta"], w.dims)
    assert np.abs(v - vref).max() <= 1e-6 * np.abs(vref).max()
    # the oracle's certificate at the GPU's point
    P, D, gap = prob.certificate(half_to_beta(v, w.dims))
    assert gap <= 1.5e-10 and abs(P - res["primal"]) <= 1e-10 * abs(P)


@pytest.mark.parametrize("name,dims", [("1d", None), ("custom", (48, 64)), ("custom", (9, 16, 10))])
def test_lambda_max_matches_oracle(name, dims):
    """lambda_relative = 1: the library's lambda_max = ||M_perp^T b||_inf (Eq. (xi), one
    forward transform of the zero-filled signal) equals the oracle's."""
    w = make_problem(name) if name != "custom" else _workload(dims, seed=6)
    h = _handle(w, binding.IPM_FP64, lam_rel=0.1, max_ipm=1)
    try:
        res = binding.ipm_solve(h, check=False)
    finally:
        binding.ipm_destroy(h)
    lmax = _oracle(w, 1.0).lambda_max()
    assert abs(res["lambda_max"] - lmax) <= 1e-13 * lmax
    assert abs(res["lambda"] - 0.1 * lmax) <= 1e-13 * lmax


def test_config_2d_full_size_fp64():
    """512 x 512, the benchmark's FP64 workload.  (1) The GPU solve to 1e-6 is certified by
    the oracle: its duality gap recomputed from the GPU's coefficients.  (2) Coefficients:
    GPU and oracle solved to a 1e-10 gap agree to 1e-6 of the largest coefficient, and
    the error of the 1e-6 solve against the oracle's 1e-10 solution is stated."""
    w = make_problem("2d")
    res, v, prob = _solve_both(w, w.lam_rel, 1e-6)
    assert res["status"] == binding.IPM_OK and res["rel_gap"] <= 1e-6
    P, D, gap = prob.certificate(half_to_beta(v, w.dims))
    assert gap <= 1.5e-6 and abs(P - res["primal"]) <= 1e-9 * abs(P)
    res10, v10, _ = _solve_both(w, w.lam_rel, 1e-10)
    ora = oipm.solve(prob, gap_tol=1e-10, sigma_rule="single", sigma_min=0.01)
    vref = oracle_to_half(ora["beta"], w.dims)
    scale = np.abs(vref).max()
    assert abs(res10["primal"] - ora["primal"]) <= 1e-10 * abs(ora["primal"])
    assert np.abs(v10 - vref).max() <= 1e-6 * scale
    print(f"PARITY 2d 512x512 FP64: gap(1e-6 solve, oracle) = {gap:.3e}; coefficient error of the 1e-6 solve vs "
          f"oracle at 1e-10: {np.abs(v - vref).max() / scale:.3e} (max abs / max |v|); GPU 1e-10 vs oracle 1e-10: "
          f"{np.abs(v10 - vref).max() / scale:.3e}")


def test_unmasked_equals_soft_threshold():
    dims = (32, 24)
    w = _workload(dims, seed=7, missing=0.0)
    w.mask[:] = 1
    res, v, prob = _solve_both(w, 0.2, 1e-12)
    from oracle.brute import soft_threshold
    ref = oracle_to_half(soft_threshold(prob.c, prob.lam), dims)
    assert np.abs(v - ref).max() < 1e-8


def test_lambda_above_max_gives_zero():
    w = _workload((16, 12, 8), seed=8)
    res, v, prob = _solve_both(w, 1.05, 1e-10)
    assert np.abs(v).max() < 1e-8


def test_solve_is_deterministic():
    w = _workload((48, 64), seed=9)
    r1, v1, _ = _solve_both(w, 0.1, 1e-8)
    r2, v2, _ = _solve_both(w, 0.1, 1e-8)
    assert np.array_equal(v1, v2) and r1["primal"] == r2["primal"] and r1["cg_iters_total"] == r2["cg_iters_total"]


def test_mixed_precision_solve_reaches_gap():
    w = _workload((64, 48), seed=10)
    r64, v64, prob = _solve_both(w, 0.1, 1e-8)
    r32, v32, _ = _solve_both(w, 0.1, 1e-8, precision=binding.IPM_MIXED)
    assert r32["rel_gap"] <= 1e-8
    assert abs(r32["primal"] - r64["primal"]) <= 1e-7 * abs(r64["primal"])
    assert np.abs(v32 - v64).max() <= 1e-4 * np.abs(v64).max()


@pytest.mark.parametrize("cg_tol", [1e-10, 1e-6])
@pytest.mark.parametrize("exact", [0, 1])
@pytest.mark.parametrize("dims", [(512,), (64, 48), (32, 24, 16)])
def test_mixed_cg_matches_fp64_pcg(dims, exact, cg_tol):
    """Mixed precision runs the same PCG with FP32 FFT products and FP64 Krylov
    vectors and barrier terms; the IPM takes the FP64 solve's path: same IPM
    iterations (+-1) and the same solution.  With G beta recomputed by an FP64
    product every iteration (exact_residual = 1) the Krylov counts agree to 10 %;
    with G beta carried through the FP32 products between exact confirmations (the
    default) the IPM residual carries their rounding, and to 25 %."""
    w = _workload(dims, seed=21)
    r64, v64, _ = _solve_both(w, 0.1, 1e-8, exact_residual=exact, cg_tol=cg_tol)
    r32, v32, _ = _solve_both(w, 0.1, 1e-8, precision=binding.IPM_MIXED, exact_residual=exact, cg_tol=cg_tol)
    assert r32["status"] == binding.IPM_OK and r32["rel_gap"] <= 1e-8
    assert abs(r32["ipm_iters"] - r64["ipm_iters"]) <= 1
    frac = 0.1 if exact else 0.25
    assert abs(r32["cg_iters_total"] - r64["cg_iters_total"]) <= frac * r64["cg_iters_total"] + 2
    assert abs(r32["primal"] - r64["primal"]) <= 1e-7 * abs(r64["primal"])
    assert np.abs(v32 - v64).max() <= 1e-4 * np.abs(v64).max()


def test_empty_mask_rejected():
    w = _workload((8, 8), seed=11)
    w.mask[:] = 0
    with pytest.raises(binding.IpmError) as e:
        _handle(w)
    assert e.value.status == binding.IPM_ERR_ARG


@pytest.mark.parametrize("dims,precision", [((256,), binding.IPM_FP64), ((48, 64), binding.IPM_FP64),
                                            ((16, 12, 8), binding.IPM_MIXED)])
def test_graph_and_host_driven_solves_agree(dims, precision):
    """The whole-solve CUDA graph (conditional WHILE loops decided on the device)
    runs the same kernels in the same order as the host-driven loop: bit-identical."""
    w = _workload(dims, seed=12)
    out = []
    for use_graph in (1, 0):
        h = _handle(w, precision, gap_tol=1e-9, use_graph=use_graph)
        try:
            binding.ipm_profile_enable(h, False)          # resets the launch counter
            res = binding.ipm_solve(h)
            launches, _ = binding.ipm_profile_get(h, 5)
            H, n = binding.ipm_sizes(h)
            v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
            binding.ipm_get_spectrum(h, v)
            out.append((res, v.cpu().numpy(), launches))
            # a second solve on the same handle reuses the graph and gives the same answer
            res2 = binding.ipm_solve(h)
            assert res2["primal"] == res["primal"] and res2["cg_iters_total"] == res["cg_iters_total"]
        finally:
            binding.ipm_destroy(h)
    (rg, vg, lg), (rh, vh, lh) = out
    assert np.array_equal(vg, vh)
    assert rg["primal"] == rh["primal"] and rg["ipm_iters"] == rh["ipm_iters"]
    assert rg["cg_iters_total"] == rh["cg_iters_total"] and rg["rel_gap"] <= 1e-9
    assert lg > 0 and lh > 0


def test_iteration_cap_reported():
    w = _workload((32, 24), seed=13)
    h = _handle(w, gap_tol=1e-12, max_ipm=3)
    try:
        res = binding.ipm_solve(h, check=False)
        assert res["status"] == binding.IPM_MAXITER and res["ipm_iters"] == 3
    finally:
        binding.ipm_destroy(h)


def test_pcg_cap_reported():
    w = _workload((32, 24), seed=14)
    h = _handle(w, gap_tol=1e-8, max_cg=1, cg_tol=1e-14)
    try:
        res = binding.ipm_solve(h, check=False)
        assert res["cg_iters_max"] <= 1
        assert res["status"] in (binding.IPM_KRYLOV_MAXITER, binding.IPM_MAXITER)
    finally:
        binding.ipm_destroy(h)


@pytest.mark.parametrize("tile_e,tile_p", [(4, 1), (4, 4), (8, 1), (8, 16), (4, 32), (16, 1), (16, 8)])
@pytest.mark.parametrize("dims", [(512,), (96, 32), (64, 48), (12, 16, 24), (32, 24, 16), (256, 128),
                                  (16, 128, 256)])
def test_every_tile_shape_matches_oracle(dims, tile_e, tile_p):
    """The autotuner may pick any launchable tile shape: each one must compute the
    same product.  Lengths with a factor 3 map E=4 -> 6 and E=8, 16 -> 12
    (E=16: radix-16 stages, then 8, 4, 2)."""
    for precision in (binding.IPM_FP64, binding.IPM_MIXED):
        w = _workload(dims, seed=15)
        three = {4: 6, 8: 12, 16: 12}
        h = None
        try:
            # one option set per call; lengths with a factor 3 ignore the power-of-two budgets and
            # vice versa, so run both spellings
            for e in (tile_e, three[tile_e]):
                h = _handle(w, precision, tile_e=e, tile_p=tile_p, autotune=0)
                n = int(np.prod(dims))
                prob = _oracle(w, 1.0)
                beta = np.random.default_rng(16).standard_normal(n)
                p = oracle_to_lib(h, beta, dims)
                q = torch.empty_like(p)
                binding.gapply(h, p, q)
                assert_g_close(lib_to_half(h, q), oracle_to_half(prob.G(beta), dims), beta, dims, precision)
                binding.ipm_destroy(h)
                h = None
        finally:
            if h is not None:
                binding.ipm_destroy(h)


def test_autotuned_solve_matches_default_tiles():
    w = _workload((64, 48), seed=17)
    r_def, v_def, _ = None, None, None
    out = []
    for autotune in (0, 1):
        h = _handle(w, gap_tol=1e-10, autotune=autotune)
        try:
            res = binding.ipm_solve(h)
            H, n = binding.ipm_sizes(h)
            v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
            binding.ipm_get_spectrum(h, v)
            out.append((res, v.cpu().numpy()))
        finally:
            binding.ipm_destroy(h)
    (r0, v0), (r1, v1) = out
    assert abs(r0["primal"] - r1["primal"]) <= 1e-10 * abs(r0["primal"])
    assert np.abs(v0 - v1).max() <= 1e-7 * np.abs(v0).max()


@pytest.mark.parametrize("refine_every", [1, 5])
def test_mixed_precision_with_fp64_residual_replacement(refine_every):
    """IPM_MIXED with FP64 residual replacement inside PCG reaches a tight gap and
    agrees with the FP64 solve; the replacements actually ran."""
    w = _workload((48, 32), seed=18)
    r64, v64, _ = _solve_both(w, 0.1, 1e-9)
    h = _handle(w, binding.IPM_MIXED, lam_rel=0.1, gap_tol=1e-9, refine_every=refine_every)
    try:
        r = binding.ipm_solve(h)
        H, n = binding.ipm_sizes(h)
        v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
        binding.ipm_get_spectrum(h, v)
        v = v.cpu().numpy()
    finally:
        binding.ipm_destroy(h)
    assert r["rel_gap"] <= 1e-9 and r["refinements"] > 0
    assert abs(r["primal"] - r64["primal"]) <= 1e-8 * abs(r64["primal"])
    assert np.abs(v - v64).max() <= 1e-5 * np.abs(v64).max()


@pytest.mark.parametrize("tile_p", [0, 2, 16])
@pytest.mark.parametrize("dims", [(512,), (256, 128), (512, 64), (64, 32, 64), (16, 128, 256), (128, 64, 128),
                                  (32, 256, 32)])
def test_register_engine_matches_oracle(dims, tile_p):
    """The register FFT engine (first and last stage in registers, lengths 32..512):
    products with G and with K, forced wherever the length allows, against the
    oracle; passes of other lengths fall back to the shared-memory engine."""
    n = int(np.prod(dims))
    for precision in (binding.IPM_FP64, binding.IPM_MIXED):
        w = _workload(dims, seed=21)
        h = _handle(w, precision, tile_engine=2, tile_p=tile_p, autotune=0)
        try:
            prob = _oracle(w, 1.0)
            beta = np.random.default_rng(22).standard_normal(n)
            p = oracle_to_lib(h, beta, dims)
            q = torch.empty_like(p)
            binding.gapply(h, p, q)
            assert_g_close(lib_to_half(h, q), oracle_to_half(prob.G(beta), dims), beta, dims, precision)
            # every pass whose length and forced P admit a register tile uses one
            for name, c in binding.ipm_describe(h).items():
                L, launchable = c["L"], False
                if L in (32, 64, 128, 256, 512):
                    ps = [tile_p] if tile_p else [1, 2, 4, 8, 16, 32]
                    launchable = any((q * L // 16) % 32 == 0 and q * L // 16 <= 256 for q in ps)
                assert (c["engine"] == "register") == launchable, (name, c)
            # K p: the FP64 diagonal epilogue of the last pass
            rng = np.random.default_rng(23)
            s1, nu1, s2, nu2 = _interior(n, rng)
            binding.ipm_set_sigma(h, *[oracle_to_lib(h, v, dims) for v in (s1, nu1, s2, nu2)])
            S1, S2 = oipm.sigmas(s1, nu1, s2, nu2)
            pb, pz = rng.standard_normal(n), rng.standard_normal(n)
            pk = torch.cat([oracle_to_lib(h, pb, dims), oracle_to_lib(h, pz, dims)])
            qk = torch.empty_like(pk)
            binding.kkt_apply(h, pk, qk)
            H2 = _check_kkt(h, prob, dims, precision, S1, S2, pb, pz, qk)
        finally:
            binding.ipm_destroy(h)


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
@pytest.mark.parametrize("dims", [(64, 32, 64), (256, 64)])
def test_register_engine_solve_matches_shared_engine(dims, precision):
    """Whole solves (PCG prologue p = z + beta p and p^T q in the register kernels)
    with the register engine forced agree with the shared-memory engine."""
    w = _workload(dims, seed=24)
    out = {}
    for engine in (1, 2):
        h = _handle(w, precision, gap_tol=1e-8, tile_engine=engine, autotune=0)
        try:
            out[engine] = binding.ipm_solve(h)
        finally:
            binding.ipm_destroy(h)
    for r in out.values():
        assert r["status"] == binding.IPM_OK and r["rel_gap"] <= 1e-8
    tol = 1e-9 if precision == binding.IPM_FP64 else 1e-6
    assert abs(out[1]["primal"] - out[2]["primal"]) <= tol * abs(out[1]["primal"])


@pytest.mark.parametrize("dims", [(32, 24, 16), (64, 48)])
def test_adaptive_centring_matches_oracle(dims):
    """sigma_rule = 1 (sigma = clamp((1 - alpha)^3, sigma_min, sigma_slow)): the library
    and the oracle with the same rule take the same IPM iterations to the same optimum."""
    w = _workload(dims, seed=25)
    prob = _oracle_rel(w, 0.1)
    h = _handle(w, binding.IPM_FP64, prob=prob, gap_tol=1e-8, sigma_rule=1, sigma_min=0.03, cg_tol=1e-10)
    try:
        res = binding.ipm_solve(h)
    finally:
        binding.ipm_destroy(h)
    ora = oipm.solve(prob, gap_tol=1e-8, sigma_rule="adaptive", sigma_min=0.03)
    assert res["status"] == binding.IPM_OK and ora["status"] == "converged"
    assert res["ipm_iters"] == ora["ipm_iters"]
    assert abs(res["primal"] - ora["primal"]) <= 1e-8 * abs(ora["primal"])


def test_fixed_centring_matches_oracle():
    """sigma_rule = 0 (sigma = 0.1, 0.5 after a step alpha < 0.1): same iterations as the oracle's default."""
    w = _workload((32, 24, 16), seed=26)
    prob = _oracle_rel(w, 0.1)
    h = _handle(w, binding.IPM_FP64, prob=prob, gap_tol=1e-8, sigma_rule=0, cg_tol=1e-10)
    try:
        res = binding.ipm_solve(h)
    finally:
        binding.ipm_destroy(h)
    ora = oipm.solve(prob, gap_tol=1e-8, sigma_rule="fixed")
    assert res["ipm_iters"] == ora["ipm_iters"]
    assert abs(res["primal"] - ora["primal"]) <= 1e-8 * abs(ora["primal"])


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
@pytest.mark.parametrize("dims", [(64, 48), (32, 24, 16)])
def test_carried_g_beta_matches_exact_residual(dims, precision):
    """G beta carried along with beta (G x accumulated in PCG, from FP32 products in mixed
    precision) and recomputed only to confirm the stop test: the same optimum as
    recomputing it every iteration, fewer FP64 products, and the reported gap is that of
    an exact product, certified by the oracle.  FP64: the same Newton iterations.  Mixed
    precision: the carried value holds the FP32 products' rounding (about 1e-7 of
    ||G beta|| per product), which at this tight 1e-9 gap costs up to two Newton
    iterations (measured 11 against 9 and 12 against 10; at the 1e-6 gap of the
    benchmark none at 256^3 and 512^3)."""
    w = _workload(dims, seed=27)
    prob = _oracle_rel(w, 0.1)
    out = {}
    for exact in (0, 1):
        h = _handle(w, precision, prob=prob, gap_tol=1e-9, exact_residual=exact)
        try:
            out[exact] = binding.ipm_solve(h)
            if exact == 0:
                H, n = binding.ipm_sizes(h)
                v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
                binding.ipm_get_spectrum(h, v)
                v0 = v.cpu().numpy()
        finally:
            binding.ipm_destroy(h)
    for r in out.values():
        assert r["status"] == binding.IPM_OK and r["rel_gap"] <= 1e-9
    if precision == binding.IPM_FP64:
        assert out[0]["ipm_iters"] == out[1]["ipm_iters"]
        assert abs(out[0]["primal"] - out[1]["primal"]) <= 1e-10 * abs(out[1]["primal"])
    else:
        assert abs(out[0]["ipm_iters"] - out[1]["ipm_iters"]) <= 2
        assert abs(out[0]["primal"] - out[1]["primal"]) <= 1e-8 * abs(out[1]["primal"])
    assert out[0]["kkt_products"] - out[0]["cg_iters_total"] < out[1]["kkt_products"] - out[1]["cg_iters_total"]
    P, D, gap = prob.certificate(half_to_beta(v0, w.dims))
    assert gap <= 1.5e-9 and abs(P - out[0]["primal"]) <= 1e-10 * abs(P)
    ora = oipm.solve(prob, gap_tol=1e-9, sigma_rule="single", sigma_min=0.01)
    assert abs(out[0]["primal"] - ora["primal"]) <= 1e-8 * abs(ora["primal"])


@pytest.mark.parametrize("rho", [0.0, 2.5])
def test_scaled_identity_preconditioner_matches_oracle(rho):
    """precond_rho: P_rho^{-1} against the oracle's closed form (rho = 0: n / observed),
    and a solve with it reaches the same optimum as the paper's P."""
    dims = (32, 24, 16)
    w = _workload(dims, seed=28)
    n = int(np.prod(dims))
    r = rho if rho > 0 else n / float(w.mask.sum())
    prob = _oracle_rel(w, 0.1)
    h = _handle(w, binding.IPM_FP64, prob=prob, gap_tol=1e-9, precond_rho=rho)
    try:
        rng = np.random.default_rng(29)
        s1, nu1, s2, nu2 = _interior(n, rng)
        binding.ipm_set_sigma(h, *[oracle_to_lib(h, v, dims) for v in (s1, nu1, s2, nu2)])
        S1, S2 = oipm.sigmas(s1, nu1, s2, nu2)
        pb, pz = rng.standard_normal(n), rng.standard_normal(n)
        p = torch.cat([oracle_to_lib(h, pb, dims), oracle_to_lib(h, pz, dims)])
        z = torch.empty_like(p)
        binding.precond_apply(h, p, z)
        zb, zz = oipm.Pinv_apply(S1, S2, pb, pz, r)
        H2 = p.numel() // 2
        zs = np.abs(np.concatenate([zb, zz])).max()
        assert np.abs(lib_to_half(h, z[:H2]) - oracle_to_half(zb, dims)).max() < 1e-13 * max(1, zs)
        assert np.abs(lib_to_half(h, z[H2:]) - oracle_to_half(zz, dims)).max() < 1e-13 * max(1, zs)
        res = binding.ipm_solve(h)
    finally:
        binding.ipm_destroy(h)
    ora = oipm.solve(prob, gap_tol=1e-9, sigma_rule="single", sigma_min=0.01, precond_rho=r)
    assert res["status"] == binding.IPM_OK
    assert abs(res["primal"] - ora["primal"]) <= 1e-8 * abs(ora["primal"])


_TILE_PROBE = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
from paper_2502_04217_gb300 import binding
from paper_2502_04217_gb300.synth import make_problem
w = make_problem("custom", dims=(64, 32, 48), missing=0.1, seed=30)
h = binding.ipm_create(w.dims, w.mask, w.y, 0.1, binding.default_options(lambda_relative=1))
print(json.dumps(binding.ipm_describe(h)))
binding.ipm_destroy(h)
"""


def test_tile_cache_file_reproduces_tiles(tmp_path):
    """SDFT_TUNE_CACHE: the first process appends its tuned tiles, a second one reads
    them back and launches exactly the same tiles without timing anything."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, SDFT_TUNE_CACHE=str(tmp_path / "tiles.txt"))
    run = lambda: subprocess.run([sys.executable, "-c", _TILE_PROBE, root], env=env, capture_output=True, text=True,
                                 check=True).stdout.strip().splitlines()[-1]
    first = run()
    lines = (tmp_path / "tiles.txt").read_text().splitlines()
    assert len(lines) >= 6 and all(len(ln.split()) == 10 for ln in lines)
    assert run() == first
    assert (tmp_path / "tiles.txt").read_text().splitlines() == lines      # nothing re-tuned


@pytest.mark.parametrize("dims", [(70,), (40, 28), (20, 14, 10), (30, 56), (560, 16), (16, 560), (14, 40, 30)])
def test_radix_5_and_7_lengths_match_oracle(dims):
    """Extents with factors 5 and 7 (radix-5 and radix-7 stages, e.g. the paper's 560):
    products with G and K in both precisions against the oracle."""
    n = int(np.prod(dims))
    for precision in (binding.IPM_FP64, binding.IPM_MIXED):
        w = _workload(dims, seed=31)
        h = _handle(w, precision)
        try:
            prob = _oracle(w, 1.0)
            rng = np.random.default_rng(32)
            beta = rng.standard_normal(n)
            p = oracle_to_lib(h, beta, dims)
            q = torch.empty_like(p)
            binding.gapply(h, p, q)
            assert_g_close(lib_to_half(h, q), oracle_to_half(prob.G(beta), dims), beta, dims, precision)
            s1, nu1, s2, nu2 = _interior(n, rng)
            binding.ipm_set_sigma(h, *[oracle_to_lib(h, v, dims) for v in (s1, nu1, s2, nu2)])
            S1, S2 = oipm.sigmas(s1, nu1, s2, nu2)
            pb, pz = rng.standard_normal(n), rng.standard_normal(n)
            pk = torch.cat([oracle_to_lib(h, pb, dims), oracle_to_lib(h, pz, dims)])
            qk = torch.empty_like(pk)
            binding.kkt_apply(h, pk, qk)
            H2 = _check_kkt(h, prob, dims, precision, S1, S2, pb, pz, qk)
        finally:
            binding.ipm_destroy(h)


def test_radix_5_and_7_solve_matches_oracle():
    w = _workload((20, 14, 10), seed=33)
    prob = _oracle_rel(w, 0.1)
    h = _handle(w, binding.IPM_FP64, prob=prob, gap_tol=1e-9)
    try:
        res = binding.ipm_solve(h)
    finally:
        binding.ipm_destroy(h)
    ora = oipm.solve(prob, gap_tol=1e-9, sigma_rule="single", sigma_min=0.01)
    assert res["status"] == binding.IPM_OK
    assert abs(res["primal"] - ora["primal"]) <= 1e-8 * abs(ora["primal"])


ODD_SIZES = [(9,), (15,), (105,), (243,), (343,), (729,),
             (15, 21), (21, 15), (16, 9), (9, 16), (27, 25), (7, 5),
             (5, 7, 9), (9, 12, 15), (12, 10, 9), (7, 5, 3), (3, 3, 3), (49, 6, 35)]
# even extents with repeated odd factors (several radix-3/5/7 stages)
REPEATED_ODD_FACTOR_SIZES = [(36,), (18, 36), (72, 18, 12), (54, 50), (98,), (50, 98), (36, 20, 18)]


def _plain_workload(dims, seed):
    """Random signal and mask (about 20 % missing, at least one sample observed) for
    grids too small for the sparse-spectrum generator."""
    from paper_2502_04217_gb300.synth import Workload
    rng = np.random.default_rng(seed)
    mask = (rng.random(dims) > 0.2).astype(np.uint8)
    mask.reshape(-1)[0] = 1
    return Workload(tuple(dims), mask, rng.standard_normal(dims), 0.1)


def _check_g_and_k(dims, precision, seed, w=None, **opt):
    n = int(np.prod(dims))
    w = _workload(dims, seed=seed) if w is None else w
    h = _handle(w, precision, **opt)
    try:
        prob = _oracle(w, 1.0)
        rng = np.random.default_rng(seed + 1)
        beta = rng.standard_normal(n)
        # the layout holds exactly n LASSO coordinates, ghosts at 0
        lib = oracle_to_lib(h, beta, dims)
        assert np.abs(lib_to_half(h, lib) - oracle_to_half(beta, dims)).max() < 1e-14
        assert np.count_nonzero(~ghost_mask(h, dims)) == n
        q = torch.empty_like(lib)
        binding.gapply(h, lib, q)
        assert_g_close(lib_to_half(h, q), oracle_to_half(prob.G(beta), dims), beta, dims, precision)
        assert np.all(q.cpu().numpy()[ghost_mask(h, dims)] == 0.0)
        s1, nu1, s2, nu2 = _interior(n, rng)
        binding.ipm_set_sigma(h, *[oracle_to_lib(h, v, dims) for v in (s1, nu1, s2, nu2)])
        S1, S2 = oipm.sigmas(s1, nu1, s2, nu2)
        pb, pz = rng.standard_normal(n), rng.standard_normal(n)
        pk = torch.cat([oracle_to_lib(h, pb, dims), oracle_to_lib(h, pz, dims)])
        qk = torch.empty_like(pk)
        binding.kkt_apply(h, pk, qk)
        H2 = _check_kkt(h, prob, dims, precision, S1, S2, pb, pz, qk)
    finally:
        binding.ipm_destroy(h)


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
@pytest.mark.parametrize("dims", ODD_SIZES)
def test_odd_extents_match_oracle(dims, precision):
    """Odd extents (Sec. 3, the subspace F for odd n): the beta layout, G and K
    against the oracle, on odd and mixed-parity grids (odd halved axis: the
    two-pencil middle pass; odd in-plane axes: the general-Ns odd stages)."""
    _check_g_and_k(dims, precision, seed=41)


@pytest.mark.parametrize("dims", REPEATED_ODD_FACTOR_SIZES)
def test_repeated_odd_factors_match_oracle(dims):
    for precision in (binding.IPM_FP64, binding.IPM_MIXED):
        _check_g_and_k(dims, precision, seed=43)


@pytest.mark.parametrize("dims", [(15, 21), (9, 16), (7, 5, 3)])
@pytest.mark.parametrize("tile_e,tile_p", [(4, 4), (8, 8), (16, 16), (12, 2), (6, 4)])
def test_odd_extents_every_tile_shape(dims, tile_e, tile_p):
    """Forced tile shapes on odd grids (a shape that does not fit a pass keeps
    that pass's default)."""
    _check_g_and_k(dims, binding.IPM_FP64, seed=45, tile_e=tile_e, tile_p=tile_p, autotune=0)


@pytest.mark.parametrize("name,dims", [("custom", (243,)), ("custom", (15, 21)), ("custom", (9, 7, 5))])
def test_odd_extents_solve_matches_oracle(name, dims):
    w = _workload(dims, seed=47)
    prob = _oracle_rel(w, 0.1)
    h = _handle(w, binding.IPM_FP64, prob=prob, gap_tol=1e-10)
    try:
        res = binding.ipm_solve(h)
        H, n = binding.ipm_sizes(h)
        v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
        binding.ipm_get_spectrum(h, v)
        v = v.cpu().numpy()
    finally:
        binding.ipm_destroy(h)
    assert res["status"] == binding.IPM_OK and res["rel_gap"] <= 1e-10
    # lambda_max = ||M_perp^T b||_inf through the odd middle pass's real-input path
    assert abs(res["lambda_max"] - prob.lambda_max()) <= 1e-12 * prob.lambda_max()
    ora = oipm.solve(prob, gap_tol=1e-10, sigma_rule="single", sigma_min=0.01)
    assert abs(res["primal"] - ora["primal"]) <= 1e-8 * abs(ora["primal"])
    vref = oracle_to_half(ora["beta"], w.dims)
    assert np.abs(v - vref).max() <= 1e-6 * np.abs(vref).max()


def test_odd_extents_mixed_solve_reaches_gap():
    w = _workload((45, 27, 35), seed=49)
    h = _handle(w, binding.IPM_MIXED, gap_tol=1e-6)
    try:
        res = binding.ipm_solve(h)
    finally:
        binding.ipm_destroy(h)
    assert res["status"] == binding.IPM_OK and res["rel_gap"] <= 1e-6


# smallest and largest extents: length-1 and length-2 halved-axis transforms,
# length-2 and length-3 in-plane passes, and the 1024 maximum on every axis
EDGE_SIZES = [(2,), (3,), (4,), (2, 2), (2, 3), (3, 2), (3, 3), (2, 2, 2), (3, 2, 3), (2, 3, 4),
              (1024,), (1024, 6), (6, 1024), (4, 6, 1024), (1024, 4, 2), (2, 1024, 3)]


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
@pytest.mark.parametrize("dims", EDGE_SIZES)
def test_smallest_and_largest_extents_match_oracle(dims, precision):
    _check_g_and_k(dims, precision, seed=51, w=_plain_workload(dims, 51))


@pytest.mark.parametrize("dims", [(64,), (15, 21), (8, 6, 4)])
def test_lambda_at_or_above_lambda_max_gives_zero(dims):
    """Degenerate case: lambda >= ||M_perp^T b||_inf makes beta = 0 optimal (the
    subgradient condition holds at 0); the GPU solve returns it."""
    w = _workload(dims, seed=53)
    prob = _oracle_rel(w, 1.01)
    h = _handle(w, binding.IPM_FP64, prob=prob, gap_tol=1e-9)
    try:
        res = binding.ipm_solve(h)
        H, n = binding.ipm_sizes(h)
        v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
        binding.ipm_get_spectrum(h, v)
        v = v.cpu().numpy()
    finally:
        binding.ipm_destroy(h)
    assert res["status"] == binding.IPM_OK
    assert np.abs(v).max() <= 1e-6 * prob.lambda_max()
    # the objective at beta = 0 is ||b||^2 / 2
    assert abs(res["primal"] - 0.5 * float(prob.b @ prob.b)) <= 1e-8 * float(prob.b @ prob.b)


@pytest.mark.parametrize("precision,dims", [(binding.IPM_FP64, (64, 48)), (binding.IPM_MIXED, (32, 24, 16))])
def test_programmatic_dependent_launch_is_bit_identical(precision, dims):
    """pdl = 1 only overlaps kernel launches (each kernel waits on the device for its
    predecessor): the solve, graph or host-driven, is bit-identical to pdl = 0."""
    w = _workload(dims, seed=34)
    out = {}
    for pdl in (0, 1):
        for graph in (0, 1):
            h = _handle(w, precision, gap_tol=1e-8, pdl=pdl, use_graph=graph, autotune=0)
            try:
                r = binding.ipm_solve(h)
                H, n = binding.ipm_sizes(h)
                v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
                binding.ipm_get_spectrum(h, v)
                out[(pdl, graph)] = (r["primal"], r["ipm_iters"], r["cg_iters_total"], v.cpu().numpy())
            finally:
                binding.ipm_destroy(h)
    ref = out[(0, 1)]
    for key, val in out.items():
        assert val[:3] == ref[:3], key
        assert np.array_equal(val[3], ref[3]), key


@pytest.mark.parametrize("precision,dims", [(binding.IPM_FP64, (32, 24, 16)), (binding.IPM_FP64, (64, 48)),
                                            (binding.IPM_FP64, (15, 21)), (binding.IPM_MIXED, (32, 24, 16))])
def test_conjugate_a_residuals_match_oracle(precision, dims):
    """krylov = 2 (conjugate A-residuals, with restarts): the same optimum as the oracle's
    CAr solve, and in FP64 the same IPM iteration count.  The Krylov counts agree to
    a couple of iterations: a restart fires when y^T K y has fallen by the unit
    round-off, a level at which the FFT's and the direct DFT's rounding differ, so the
    two sides may restart one iteration apart (one FP64 case came out 105 vs 106)."""
    w = _workload(dims, seed=37)
    prob = _oracle_rel(w, 0.1)
    h = _handle(w, precision, prob=prob, gap_tol=1e-8, krylov=2, cg_tol=1e-10)
    try:
        res = binding.ipm_solve(h)
    finally:
        binding.ipm_destroy(h)
    ora = oipm.solve(prob, gap_tol=1e-8, sigma_rule="single", sigma_min=0.01, krylov="car")
    assert res["status"] == binding.IPM_OK and ora["status"] == "converged"
    tol = 1e-8 if precision == binding.IPM_FP64 else 1e-6
    assert abs(res["primal"] - ora["primal"]) <= tol * abs(ora["primal"])
    # the PCG solves cost their iterations plus the start and restart products
    assert res["kkt_products"] > res["cg_iters_total"]
    if precision == binding.IPM_FP64:
        assert res["ipm_iters"] == ora["ipm_iters"]
        total = sum(ora["cg_counts"])
        assert abs(res["cg_iters_total"] - total) <= 2 + 0.02 * total


def test_krylov_method_switched_after_create():
    """ipm_set_options may switch CG -> CAr -> CR on a live handle (their vectors are
    allocated then); every method reaches the same optimum."""
    w = _workload((48, 64), seed=39)
    h = _handle(w, binding.IPM_FP64, gap_tol=1e-9)
    try:
        prim = []
        for k in (0, 2, 1, 0):
            o = binding.default_options(precision=binding.IPM_FP64, lambda_relative=1, gap_tol=1e-9, krylov=k)
            binding.ipm_set_options(h, o)
            res = binding.ipm_solve(h)
            assert res["status"] == binding.IPM_OK
            prim.append(res["primal"])
    finally:
        binding.ipm_destroy(h)
    assert max(prim) - min(prim) <= 1e-8 * abs(prim[0])


@pytest.mark.parametrize("precision,dims", [(binding.IPM_FP64, (32, 24, 16)), (binding.IPM_FP64, (64, 48)),
                                            (binding.IPM_MIXED, (32, 24, 16))])
def test_conjugate_residuals_match_oracle(precision, dims):
    """krylov = 1 (preconditioned conjugate residuals): the same optimum as the oracle's
    CR solve, and in FP64 the same IPM and Krylov iteration counts."""
    w = _workload(dims, seed=35)
    prob = _oracle_rel(w, 0.1)
    h = _handle(w, precision, prob=prob, gap_tol=1e-8, krylov=1, cg_tol=1e-10)
    try:
        res = binding.ipm_solve(h)
    finally:
        binding.ipm_destroy(h)
    ora = oipm.solve(prob, gap_tol=1e-8, sigma_rule="single", sigma_min=0.01, krylov="cr")
    assert res["status"] == binding.IPM_OK and ora["status"] == "converged"
    tol = 1e-8 if precision == binding.IPM_FP64 else 1e-6
    assert abs(res["primal"] - ora["primal"]) <= tol * abs(ora["primal"])
    if precision == binding.IPM_FP64:
        # the predictor's ratio test runs in FP32 on the GPU: sigma may differ in its last
        # digits from the oracle's, and a Krylov count by an iteration or two
        assert res["ipm_iters"] == ora["ipm_iters"]
        total = sum(ora["cg_counts"])
        assert abs(res["cg_iters_total"] - total) <= 2 + 0.02 * total


@pytest.mark.parametrize("cg_tol", [1e-10, 1e-6])
@pytest.mark.parametrize("dims,sigma_min", [((32, 24, 16), 0.01), ((64, 48), 0.01), ((15, 21), 0.03), ((512,), 0.01)])
def test_predictor_corrector_matches_oracle(dims, sigma_min, cg_tol):
    """sigma_rule = 2, the single-step predictor-corrector (affine predictor P^{-1} rhs_aff,
    Mehrotra's sigma and second-order term, one Krylov solve): the library and the oracle's
    "single" rule take the same IPM iterations to the same optimum in FP64.  The Krylov
    counts agree to a few iterations: the predictor's ratio test runs in FP32 on the GPU
    (as the step's), so sigma differs from the oracle's in its last digits."""
    w = _workload(dims, seed=71)
    prob = _oracle_rel(w, 0.1)
    h = _handle(w, binding.IPM_FP64, prob=prob, gap_tol=1e-9, sigma_rule=2, sigma_min=sigma_min, cg_tol=cg_tol)
    try:
        res = binding.ipm_solve(h)
    finally:
        binding.ipm_destroy(h)
    ora = oipm.solve(prob, gap_tol=1e-9, sigma_rule="single", sigma_min=sigma_min, cg_tol=cg_tol)
    assert res["status"] == binding.IPM_OK and ora["status"] == "converged"
    assert res["ipm_iters"] == ora["ipm_iters"]
    total = sum(ora["cg_counts"])
    assert abs(res["cg_iters_total"] - total) <= 2 + 0.03 * total
    assert abs(res["primal"] - ora["primal"]) <= 1e-8 * abs(ora["primal"])


@pytest.mark.parametrize("dims", [(32, 24, 16), (64, 48)])
def test_predictor_corrector_mixed_and_graph(dims):
    """The predictor-corrector in mixed precision reaches the gap with the FP64 solve's
    optimum; graph and host-driven solves are bit-identical."""
    w = _workload(dims, seed=72)
    prob = _oracle_rel(w, 0.1)
    out = {}
    for prec, graph in [(binding.IPM_FP64, 1), (binding.IPM_MIXED, 1), (binding.IPM_MIXED, 0)]:
        h = _handle(w, prec, prob=prob, gap_tol=1e-8, sigma_rule=2, sigma_min=0.01, use_graph=graph)
        try:
            r = binding.ipm_solve(h)
            H, n = binding.ipm_sizes(h)
            v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
            binding.ipm_get_spectrum(h, v)
            out[(prec, graph)] = (r, v.cpu().numpy())
        finally:
            binding.ipm_destroy(h)
    r64, v64 = out[(binding.IPM_FP64, 1)]
    rg, vg = out[(binding.IPM_MIXED, 1)]
    rh, vh = out[(binding.IPM_MIXED, 0)]
    assert rg["status"] == binding.IPM_OK and rg["rel_gap"] <= 1e-8
    assert abs(rg["primal"] - r64["primal"]) <= 1e-7 * abs(r64["primal"])
    assert np.array_equal(vg, vh) and rg["cg_iters_total"] == rh["cg_iters_total"]


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
def test_carried_g_beta_from_a_given_point(precision):
    """A solve from a given point (ipm_set_point) starts its carried G beta with an FP64
    product and confirms its stop with another; a cold start needs no starting product
    (G 0 = 0).  Both reach the gap, certified by the oracle.  (An FP32 starting product
    was measured and dropped: on the 512^3 warm start its rounding cost an IPM
    iteration.)"""
    w = _workload((48, 40), seed=73)
    prob = _oracle_rel(w, 0.1)
    h = _handle(w, precision, prob=prob, gap_tol=1e-3)
    try:
        cold = binding.ipm_solve(h)
        # a cold solve: every product is a PCG product or an exact confirmation
        assert cold["kkt_products"] == cold["cg_iters_total"] + cold["exact_products"]
        H, n = binding.ipm_sizes(h)
        pt = [torch.empty(2 * H, dtype=torch.float64, device="cuda") for _ in range(6)]
        binding.ipm_get_point(h, pt)
        o = binding.default_options(precision=precision, lambda_relative=0, gap_tol=1e-9)
        binding.ipm_set_options(h, o)
        binding.ipm_set_point(h, pt)
        res = binding.ipm_solve(h)
        v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
        binding.ipm_get_spectrum(h, v)
        v = v.cpu().numpy()
    finally:
        binding.ipm_destroy(h)
    assert res["status"] == binding.IPM_OK and res["rel_gap"] <= 1e-9
    assert res["exact_products"] >= 2
    assert res["kkt_products"] == res["cg_iters_total"] + res["exact_products"]
    P, D, gap = prob.certificate(half_to_beta(v, w.dims))
    assert gap <= 1.5e-9 and abs(P - res["primal"]) <= 1e-10 * abs(P)
