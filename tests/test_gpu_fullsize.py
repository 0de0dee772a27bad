"""Full-size parity of the 3D workloads (needs a GB300): the oracle certifies the
GPU's solutions at the sizes the benchmark runs.

An IPM only approaches the LASSO minimiser of Eq. (realopt), so at full size the
parity check is the oracle's own duality-gap certificate (the LASSO dual at the
scaled residual, a bound on suboptimality by weak duality) recomputed from the
GPU's coefficients with the oracle's direct DFT: the gap must be within 1.5x the
requested tolerance and the primal objective equal to the GPU's to 1e-9.  The
product with G = M_perp^T M_perp at the GPU's solution is compared element by
element with the oracle's (the bounds of bounds.py).  The mixed-precision
coefficients are compared with those of an FP64 solve to a 1e-9 gap, itself
certified by the oracle, and the difference is printed per workload ("PARITY"
lines, collected with pytest -s).

lambda is the oracle's lambda_rel ||M_perp^T b||_inf, passed to the library as an
absolute value.
"""

import numpy as np
import pytest
import torch

from oracle.lasso import Problem
from paper_2502_04217_gb300 import binding
from paper_2502_04217_gb300.synth import batch_workloads, make_problem

from layout import half_to_beta, lib_to_half, oracle_to_half
from bounds import assert_g_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    binding.load()


def _oracle_problem(w):
    prob = Problem(w.dims, w.mask.astype(bool), w.y, 1.0)
    prob.lam = w.lam_rel * prob.lambda_max()
    return prob


def _create(w, prob, precision, gap_tol):
    opt = binding.default_options(precision=precision, lambda_relative=0, gap_tol=gap_tol)
    mask_d = torch.from_numpy(np.ascontiguousarray(w.mask)).cuda()
    y_d = torch.from_numpy(np.ascontiguousarray(w.y)).cuda()
    return binding.ipm_create(w.dims, mask_d, y_d, prob.lam, opt)


def _beta_lib(h):
    H, n = binding.ipm_sizes(h)
    pt = [torch.empty(2 * H, dtype=torch.float64, device="cuda") for _ in range(6)]
    binding.ipm_get_point(h, pt)
    return pt[0]


def _certify(prob, h, res, gap_tol, label):
    """The oracle's certificate at the GPU's coefficients; returns (beta in the oracle's
    order, half spectrum)."""
    beta_lib = _beta_lib(h)
    v = lib_to_half(h, beta_lib)
    beta = half_to_beta(v, prob.dims)
    P, D, gap = prob.certificate(beta)
    assert gap <= 1.5 * gap_tol, (label, gap)
    assert abs(P - res["primal"]) <= 1e-9 * abs(P), (label, P, res["primal"])
    return beta, v, gap


def _check_g(h, prob, beta, precision):
    """G beta at the solution: the library's gapply against the oracle's G."""
    from layout import oracle_to_lib
    p = oracle_to_lib(h, beta, prob.dims)
    q = torch.empty_like(p)
    binding.gapply(h, p, q)
    assert_g_close(lib_to_half(h, q), oracle_to_half(prob.G(beta), prob.dims), beta, prob.dims, precision)


def _coefficient_error(v, v_ref):
    return float(np.abs(v - v_ref).max() / np.abs(v_ref).max())


def test_config_3d_256_mixed_certified():
    """256^3 (5000 frequencies, background, noise, radius-2 balls on a period-8 lattice),
    mixed precision to a 1e-6 gap: certified by the oracle; G at the solution element by
    element in both precisions; coefficient error against a certified FP64 1e-9 solve."""
    w = make_problem("3d")
    prob = _oracle_problem(w)
    h32 = _create(w, prob, binding.IPM_MIXED, 1e-6)
    h64 = _create(w, prob, binding.IPM_FP64, 1e-9)
    try:
        r32 = binding.ipm_solve(h32)
        assert r32["status"] == binding.IPM_OK and r32["rel_gap"] <= 1e-6
        beta32, v32, gap32 = _certify(prob, h32, r32, 1e-6, "256^3 mixed")
        _check_g(h32, prob, beta32, binding.IPM_MIXED)
        _check_g(h64, prob, beta32, binding.IPM_FP64)
        r64 = binding.ipm_solve(h64)
        assert r64["status"] == binding.IPM_OK
        beta64, v64, gap64 = _certify(prob, h64, r64, 1e-9, "256^3 FP64 1e-9")
        err = _coefficient_error(v32, v64)
        assert err <= 1e-3
        print(f"PARITY 3d 256^3 mixed: oracle gap {gap32:.3e} (GPU {r32['rel_gap']:.3e}), "
              f"{r32['ipm_iters']} IPM / {r32['cg_iters_total']} PCG; coefficient error vs certified FP64 "
              f"(oracle gap {gap64:.3e}): {err:.3e} of max |v|")
    finally:
        binding.ipm_destroy(h32)
        binding.ipm_destroy(h64)


def test_config_batch_member_sizes_certified():
    """One member of each batch side (32^3, 48^3, 64^3, 96^3, 128^3) of the 48-problem
    batch, solved together in one batch launch in mixed precision: each certified by the
    oracle, coefficient error against a certified FP64 1e-9 solve."""
    allw = batch_workloads(48)
    picked = {}
    for w in allw:
        picked.setdefault(w.dims[0], w)
    assert sorted(picked) == [32, 48, 64, 96, 128]
    ws = [picked[s] for s in sorted(picked)]
    probs = [_oracle_problem(w) for w in ws]
    opt = binding.default_options(precision=binding.IPM_MIXED, lambda_relative=0, gap_tol=1e-6)
    b = binding.ipm_create_batch([(w.dims, w.mask, w.y, p.lam) for w, p in zip(ws, probs)], opt)
    try:
        res = binding.ipm_solve_batch(b)
        for i, (w, prob) in enumerate(zip(ws, probs)):
            h = binding.ipm_batch_member(b, i)
            assert res[i]["status"] == binding.IPM_OK and res[i]["rel_gap"] <= 1e-6
            beta32, v32, gap32 = _certify(prob, h, res[i], 1e-6, f"batch {w.dims}")
            _check_g(h, prob, beta32, binding.IPM_MIXED)
            h64 = _create(w, prob, binding.IPM_FP64, 1e-9)
            try:
                r64 = binding.ipm_solve(h64)
                _, v64, gap64 = _certify(prob, h64, r64, 1e-9, f"batch {w.dims} FP64")
            finally:
                binding.ipm_destroy(h64)
            err = _coefficient_error(v32, v64)
            assert err <= 1e-3
            print(f"PARITY batch member {w.name} {w.dims[0]}^3 mixed: oracle gap {gap32:.3e}, "
                  f"{res[i]['ipm_iters']} IPM / {res[i]['cg_iters_total']} PCG; coefficient error vs certified "
                  f"FP64: {err:.3e} of max |v|")
    finally:
        binding.ipm_destroy_batch(b)


def test_config_512_warm_start_mixed_certified():
    """512^3 (100000 frequencies): the learned warm start (network inference, the
    predicted interior point) and the mixed-precision solve to a 1e-6 gap, exactly as the
    benchmark runs them, certified by the oracle; the cold FP64 solve of the same
    instance certified too, and the coefficient difference between the two stated."""
    from paper_2502_04217_gb300 import warmstart as wsm
    w = make_problem("3d512")
    prob = _oracle_problem(w)
    h32 = _create(w, prob, binding.IPM_MIXED, 1e-6)
    net = wsm.load()
    try:
        binding.ws_predict(net, h32, wsm.MU_SCALE)
        rw = binding.ipm_solve(h32)
        assert rw["status"] == binding.IPM_OK and rw["rel_gap"] <= 1e-6
        betaw, vw, gapw = _certify(prob, h32, rw, 1e-6, "512^3 warm mixed")
    finally:
        binding.ws_destroy(net)
        binding.ipm_destroy(h32)
    h64 = _create(w, prob, binding.IPM_FP64, 1e-6)
    try:
        r64 = binding.ipm_solve(h64)
        assert r64["status"] == binding.IPM_OK and r64["rel_gap"] <= 1e-6
        _, v64, gap64 = _certify(prob, h64, r64, 1e-6, "512^3 cold FP64")
    finally:
        binding.ipm_destroy(h64)
    err = _coefficient_error(vw, v64)
    assert err <= 1e-3
    print(f"PARITY 3d 512^3 warm mixed: oracle gap {gapw:.3e} (GPU {rw['rel_gap']:.3e}), {rw['ipm_iters']} IPM / "
          f"{rw['cg_iters_total']} PCG; cold FP64: oracle gap {gap64:.3e}, {r64['ipm_iters']} IPM; coefficient "
          f"difference warm mixed vs cold FP64 (both at 1e-6): {err:.3e} of max |v|")
