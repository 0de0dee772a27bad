"""Batched solve: many independent problems in one graph launch (needs a GPU).

Each problem of the batch runs exactly the kernels of a standalone handle, so
its result must be bit-identical to a standalone solve; small members are also
checked against the CPU oracle.
"""

import numpy as np
import pytest
import torch

from oracle import ipm as oipm
from oracle.lasso import Problem
from paper_2502_04217_gb300 import binding
from paper_2502_04217_gb300.synth import lattice_mask, make_problem

from layout import oracle_to_half

pytestmark = pytest.mark.gpu

DIMS = [(16, 12, 8), (8, 8, 8), (24, 16, 12), (32, 24), (256,), (12, 16, 24), (16, 16, 16)]


def _problems(precision_mixed=False):
    out = []
    for i, d in enumerate(DIMS):
        w = make_problem("custom", dims=d, missing=0.12, seed=40 + i)
        out.append(w)
    return out


def _spectrum(h):
    H, n = binding.ipm_sizes(h)
    v = torch.empty(2 * H, dtype=torch.float64, device="cuda")
    binding.ipm_get_spectrum(h, v)
    return v.cpu().numpy()


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
def test_batch_equals_standalone_solves(precision):
    ws = _problems()
    opt = binding.default_options(precision=precision, lambda_relative=1, gap_tol=1e-9)
    b = binding.ipm_create_batch([(w.dims, w.mask, w.y, 0.1) for w in ws], opt)
    try:
        res_b = binding.ipm_solve_batch(b)
        spec_b = [_spectrum(binding.ipm_batch_member(b, i)) for i in range(len(ws))]
        # solving the same batch again gives the same answer (graph reused)
        res_b2 = binding.ipm_solve_batch(b)
        assert [r["primal"] for r in res_b2] == [r["primal"] for r in res_b]
    finally:
        binding.ipm_destroy_batch(b)
    for w, rb, vb in zip(ws, res_b, spec_b):
        h = binding.ipm_create(w.dims, w.mask, w.y, 0.1, opt)
        try:
            r = binding.ipm_solve(h)
            v = _spectrum(h)
        finally:
            binding.ipm_destroy(h)
        assert rb["rel_gap"] <= 1e-9
        assert rb["primal"] == r["primal"] and rb["cg_iters_total"] == r["cg_iters_total"]
        assert np.array_equal(vb, v)


@pytest.mark.parametrize("precision", [binding.IPM_FP64, binding.IPM_MIXED])
def test_batch_with_odd_members_equals_standalone_solves(precision):
    """Odd and mixed-parity grids (Sec. 3, F for odd n) beside even ones in one batch."""
    ws = [make_problem("custom", dims=d, missing=0.12, seed=60 + i)
          for i, d in enumerate([(15, 21), (9, 7, 5), (45,), (16, 12, 8), (27, 10, 9)])]
    opt = binding.default_options(precision=precision, lambda_relative=1, gap_tol=1e-9)
    b = binding.ipm_create_batch([(w.dims, w.mask, w.y, 0.1) for w in ws], opt)
    try:
        res_b = binding.ipm_solve_batch(b)
        spec_b = [_spectrum(binding.ipm_batch_member(b, i)) for i in range(len(ws))]
    finally:
        binding.ipm_destroy_batch(b)
    for w, rb, vb in zip(ws, res_b, spec_b):
        h = binding.ipm_create(w.dims, w.mask, w.y, 0.1, opt)
        try:
            r = binding.ipm_solve(h)
            v = _spectrum(h)
        finally:
            binding.ipm_destroy(h)
        assert rb["rel_gap"] <= 1e-9
        assert rb["primal"] == r["primal"] and rb["cg_iters_total"] == r["cg_iters_total"]
        assert np.array_equal(vb, v)


def test_batch_of_multi_wave_members_equals_standalone_solves():
    """Members of 32^3 to 128^3 (grids of many blocks, several waves) in mixed precision
    with G beta carried through PCG: concurrent members delay one another's blocks, so a
    kernel whose blocks disagree on a flag that the same launch rewrites shows up here as
    a trajectory that differs from the standalone solve."""
    from paper_2502_04217_gb300.synth import batch_workloads
    picked = {}
    for w in batch_workloads(48):
        picked.setdefault(w.dims[0], w)
    ws = [picked[s] for s in sorted(picked)]
    opt = binding.default_options(precision=binding.IPM_MIXED, lambda_relative=1, gap_tol=1e-6)
    assert opt.exact_residual == 0
    b = binding.ipm_create_batch([(w.dims, w.mask, w.y, w.lam_rel) for w in ws], opt)
    try:
        res_b = binding.ipm_solve_batch(b)
    finally:
        binding.ipm_destroy_batch(b)
    for w, rb in zip(ws, res_b):
        h = binding.ipm_create(w.dims, w.mask, w.y, w.lam_rel, opt)
        try:
            r = binding.ipm_solve(h)
        finally:
            binding.ipm_destroy(h)
        assert rb["status"] == binding.IPM_OK and rb["rel_gap"] <= 1e-6
        assert (rb["ipm_iters"], rb["cg_iters_total"], rb["primal"]) == (r["ipm_iters"], r["cg_iters_total"], r["primal"])


def test_batch_members_match_oracle():
    ws = _problems()[:4]
    probs = []
    for w in ws:
        prob = Problem(w.dims, w.mask.astype(bool), w.y, 1.0)
        prob.lam = 0.1 * prob.lambda_max()          # the oracle's lambda, passed as an absolute value
        probs.append(prob)
    opt = binding.default_options(lambda_relative=0, gap_tol=1e-10)
    b = binding.ipm_create_batch([(w.dims, w.mask, w.y, p.lam) for w, p in zip(ws, probs)], opt)
    try:
        res = binding.ipm_solve_batch(b)
        for i, (w, prob) in enumerate(zip(ws, probs)):
            ora = oipm.solve(prob, gap_tol=1e-10)
            assert abs(res[i]["primal"] - ora["primal"]) <= 1e-8 * abs(ora["primal"])
            v = _spectrum(binding.ipm_batch_member(b, i))
            vref = oracle_to_half(ora["beta"], w.dims)
            assert np.abs(v - vref).max() <= 1e-6 * np.abs(vref).max()
    finally:
        binding.ipm_destroy_batch(b)


def test_batch_rejects_a_bad_member_and_keeps_nothing():
    w = make_problem("custom", dims=(8, 8), seed=50)
    with pytest.raises(binding.IpmError) as e:
        binding.ipm_create_batch([(w.dims, w.mask, w.y, 0.1), ((11, 8), w.mask, w.y, 0.1)])
    assert e.value.status == binding.IPM_ERR_ARG
    assert "problem 1" in binding.ipm_last_error(None)

