"""gapply_noalloc: the allocation-free product with M_perp^T M_perp (needs a GPU).

Some callers cannot call cudaMalloc (an application that owns all device
memory through its own allocator or a fixed budget, a pipeline that must not
take the device-wide synchronisation of cudaMalloc/cudaFree, a plugin inside
another program's CUDA context).  For them gapply_noalloc computes the same
product as the handle-based gapply using only a fixed device array compiled
into the library.  These tests call it through the C ABI and compare it with
gapply on the same inputs, twice in a row (the second call finds the first
call's scratch contents), within the FP64 tolerance of the parity tests.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""

import numpy as np
import pytest
import torch

from paper_2502_04217_gb300 import binding
from paper_2502_04217_gb300.synth import make_problem

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12        # max-norm error bound relative to ||p||_2, as in test_gpu_parity


def _reference_and_inputs(dims, seed):
    w = make_problem("custom", dims=dims, missing=0.15, seed=seed)
    opt = binding.default_options(lambda_relative=1)
    h = binding.ipm_create(w.dims, np.ascontiguousarray(w.mask), np.ascontiguousarray(w.y), 0.1, opt)
    try:
        H, n = binding.ipm_sizes(h)
        rng = np.random.default_rng(seed + 100)
        vh = torch.as_tensor(rng.standard_normal(2 * H), dtype=torch.float64, device="cuda")
        p = torch.empty_like(vh)
        binding.ipm_pack_beta(h, vh, p)             # a valid beta-layout vector (ghosts 0)
        q_ref = torch.empty_like(p)
        binding.gapply(h, p, q_ref)
    finally:
        binding.ipm_destroy(h)
    mask_d = torch.as_tensor(np.ascontiguousarray(w.mask).reshape(-1), dtype=torch.uint8, device="cuda")
    return mask_d, p, q_ref


@pytest.mark.parametrize("dims", [(256,), (512, 512), (48, 64), (16, 12, 8), (64, 64, 64)])
def test_noalloc_matches_gapply_twice(dims):
    mask_d, p, q_ref = _reference_and_inputs(dims, seed=21)
    stream = torch.cuda.current_stream()
    tol = FP64_TOL * torch.linalg.vector_norm(p).item()
    for _ in range(2):
        q = torch.full_like(p, float("nan"))
        binding.gapply_noalloc(dims, mask_d, p, q, stream=stream.cuda_stream)
        stream.synchronize()
        assert torch.isfinite(q).all()
        assert (q - q_ref).abs().max().item() <= tol


def test_noalloc_alternating_grids_reuse_scratch():
    """Calls on different grids in a row: each call rewrites what it needs."""
    cases = [_reference_and_inputs(d, seed=22) + (d,) for d in [(96, 32), (8, 6, 4), (96, 32)]]
    stream = torch.cuda.current_stream()
    for mask_d, p, q_ref, d in cases:
        q = torch.empty_like(p)
        binding.gapply_noalloc(d, mask_d, p, q, stream=stream.cuda_stream)
        stream.synchronize()
        assert (q - q_ref).abs().max().item() <= FP64_TOL * torch.linalg.vector_norm(p).item()


def test_noalloc_rejects_grids_beyond_its_scratch():
    mask = torch.ones(1, dtype=torch.uint8, device="cuda")
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.IpmError) as e:
        binding.gapply_noalloc((512, 512, 4), mask, v, v)
    assert e.value.status == binding.IPM_ERR_ARG
    assert "too large" in binding.ipm_last_error(None)
