"""gapply_noalloc: the allocation-free product with M_perp^T M_perp (needs a GPU).

Some callers cannot call cudaMalloc (an application that owns all device
memory through its own allocator or a fixed budget, a pipeline that must not
take the device-wide synchronisation of cudaMalloc/cudaFree, a plugin inside
another program's CUDA context).  For them gapply_noalloc computes the same
product as the handle-based gapply using only a fixed device array compiled
into the library.  These tests call it through the C ABI and compare it with
gapply on the same inputs, twice in a row (the second call finds the first
call's scratch contents), within twice the FP64 FFT error bound of the parity
tests (both sides round), and check that a call only queues work on its stream.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""

import numpy as np
import pytest
import torch

from paper_2502_04217_gb300 import binding
from paper_2502_04217_gb300.synth import Workload, make_problem

from bounds import fft_bound

pytestmark = pytest.mark.gpu


def _close(q, q_ref, p, dims):
    """Both products carry FP64 FFT rounding (the bounds of bounds.py): their difference is
    held to twice the bound, norm-wise against ||p|| and element by element against max |G p|."""
    err = (q - q_ref).abs()
    b = 2 * fft_bound(dims, binding.IPM_FP64)
    return (torch.linalg.vector_norm(err).item() <= b * torch.linalg.vector_norm(p).item()
            and err.max().item() <= b * q_ref.abs().max().item())


def _reference_and_inputs(dims, seed):
    if int(np.prod(dims)) >= 64:
        w = make_problem("custom", dims=dims, missing=0.15, seed=seed)
    else:                   # too small for the sparse-spectrum generator: a random signal and mask
        rng = np.random.default_rng(seed)
        mask = (rng.random(dims) > 0.2).astype(np.uint8)
        mask.reshape(-1)[0] = 1
        w = Workload(tuple(dims), mask, rng.standard_normal(dims), 0.1)
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


# (2,) and (8, 2): a halved axis of length 2 (middle transform of length 1, no FFT stage);
# (384,), (16, 96), (4, 6, 6): middle lengths with a factor 3 (the E = 12 tiles)
@pytest.mark.parametrize("dims", [(256,), (512, 512), (48, 64), (16, 12, 8), (64, 64, 64), (2,), (8, 2), (384,),
                                  (16, 96), (4, 6, 6)])
def test_noalloc_matches_gapply_twice(dims):
    mask_d, p, q_ref = _reference_and_inputs(dims, seed=21)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        q = torch.full_like(p, float("nan"))
        binding.gapply_noalloc(dims, mask_d, p, q, stream=stream.cuda_stream)
        stream.synchronize()
        assert torch.isfinite(q).all()
        assert _close(q, q_ref, p, dims)


def test_noalloc_returns_without_waiting_for_the_stream():
    """The call only queues work: behind a kernel that keeps a side stream busy for tens
    of milliseconds, two back-to-back calls return while that kernel still runs (no
    pageable copy, no synchronisation), and their results are right once it ends."""
    dims = (64, 48)
    mask_d, p, q_ref = _reference_and_inputs(dims, seed=23)
    side = torch.cuda.Stream()
    q1, q2 = torch.empty_like(p), torch.empty_like(p)
    busy_done = torch.cuda.Event()
    binding.gapply_noalloc(dims, mask_d, p, q1, stream=side.cuda_stream)   # first call in this context
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        torch.cuda._sleep(200_000_000)               # about 0.1 s of device clock cycles
        busy_done.record(side)
        binding.gapply_noalloc(dims, mask_d, p, q1, stream=side.cuda_stream)
        binding.gapply_noalloc(dims, mask_d, p, q2, stream=side.cuda_stream)
        still_busy = not busy_done.query()
    side.synchronize()
    assert still_busy, "the calls waited for the stream"
    assert _close(q1, q_ref, p, dims) and _close(q2, q_ref, p, dims)


def test_noalloc_alternating_grids_reuse_scratch():
    """Calls on different grids in a row: each call rewrites what it needs."""
    cases = [_reference_and_inputs(d, seed=22) + (d,) for d in [(96, 32), (8, 6, 4), (96, 32)]]
    stream = torch.cuda.current_stream()
    for mask_d, p, q_ref, d in cases:
        q = torch.empty_like(p)
        binding.gapply_noalloc(d, mask_d, p, q, stream=stream.cuda_stream)
        stream.synchronize()
        assert _close(q, q_ref, p, d)


def test_noalloc_rejects_grids_beyond_its_scratch():
    mask = torch.ones(1, dtype=torch.uint8, device="cuda")
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.IpmError) as e:
        binding.gapply_noalloc((512, 512, 4), mask, v, v)
    assert e.value.status == binding.IPM_ERR_ARG
    assert "too large" in binding.ipm_last_error(None)
