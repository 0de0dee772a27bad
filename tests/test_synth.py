"""The seeded workload generator (no GPU): shapes, mask geometry, seeds."""

import numpy as np
import pytest

from paper_2502_04217_gb300.synth import batch_workloads, lattice_mask, make_problem, paper_signal


def test_config_masks_have_the_stated_missing_fractions():
    # 2d: discs of radius 3 (29 pixels) on a period-16 lattice -> 29/256
    w2 = make_problem("2d")
    assert w2.dims == (512, 512) and abs((1 - w2.mask.mean()) - 29 / 256) < 1e-12
    # 3d: balls |d|^2 <= 4 (33 voxels) on a period-8 lattice -> 33/512
    m3 = lattice_mask((64, 64, 64), 8, 4)
    assert abs((1 - m3.mean()) - 33 / 512) < 1e-12
    w1 = make_problem("1d")
    assert w1.dims == (256,) and int((1 - w1.mask).sum()) == 26


def test_generator_is_seeded_and_deterministic():
    a, b = make_problem("1d"), make_problem("1d")
    assert np.array_equal(a.y, b.y) and np.array_equal(a.mask, b.mask)
    c = make_problem("2d", index=1)
    assert not np.array_equal(c.y, make_problem("2d").y)


def test_batch_workload_shapes():
    ws = batch_workloads(8)
    assert all(w.dims[0] in (32, 48, 64, 96, 128) and len(set(w.dims)) == 1 for w in ws)
    assert all(0.0 < 1 - w.mask.mean() < 0.5 for w in ws)
    assert len({w.dims[0] for w in ws}) >= 2


@pytest.mark.parametrize("dims", [(16, 12), (15, 9), (16, 9), (9, 16), (7, 5, 9)])
def test_sparse_spectrum_is_what_was_planted(dims):
    """The planted frequencies lie on interior slots of the halved axis (for odd
    extents too), so the signal's half spectrum has exactly those entries."""
    w = make_problem("custom", dims=dims, k=5, noise=0.0, missing=0.0, seed=3)
    spec = np.fft.rfftn(w.y, norm="ortho").reshape(-1)
    big = np.flatnonzero(np.abs(spec) > 1e-9)
    assert sorted(big.tolist()) == sorted(int(f) for f in w.freqs)


def test_paper_generator():
    """Sec. 4.1: the separable signal has exactly the frequencies (+-1, +-2, +-3) (four
    slots of the half spectrum), the noise is U(0, 1), and balls of radius 2 on a
    period-6 lattice remove 33/216 = 15.3 % of the samples ("about 15 %")."""
    N = 24
    spec = np.fft.rfftn(paper_signal(N), norm="ortho")
    big = {tuple(int(v) for v in k) for k in np.argwhere(np.abs(spec) > 1e-9)}
    assert big == {(1, 2, 3), (1, N - 2, 3), (N - 1, 2, 3), (N - 1, N - 2, 3)}
    # an odd side: the same three frequencies, no Nyquist entry
    N = 27
    spec = np.fft.rfftn(paper_signal(N), norm="ortho")
    big = {tuple(int(v) for v in k) for k in np.argwhere(np.abs(spec) > 1e-9)}
    assert big == {(1, 2, 3), (1, N - 2, 3), (N - 1, 2, 3), (N - 1, N - 2, 3)}
    w = make_problem("paper", dims=(96,))
    assert w.dims == (96, 96, 96)
    noise = w.y - paper_signal(96)
    assert noise.min() >= 0.0 and noise.max() < 1.0 and abs(noise.mean() - 0.5) < 0.01
    assert abs((1 - w.mask.mean()) - 33 / 216) < 1e-12
