"""Test-side layout helpers (no GPU): the half spectrum <-> beta conversions used to
hand the GPU's results to the oracle are exact permutations and scalings."""

import numpy as np
import pytest

from layout import half_to_beta, oracle_to_half


@pytest.mark.parametrize("dims", [(8,), (9,), (6, 10), (7, 5), (4, 6, 8), (5, 3, 7), (2, 2, 2), (3, 4, 5)])
def test_half_to_beta_inverts_oracle_to_half(dims):
    beta = np.random.default_rng(0).standard_normal(int(np.prod(dims)))
    assert np.abs(half_to_beta(oracle_to_half(beta, dims), dims) - beta).max() < 1e-14
