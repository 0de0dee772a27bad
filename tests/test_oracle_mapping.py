"""Pins for the oracle's beta <-> v map and its direct DFT (no GPU).

Each check is something other than the oracle itself: hand-derived values,
numpy's FFT, the textbook multi-index DFT sum, or orthogonality facts the paper
states (Sec. 3: B unitary, A = C^H B^H real orthogonal, Parseval).
"""

import itertools
import os

import numpy as np
import pytest

from oracle import dft as odft
from oracle import mapping
from oracle.lasso import Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DIMS = [(2,), (4,), (8,), (10,), (4, 6), (6, 4), (2, 8), (4, 4, 4), (2, 4, 6), (6, 2, 4),
        # odd extents (the odd-n subspace of Sec. 3), alone and mixed with even ones
        (3,), (5,), (9,), (15,), (3, 5), (5, 4), (4, 5), (3, 3, 3), (3, 4, 5), (2, 3, 2)]


def _read_golden(name):
    rows = {}
    r2 = np.sqrt(2.0)
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            conv = [float(v.replace("2r", str(2 * r2)).replace("3r", str(3 * r2))
                          .replace("-r", str(-r2)).replace("r", str(r2))) for v in vals]
            rows.setdefault(key, []).append(conv)
    return rows


def _dense_A(dims):
    n = int(np.prod(dims))
    prob = Problem(dims, np.ones(dims, bool), np.zeros(dims), 1.0)
    return np.stack([np.ravel(prob.A(e)) for e in np.eye(n)], axis=1)


def _textbook_idft(v):
    """x_j = n^{-1/2} sum_k exp(+2 pi i k.j / N) v_k, summed over multi-indices."""
    dims = v.shape
    n = v.size
    x = np.zeros(dims, dtype=np.complex128)
    for j in itertools.product(*[range(N) for N in dims]):
        acc = 0j
        for k in itertools.product(*[range(N) for N in dims]):
            ph = sum(ki * ji / Ni for ki, ji, Ni in zip(k, j, dims))
            acc += np.exp(2j * np.pi * ph) * v[k]
        x[j] = acc / np.sqrt(n)
    return x


@pytest.mark.parametrize("dims", DIMS)
def test_B_unitary(dims):
    B = mapping.dense_B(dims)
    n = B.shape[0]
    assert np.abs(B @ B.conj().T - np.eye(n)).max() < 1e-14
    assert np.abs(B.conj().T @ B - np.eye(n)).max() < 1e-14


@pytest.mark.parametrize("dims", DIMS)
def test_maps_are_inverse_and_conjugate_symmetric(dims):
    rng = np.random.default_rng(1)
    n = int(np.prod(dims))
    beta = rng.standard_normal(n)
    v = mapping.beta_to_v(beta, dims)
    neg = v[tuple(np.ix_(*[(-np.arange(N)) % N for N in dims]))]
    assert np.abs(v - np.conj(neg)).max() < 1e-15            # v lies in F
    assert np.abs(mapping.v_to_beta(v, dims) - beta).max() < 1e-14
    # B^H beta via the dense matrix agrees with the indexed map
    assert np.abs(mapping.dense_B(dims).conj().T @ beta - v.reshape(-1)).max() < 1e-14


@pytest.mark.parametrize("dims", DIMS)
def test_A_real_orthogonal(dims):
    A = _dense_A(dims)
    n = A.shape[0]
    assert np.abs(A.T @ A - np.eye(n)).max() < 1e-13
    # A beta = IDFT(B^H beta) really is real, not only its real part
    rng = np.random.default_rng(2)
    beta = rng.standard_normal(n)
    assert np.abs(odft.idft(mapping.beta_to_v(beta, dims)).imag).max() < 1e-13


@pytest.mark.parametrize("dims", [(4,), (6,), (4, 2), (2, 4), (2, 2, 4), (5,), (3, 4), (4, 3), (3, 3, 2)])
def test_A_beta_equals_textbook_sum(dims):
    rng = np.random.default_rng(3)
    beta = rng.standard_normal(int(np.prod(dims)))
    v = mapping.beta_to_v(beta, dims)
    x = _textbook_idft(v)
    prob = Problem(dims, np.ones(dims, bool), np.zeros(dims), 1.0)
    assert np.abs(x.imag).max() < 1e-13
    assert np.abs(prob.A(beta) - x.real).max() < 1e-13


@pytest.mark.parametrize("n", [4, 8, 16, 30])
def test_A_1d_matches_closed_form_of_eq_map(n):
    """Last line of Eq. (map): the real row A_k written out with cos and sin."""
    A = _dense_A((n,))
    h = n // 2
    ref = np.zeros((n, n))
    for k in range(n):
        ref[k, 0] = 1.0
        ref[k, 1] = (-1.0) ** k
        for j in range(1, h):
            ref[k, j + 1] = np.sqrt(2) * np.cos(2 * np.pi * j * k / n)
            ref[k, j + h] = -np.sqrt(2) * np.sin(2 * np.pi * j * k / n)
    ref /= np.sqrt(n)
    assert np.abs(A - ref).max() < 1e-13


@pytest.mark.parametrize("n", [3, 5, 9, 15, 21])
def test_A_1d_odd_closed_form(n):
    """Eq. (map) redone for odd n: no Nyquist term, h = (n-1)/2 pairs, so
    x_k = n^{-1/2} (beta_0 + sum_{j=1}^{h} sqrt2 cos(2 pi jk/n) beta_j
                    - sum_{j=1}^{h} sqrt2 sin(2 pi jk/n) beta_{j+h})."""
    A = _dense_A((n,))
    h = (n - 1) // 2
    ref = np.zeros((n, n))
    for k in range(n):
        ref[k, 0] = 1.0
        for j in range(1, h + 1):
            ref[k, j] = np.sqrt(2) * np.cos(2 * np.pi * j * k / n)
            ref[k, j + h] = -np.sqrt(2) * np.sin(2 * np.pi * j * k / n)
    ref /= np.sqrt(n)
    assert np.abs(A - ref).max() < 1e-13


def test_A_n3_by_hand():
    """n = 3 worked by hand: beta = [v_0, sqrt2 Re v_1, sqrt2 Im v_1],
    cos(2 pi/3) = -1/2, sin(2 pi/3) = sqrt3/2, so sqrt3 A is
    [[1, sqrt2, 0], [1, -1/sqrt2, -sqrt6/2], [1, -1/sqrt2, sqrt6/2]]."""
    r2, r6 = np.sqrt(2.0), np.sqrt(6.0)
    ref = np.array([[1.0, r2, 0.0], [1.0, -1 / r2, -r6 / 2], [1.0, -1 / r2, r6 / 2]]) / np.sqrt(3.0)
    assert np.abs(_dense_A((3,)) - ref).max() < 1e-15


@pytest.mark.parametrize("n", [3, 7, 9, 25])
def test_odd_subspace_of_real_signals(n):
    """Sec. 3, the odd-n subspace: the DFT of a real signal has v_0 real and
    v_k = conj(v_{n-k}) for k = 1 .. (n-1)/2, and no other real entry; the map
    beta = B v then round-trips through x exactly."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    v = np.fft.fft(x, norm="ortho")
    assert abs(v[0].imag) < 1e-14
    for k in range(1, (n - 1) // 2 + 1):
        assert abs(v[k] - np.conj(v[n - k])) < 1e-13
    beta = mapping.v_to_beta(v, (n,))
    prob = Problem((n,), np.ones(n, bool), np.zeros(n), 1.0)
    assert np.abs(prob.A(beta) - x).max() < 1e-13
    assert np.abs(prob.At(x) - beta).max() < 1e-13


def test_representatives_of_odd_1d_order():
    sc, rep, twin = mapping.frequency_classes((7,))
    assert list(sc) == [0] and list(rep) == [1, 2, 3] and list(twin) == [6, 5, 4]


def test_self_conjugate_count_mixed_parity():
    # one self-conjugate index per odd axis, two per even axis
    for dims, count in [((3, 5), 1), ((4, 5), 2), ((5, 4), 2), ((4, 3, 6), 4), ((3, 3, 3), 1)]:
        sc, rep, _ = mapping.frequency_classes(dims)
        assert sc.size == count and sc.size + 2 * rep.size == int(np.prod(dims))


def test_golden_n4():
    g = _read_golden("mapping_n4.txt")
    A_ref = np.array([row[1:] for row in g["A"]]) / 2.0
    assert np.abs(_dense_A((4,)) - A_ref).max() < 1e-15
    vv = np.array(g["V"][0]).reshape(4, 2)
    v = vv[:, 0] + 1j * vv[:, 1]
    assert np.abs(mapping.v_to_beta(v, (4,)) - np.array(g["BETA"][0])).max() < 1e-14
    assert np.abs(mapping.beta_to_v(np.array(g["BETA"][0]), (4,)) - v).max() < 1e-14


@pytest.mark.parametrize("dims", [(8,), (12,), (6, 10), (4, 6, 8), (16, 16), (9,), (15,), (5, 7), (3, 5, 7)])
def test_dft_matches_numpy_fft(dims):
    rng = np.random.default_rng(4)
    x = rng.standard_normal(dims) + 1j * rng.standard_normal(dims)
    assert np.abs(odft.dft(x) - np.fft.fftn(x, norm="ortho")).max() < 1e-13
    assert np.abs(odft.idft(x) - np.fft.ifftn(x, norm="ortho")).max() < 1e-13
    # Parseval (C unitary)
    assert abs(np.linalg.norm(odft.dft(x)) - np.linalg.norm(x)) < 1e-12


def test_representatives_of_paper_1d_order():
    sc, rep, twin = mapping.frequency_classes((8,))
    assert list(sc) == [0, 4] and list(rep) == [1, 2, 3] and list(twin) == [7, 6, 5]


@pytest.mark.parametrize("dims", [(6, 8), (6, 7), (5, 9), (3, 4, 7)])
def test_representatives_cover_half_spectrum_2d(dims):
    # every representative lies in the half spectrum k_d <= N_d/2 used by a real FFT
    sc, rep, twin = mapping.frequency_classes(dims)
    k = np.array(np.unravel_index(rep, dims))
    assert np.all(k[-1] <= dims[-1] // 2)
    allk = np.concatenate([sc, rep, twin])
    assert sorted(allk.tolist()) == list(range(int(np.prod(dims))))
