"""Real parametrisation beta = B v of a conjugate-symmetric spectrum.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed
-----------------------
* Sec. 3, definition of the subspace F: a real signal has a conjugate-symmetric
  DFT, v_k = conj(v_{-k}); for even n the entries v_0 and v_{n/2} are real, for
  odd n only v_0 is (the paper's second definition of F, for odd n).
* Sec. 3, Eq. (beta): beta = [v_0, v_{n/2}, sqrt2 Re v_{1:n/2-1},
  sqrt2 Im v_{1:n/2-1}] and its inverse Eq. (v).
* Sec. 3, Eq. (map): with these maps IDFT(v) = A beta with A real orthogonal.

The paper gives the 1D map for even n only and states that 2D/3D analogues
exist.  Our reading for d-dimensional grids N = (N_1, ..., N_d), each N_i even
or odd:

* a frequency k (multi-index, k_i in [0, N_i)) is *self-conjugate* when
  2k = 0 mod N, i.e. every k_i is 0 or (N_i even) N_i/2; there are
  S = prod_i (2 if N_i is even else 1) such points, each contributing the
  single real coordinate v_k;
* every other frequency pairs with -k.  The pair's *representative* is k when
  1 <= k_d and 2 k_d < N_d, and, on the edge planes 2 k_d = 0 mod N_d
  (k_d = 0, and k_d = N_d/2 for even N_d), the member whose leading indices
  (k_1..k_{d-1}) are lexicographically smaller than those of -k.  A
  representative contributes sqrt2 Re v_k and sqrt2 Im v_k;
* beta is ordered as [self-conjugate values, sqrt2 Re of representatives,
  sqrt2 Im of representatives], each group in row-major order of k.

For d = 1 and even n this is exactly Eq. (beta); for odd n it is
[v_0, sqrt2 Re v_{1:(n-1)/2}, sqrt2 Im v_{1:(n-1)/2}], the same construction on
the odd-n subspace (whose printed index range runs to (n+1)/2; the pairs are
k = 1 .. (n-1)/2).  The count is S + (n - S) = n and B stays unitary, so
A = C^H B^H stays real orthogonal (checked by the tests).
"""

import functools

import numpy as np

SQRT2 = np.sqrt(2.0)


@functools.lru_cache(maxsize=None)
def frequency_classes(dims):
    """Flat (row-major) indices of the self-conjugate frequencies, of the
    pair representatives, and of the twin -k of each representative."""
    dims = tuple(int(d) for d in dims)
    for d in dims:
        if d < 2:
            raise ValueError("every grid dimension must be >= 2")
    k = np.indices(dims).reshape(len(dims), -1)          # k[i] = k_i for every flat index
    neg = (-k) % np.asarray(dims)[:, None]                # the multi-index of -k
    self_conj = np.all(neg == k, axis=0)
    kd, Nd = k[-1], dims[-1]
    interior = (kd >= 1) & (2 * kd < Nd)
    edge = (2 * kd) % Nd == 0
    # lexicographic "k[:-1] < neg[:-1]": decided by the first leading index that differs
    lead_less = np.zeros(k.shape[1], dtype=bool)
    undecided = np.ones(k.shape[1], dtype=bool)
    for i in range(len(dims) - 1):
        lead_less |= undecided & (k[i] < neg[i])
        undecided &= k[i] == neg[i]
    is_rep = ~self_conj & (interior | (edge & lead_less))
    sc = np.flatnonzero(self_conj)
    rep = np.flatnonzero(is_rep)
    twin = np.ravel_multi_index(tuple(neg[:, rep]), dims).astype(np.int64)
    n_sc = int(np.prod([2 if N % 2 == 0 else 1 for N in dims]))
    assert sc.size == n_sc and sc.size + 2 * rep.size == int(np.prod(dims))
    return sc.astype(np.int64), rep.astype(np.int64), twin


def beta_to_v(beta, dims):
    """v = B^H beta (Eq. (v)), returned as a complex array of shape ``dims``."""
    dims = tuple(dims)
    sc, rep, twin = frequency_classes(dims)
    beta = np.asarray(beta, dtype=np.float64)
    nsc, nrep = sc.size, rep.size
    v = np.zeros(int(np.prod(dims)), dtype=np.complex128)
    v[sc] = beta[:nsc]
    vr = (beta[nsc:nsc + nrep] + 1j * beta[nsc + nrep:]) / SQRT2
    v[rep] = vr
    v[twin] = np.conj(vr)
    return v.reshape(dims)


def v_to_beta(v, dims):
    """beta = B v (Eq. (beta)) for a conjugate-symmetric v of shape ``dims``."""
    dims = tuple(dims)
    sc, rep, _ = frequency_classes(dims)
    v = np.asarray(v, dtype=np.complex128).reshape(-1)
    return np.concatenate([v[sc].real, SQRT2 * v[rep].real, SQRT2 * v[rep].imag])


def dense_B(dims):
    """The unitary matrix B of Sec. 3 (n x n complex) with beta = B v."""
    n = int(np.prod(dims))
    sc, rep, twin = frequency_classes(tuple(dims))
    B = np.zeros((n, n), dtype=np.complex128)
    for row, k in enumerate(sc):
        B[row, k] = 1.0
    nsc, nrep = sc.size, rep.size
    for i, (k, t) in enumerate(zip(rep, twin)):
        # sqrt2 Re v_k = (v_k + v_{-k}) / sqrt2 ; sqrt2 Im v_k = (v_k - v_{-k}) / (sqrt2 i)
        B[nsc + i, k] = 1 / SQRT2
        B[nsc + i, t] = 1 / SQRT2
        B[nsc + nrep + i, k] = -1j / SQRT2
        B[nsc + nrep + i, t] = 1j / SQRT2
    return B
