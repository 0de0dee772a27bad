"""Orthonormal DFT and IDFT by explicit Vandermonde matrices.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 3 (Eq. FTdef, FTdef2 and the matrix C): v_k = n^{-1/2} sum_j omega^{jk} x_j
with omega = exp(-2 pi i / n), x_k = n^{-1/2} sum_j conj(omega)^{jk} v_j, i.e.
v = C x and x = C^H v with C unitary.  A d-dimensional grid uses the product of
the one-dimensional matrices, applied one axis at a time (the d-dimensional DFT
is separable by definition).  This is direct summation, O(n * sum N_i): no FFT.
"""

import functools

import numpy as np


@functools.lru_cache(maxsize=None)
def vandermonde(N):
    """The unitary N x N matrix C with C[k, j] = omega^{jk} / sqrt(N)."""
    j = np.arange(N)
    jk = np.outer(j, j) % N                    # reduce the exponent before exp()
    C = np.exp(-2j * np.pi * jk / N) / np.sqrt(N)
    C.setflags(write=False)
    return C


def _apply_each_axis(x, conj):
    out = np.asarray(x, dtype=np.complex128)
    for axis, N in enumerate(out.shape):
        C = vandermonde(N)
        M = np.conj(C) if conj else C           # C is symmetric, so C^H = conj(C)
        out = np.moveaxis(np.tensordot(M, out, axes=([1], [axis])), 0, axis)
    return out


def dft(x):
    """v = C x along every axis (Eq. FTdef)."""
    return _apply_each_axis(x, conj=False)


def idft(v):
    """x = C^H v along every axis (Eq. FTdef2)."""
    return _apply_each_axis(v, conj=True)
