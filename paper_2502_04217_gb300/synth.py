"""Seeded synthetic workloads: sparse-spectrum real signals with Bragg-like masks.

This module only draws inputs.  It holds none of the recovery method's
arithmetic (no beta map, no masked operators, no KKT algebra): a signal with a
sparse spectrum is synthesised with numpy's inverse real FFT, and masks are
plain geometry.  Both the CUDA path and the CPU oracle consume its outputs.

Workloads (the paper's real X-ray volume is not available; these synthetic
"crystal-like" inputs stand in for it):

* ``1d``     n = 256, 8 frequencies, N(0,1) amplitudes, noise 0.01, 10 % of samples
             missing at uniform positions, lambda = 0.05 lambda_max.
* ``2d``     512 x 512, 200 frequencies, Laplace(0,1) amplitudes, noise 0.02, discs
             of radius 3 removed around every point of a period-16 lattice
             (11.3 % missing), lambda = 0.02 lambda_max.
* ``3d``     256^3, 5000 frequencies, N(0,1) amplitudes, background 1e-3 N(0,1),
             noise 0.01, balls of radius 2 on a period-8 lattice (6.4 % missing),
             lambda = 0.05 lambda_max.
* ``batch``  48 problems with sides drawn from {32, 48, 64, 96, 128}, 0.25 % of the
             frequencies occupied, lattice period 8..16, radius 1..2, random
             lattice offsets, noise 0.01, lambda = 0.05 lambda_max.
* ``3d512``  512^3, 100000 frequencies, background and noise as ``3d``, radius-2
             balls on a period-8 lattice.
* ``paper``  the paper's own synthetic generator (Sec. 4.1), any N x N x N: the
             separable signal x_ijk = f(i, 1, N) f(j, 2, N) f(k, 3, N) with
             f(t, q, N) = cos(2 pi q t / N) + 2 sin(2 pi q t / N), plus iid U(0, 1)
             noise; about 15 % missing "around the Bragg peaks", read as balls of
             radius 2 on a period-6 lattice (15.3 % missing); lambda = 0.05
             lambda_max (the paper does not state its lambda).
* ``custom`` any grid (even or odd extents), see ``make_problem``.

lambda is returned as a *fraction* of lambda_max = ||M_perp^T b||_inf; each
solver computes lambda_max itself.
"""

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2502042170


@dataclass
class Workload:
    dims: tuple
    mask: np.ndarray          # uint8, 1 = observed, shape dims
    y: np.ndarray             # float64, shape dims (values at missing samples are noise)
    lam_rel: float            # lambda / lambda_max
    freqs: np.ndarray = field(repr=False, default=None)   # flat half-spectrum indices used
    amps: np.ndarray = field(repr=False, default=None)    # their complex amplitudes
    name: str = "custom"


def _sparse_signal(rng, dims, k, amp="normal"):
    half = tuple(dims[:-1]) + (dims[-1] // 2 + 1,)
    spec = np.zeros(half, dtype=np.complex128)
    # interior of the last (halved) axis: every such frequency is its own representative
    interior = np.arange(int(np.prod(half)))
    last = interior % half[-1]
    interior = interior[(last >= 1) & (2 * last < dims[-1])]
    freqs = np.sort(rng.choice(interior, size=k, replace=False))
    if amp == "laplace":
        amps = rng.laplace(0.0, 1.0, k) + 1j * rng.laplace(0.0, 1.0, k)
    else:
        amps = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    spec.reshape(-1)[freqs] = amps
    x = np.fft.irfftn(spec, s=dims, axes=tuple(range(len(dims))), norm="ortho")
    return x, freqs, amps


def paper_signal(N):
    """The paper's separable test signal on an N x N x N grid (Sec. 4.1):
    x_ijk = f(i, 1) f(j, 2) f(k, 3), f(t, q) = cos(2 pi q t / N) + 2 sin(2 pi q t / N)."""
    t = np.arange(N)
    f = [np.cos(2 * np.pi * q * t / N) + 2 * np.sin(2 * np.pi * q * t / N) for q in (1, 2, 3)]
    return f[0][:, None, None] * f[1][None, :, None] * f[2][None, None, :]


def lattice_mask(dims, period, radius2, offset=None):
    """uint8 mask: 0 inside every ball |d|^2 <= radius2 around the points of a
    periodic lattice (per-axis period, optional per-axis offset), 1 elsewhere."""
    dims = tuple(dims)
    period = np.broadcast_to(np.asarray(period), (len(dims),))
    offset = np.zeros(len(dims), dtype=np.int64) if offset is None else np.asarray(offset)
    d2 = np.zeros(dims, dtype=np.int64)
    for ax, (N, P, o) in enumerate(zip(dims, period, offset)):
        j = np.arange(N)
        r = (j - o) % P
        dist = np.minimum(r, P - r)                       # distance to the nearest lattice plane
        shape = [1] * len(dims)
        shape[ax] = N
        d2 = d2 + (dist ** 2).reshape(shape)
    return (d2 > radius2).astype(np.uint8)


def make_problem(name, index=0, dims=None, k=None, noise=0.01, missing=0.1, lam_rel=0.05, seed=None):
    cfg = {"1d": 1, "2d": 2, "3d": 3, "batch": 4, "3d512": 5}.get(name, 0)
    rng = np.random.default_rng(SEED_BASE + cfg + 1000 * index + (seed if seed is not None else 0))
    if name == "1d":
        dims = (256,)
        x, f, a = _sparse_signal(rng, dims, 8)
        y = x + 0.01 * rng.standard_normal(dims)
        mask = np.ones(dims, dtype=np.uint8)
        mask[rng.choice(256, size=round(0.1 * 256), replace=False)] = 0
        return Workload(dims, mask, y, 0.05, f, a, name)
    if name == "2d":
        dims = (512, 512)
        x, f, a = _sparse_signal(rng, dims, 200, amp="laplace")
        y = x + 0.02 * rng.standard_normal(dims)
        return Workload(dims, lattice_mask(dims, 16, 9), y, 0.02, f, a, name)
    if name in ("3d", "3d512"):
        big = name == "3d512"
        dims = (512,) * 3 if big else (256,) * 3
        x, f, a = _sparse_signal(rng, dims, 100000 if big else 5000)
        y = x + 1e-3 * rng.standard_normal(dims) + 0.01 * rng.standard_normal(dims)
        return Workload(dims, lattice_mask(dims, 8, 4), y, 0.05, f, a, name)
    if name == "batch":
        side = int(rng.choice([32, 48, 64, 96, 128]))
        dims = (side,) * 3
        n = side ** 3
        x, f, a = _sparse_signal(rng, dims, max(1, round(0.0025 * n)))
        y = x + 0.01 * rng.standard_normal(dims)
        period = int(rng.integers(8, 17))
        radius = int(rng.integers(1, 3))
        offset = rng.integers(0, period, size=3)
        return Workload(dims, lattice_mask(dims, period, radius * radius, offset), y, 0.05, f, a,
                        f"batch[{index}]")
    if name == "paper":
        N = int(dims[0]) if dims is not None else 64
        dims = (N, N, N)
        rng = np.random.default_rng(SEED_BASE + 6 + (seed if seed is not None else 0))
        y = paper_signal(N) + rng.uniform(0.0, 1.0, dims)
        return Workload(dims, lattice_mask(dims, 6, 4), y, 0.05, None, None, f"paper[{N}]")
    if name == "custom":
        dims = tuple(int(d) for d in dims)
        n = int(np.prod(dims))
        x, f, a = _sparse_signal(rng, dims, k if k is not None else max(1, n // 32))
        y = x + noise * rng.standard_normal(dims)
        mask = np.ones(n, dtype=np.uint8)
        mask[rng.choice(n, size=int(round(missing * n)), replace=False)] = 0
        return Workload(dims, mask.reshape(dims), y, lam_rel, f, a, name)
    raise ValueError(f"unknown workload {name!r}")


def batch_workloads(count=48):
    return [make_problem("batch", index=i) for i in range(count)]
