"""Test-side conversions between the oracle's beta order and the library's layout.

The oracle orders beta as in Eq. (beta) (self-conjugate values, then sqrt2 Re and
sqrt2 Im of the representatives).  The library keeps its own slot order, and
exposes ipm_pack_beta / ipm_unpack_beta to and from the canonical half
spectrum.  Both sides use the same representative rule, so moving a vector
oracle -> half spectrum -> ipm_pack_beta is a pure permutation (positive
vectors stay positive).  Comparisons are made on the half spectrum, which is
unique.
"""

import numpy as np
import torch

from oracle import mapping
from paper_2502_04217_gb300 import binding


def half(v_full, dims):
    """Canonical half spectrum (interleaved re/im, flat) of a full complex spectrum."""
    vh = np.asarray(v_full).reshape(dims)[..., : dims[-1] // 2 + 1]
    return np.stack([vh.real, vh.imag], axis=-1).reshape(-1).copy()


def oracle_to_half(beta, dims):
    return half(mapping.beta_to_v(beta, dims), dims)


def to_device(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def oracle_to_lib(h, beta, dims):
    """Oracle-ordered real vector -> library beta layout (CUDA tensor of 2H doubles)."""
    vh = to_device(oracle_to_half(beta, dims))
    out = torch.empty_like(vh)
    binding.ipm_pack_beta(h, vh, out)
    return out


def lib_to_half(h, beta_lib):
    out = torch.empty_like(beta_lib)
    binding.ipm_unpack_beta(h, beta_lib.contiguous(), out)
    return out.cpu().numpy()


def ghost_mask(h, dims):
    """Boolean mask of ghost coordinates in the library layout (packing ones)."""
    n = int(np.prod(dims))
    # pack a vector of all ones in every beta coordinate: ghosts come back as 0
    ones = oracle_to_lib(h, np.ones(n), dims).cpu().numpy()
    return ones == 0.0


def half_to_beta(v_half, dims):
    """Canonical half spectrum (interleaved re/im, flat) -> beta in the oracle's order:
    the full spectrum is rebuilt by conjugate symmetry, v_{-k} = conj(v_k), then Eq. (beta)."""
    dims = tuple(int(d) for d in dims)
    Nl = dims[-1]
    Hl = Nl // 2 + 1
    v_half = np.asarray(v_half)
    vh = (v_half[0::2] + 1j * v_half[1::2]).reshape(dims[:-1] + (Hl,))
    full = np.zeros(dims, dtype=np.complex128)
    full[..., :Hl] = vh
    mirrored = vh[np.ix_(*[(-np.arange(N)) % N for N in dims[:-1]])] if len(dims) > 1 else vh
    for kd in range(Hl, Nl):
        full[..., kd] = np.conj(mirrored[..., Nl - kd])
    return mapping.v_to_beta(full, dims)
