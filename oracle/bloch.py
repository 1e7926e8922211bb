"""Bloch-theorem oracle for translation-invariant periodic lattices -- oracle, test-only.

The paper's cubic-scaling periodic reference (Sec. II.E, implementation details) uses Bloch's
theorem with uniform Brillouin-zone sampling.  For an L^3 simple-cubic lattice whose bond blocks
depend only on the bond direction d (h_{-d} = h_d^T) the Hamiltonian is block-diagonalised by
plane waves: H(k) = h_0 + sum_d h_d exp(i k.d), k = 2 pi m / L.

Exact observables follow from the eigenvalues of all H(k); the exact value of the probe estimator
r^T q(H) r follows from r_hat(k) = sum_R r_R exp(-i k.R):
r^T q(H) r = (1/L^3) sum_k r_hat(k)^H q(H(k)) r_hat(k).
"""
from __future__ import annotations

import numpy as np


def bloch_hamiltonians(L: int, disp: np.ndarray, blocks: np.ndarray, onsite=None):
    """H(k) for all k on the L^3 grid, shape (L, L, L, b, b) complex."""
    b = blocks.shape[-1]
    m = 2.0 * np.pi * np.arange(L) / L
    kx, ky, kz = np.meshgrid(m, m, m, indexing="ij")
    Hk = np.zeros((L, L, L, b, b), dtype=np.complex128)
    if onsite is not None:
        Hk += np.asarray(onsite, dtype=np.complex128)
    for d, h in zip(disp, blocks):
        ph = np.exp(1j * (kx * d[0] + ky * d[1] + kz * d[2]))
        Hk += ph[..., None, None] * h[None, None, None]
    return Hk


def bands(L, disp, blocks, onsite=None):
    """All eigenvalues (L^3 * b) and eigenvectors of the Bloch Hamiltonians."""
    Hk = bloch_hamiltonians(L, disp, blocks, onsite)
    w, U = np.linalg.eigh(Hk)
    return w, U


def estimator_weights(L: int, R: np.ndarray, U: np.ndarray) -> np.ndarray:
    """w[k, n] = (1/s) sum_i |u_kn^H r_hat_i(k)|^2 / L^3 for probe rows ordered (site, orbital),
    site index (i*L + j)*L + k.  Then (1/s) sum_i r_i^T q(H) r_i = sum_{k,n} w[k,n] q(eps_kn)."""
    b = U.shape[-1]
    s = R.shape[1]
    w = np.zeros(U.shape[:-1])
    for i in range(s):
        r = R[:, i].reshape(L, L, L, b)
        rh = np.fft.fftn(r, axes=(0, 1, 2))            # sum_R r_R exp(-i k.R)
        c = np.einsum("xyzab,xyza->xyzb", U.conj(), rh)
        w += np.abs(c) ** 2
    return w / (s * L ** 3)
