"""Direct random estimates of the sampled density and energy-density matrices -- oracle,
test-only.

Eq. poly_PQ with S = I: for a vector y, P y ~ sum_k alpha_k y_k and Q y ~ H sum_k alpha_k y_k,
where y_k = C_k(H^) y and alpha_k are the Chebyshev coefficients of the Fermi function f
(Sec. II.B.1).  Eq. random_density: the pattern-sampled estimates are
M o P~_R = (1/s) sum_i M o (P r_i r_i^T), likewise for Q.  Unlike the exact M o P they are not
symmetric.

The oracle evaluates them exactly through the eigen-decomposition H = V diag(eps) V^T:
p_f(H^) R = V diag(p_f(x)) V^T R with p_f = sum_k g_k alpha_k C_k, so
P~ = p_f(H^) R R^T / s and Q~ = H P~.  Elementwise, (P r r^T)_jl = sum_m P_jm r_m r_l, whose
variance over Rademacher signs is sum_{m != l} P_jm^2 (the E = 1 - delta of Sec. II.C.2).
"""
from __future__ import annotations

import numpy as np

from . import chebyshev as ch


def block_mask(row_ptr: np.ndarray, col: np.ndarray, n_orb: int) -> np.ndarray:
    """Dense boolean mask M of the block pattern (atom pairs of the CSR, n_orb x n_orb each)."""
    n = len(row_ptr) - 1
    A = np.zeros((n, n), dtype=bool)
    A[np.repeat(np.arange(n), np.diff(row_ptr)), col] = True
    return np.kron(A, np.ones((n_orb, n_orb), dtype=bool))


def fermi_polynomial(eps, emin, emax, mu, T, p, use_jackson=False) -> np.ndarray:
    """p_f(x_n) = sum_k g_k alpha_k C_k(x_n) at the mapped eigenvalues."""
    af, _, _ = ch.fd_coefficients(p, emin, emax, mu, T)
    return ch.poly_values(ch.damping(p, use_jackson) * af, ch.mapped(eps, emin, emax))


def direct_density(eps, V, R, emin, emax, mu, T, p, use_jackson=False):
    """(P~, Q~), dense and unmasked: P~ = p_f(H^) R R^T / s, Q~ = H P~ (Eq. poly_PQ,
    Eq. random_density)."""
    pf = fermi_polynomial(eps, emin, emax, mu, T, p, use_jackson)
    X = V @ (pf[:, None] * (V.T @ R))               # p_f(H^) R
    Pt = X @ R.T / R.shape[1]
    HX = V @ ((eps * pf)[:, None] * (V.T @ R))       # H p_f(H^) R
    Qt = HX @ R.T / R.shape[1]
    return Pt, Qt


def direct_density_sigma(X: np.ndarray, s: int) -> np.ndarray:
    """Standard error of each element of (1/s) sum_i X r_i r_i^T for Rademacher probes:
    sqrt(sum_{m != l} X_jm^2 / s)."""
    row2 = (X * X).sum(axis=1)[:, None]
    return np.sqrt((row2 - X * X) / s)
