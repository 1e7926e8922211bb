"""Rational (pole) approximation of the Fermi function and its CGLS solves -- oracle, test-only.

Sec. II.B.2: f(x) is approximated in residue-pole form, and P y, Q y follow from one linear
system (H - z_k) g_k = y per pole (Eq. rational_PQ with S = I), solved by CGLS (the conjugate
gradient method on the normal equations, Hestenes & Stiefel 1952), which keeps the structure of
CG for the indefinite complex-shifted matrices.

The paper's own pole fit is numerical and not printed.  This oracle takes the poles and residues
of the continued-fraction expansion of the Fermi function (Ozaki, Phys. Rev. B 75, 035123
(2007)): with the 2N x 2N symmetric tridiagonal matrix B, B_{m,m+1} = 1/(2 sqrt((2m-1)(2m+1))),
its positive eigenvalues b_p and normalised eigenvectors v_p,
    1/(1 + e^u) = 1/2 + sum_p R_p [1/(u - i z_p) + 1/(u + i z_p)],   z_p = 1/b_p,
    R_p = -v_p[0]^2 / (4 b_p^2),
exactly the N-th convergent of the continued fraction, whose error falls exponentially with N.
With u = (x - mu)/T and the spin factor 2 of f (Sec. II.A),
    f(x) = 1 + 2 Re sum_p w_p / (x - zeta_p),   zeta_p = mu + i T z_p,   w_p = 2 T R_p,
the residue-pole form of Eq. rational_fit plus the constant 1 that the expansion carries.
"""
from __future__ import annotations

import numpy as np


def cfe_poles(n_pairs: int):
    """(z_p, R_p), p < n_pairs, ascending z_p > 0, of the continued-fraction expansion above."""
    m = 2 * n_pairs
    B = np.zeros((m, m))
    for k in range(1, m):
        B[k - 1, k] = B[k, k - 1] = 1.0 / (2.0 * np.sqrt((2 * k - 1) * (2 * k + 1)))
    lam, V = np.linalg.eigh(B)
    pos = lam > 0
    b, v0 = lam[pos], V[0, pos]
    z = 1.0 / b
    R = -v0 ** 2 / (4.0 * b ** 2)
    order = np.argsort(z)
    return z[order], R[order]


def fermi_poles(mu: float, T: float, n_pairs: int):
    """(zeta_p, w_p) with f(x) = 1 + 2 Re sum_p w_p / (x - zeta_p), ascending |zeta_p - mu|."""
    z, R = cfe_poles(n_pairs)
    return mu + 1j * T * z, 2.0 * T * R


def fermi_rational(x, mu: float, T: float, n_pairs: int) -> np.ndarray:
    """The rational approximation of f(x) = 2 / (1 + exp((x - mu)/T)) at real x."""
    zeta, w = fermi_poles(mu, T, n_pairs)
    x = np.asarray(x, dtype=np.float64)
    return 1.0 + 2.0 * np.real((w[None, :] / (x[..., None] - zeta[None, :])).sum(axis=-1))


def rational_density(eps, V, R, mu, T, n_pairs):
    """(P~, Q~), dense and unmasked: P~ = f_r(H) R R^T / s, Q~ = H P~ with f_r the rational
    approximation, evaluated through the eigenpairs H = V diag(eps) V^T."""
    fr = fermi_rational(eps, mu, T, n_pairs)
    X = V @ (fr[:, None] * (V.T @ R))
    HX = V @ ((eps * fr)[:, None] * (V.T @ R))
    s = R.shape[1]
    return X @ R.T / s, HX @ R.T / s


def cgls(apply_A, apply_AH, b, x0=None, tol=1e-12, max_iter=10000):
    """CGLS for A x = b (complex), one column at a time or a block with per-column scalars:
    x, the relative residuals ||b - A x|| / ||b|| and the iterations used."""
    x = np.zeros_like(b, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - apply_A(x)
    s = apply_AH(r)
    p = s.copy()
    gamma = np.sum(np.abs(s) ** 2, axis=0)
    bn = np.sqrt(np.sum(np.abs(b) ** 2, axis=0))
    it = 0
    while it < max_iter:
        res = np.sqrt(np.sum(np.abs(r) ** 2, axis=0)) / bn
        if np.all(res < tol):
            break
        q = apply_A(p)
        delta = np.sum(np.abs(q) ** 2, axis=0)
        alpha = np.where(delta > 0, gamma / np.where(delta > 0, delta, 1.0), 0.0)
        x = x + alpha * p
        r = r - alpha * q
        s = apply_AH(r)
        gnew = np.sum(np.abs(s) ** 2, axis=0)
        beta = np.where(gamma > 0, gnew / np.where(gamma > 0, gamma, 1.0), 0.0)
        p = s + beta * p
        gamma = gnew
        it += 1
    res = np.sqrt(np.sum(np.abs(b - apply_A(x)) ** 2, axis=0)) / bn
    return x, res, it


def rational_apply(H, Y, mu, T, n_pairs, tol=1e-12):
    """f_r(H) Y = Y + 2 Re sum_p w_p g_p with (H - zeta_p) g_p = Y solved by CGLS, the poles taken
    from the farthest from mu to the nearest, each solve started from the previous solution."""
    zeta, w = fermi_poles(mu, T, n_pairs)
    out = np.array(Y, dtype=np.float64)
    g = None
    for k in range(n_pairs - 1, -1, -1):
        z = zeta[k]
        g, res, _ = cgls(lambda v: H @ v - z * v, lambda v: H @ v - np.conj(z) * v,
                         Y.astype(np.complex128), g, tol)
        out = out + 2.0 * np.real(w[k] * g)
    return out
