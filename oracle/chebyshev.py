"""Chebyshev expansion and the random-probe estimator, evaluated exactly -- oracle, test-only.

Sec. II.B.1 (polynomial approximation): on the spectral interval [emin, emax] the mapped
function h^(x) = h(emin (1 - x)/2 + emax (1 + x)/2) is projected on p Chebyshev polynomials
C_k(cos t) = cos(k t) with coefficients

    alpha_k = (2 - delta_k0)/pi  int_{-1}^{1} C_k(x) h^(x) dx / sqrt(1 - x^2),

evaluated by M-point Chebyshev-Gauss quadrature (nodes t_j = pi (j + 1/2)/M) and a cosine
transform.  Mapped Hamiltonian: H^ = (2H - (emax + emin) I)/(emax - emin).

Sec. II.C.2 (random approximation): with s Rademacher probes r_i (E[r r^T] = I) the trace of a
matrix function is estimated as (1/s) sum_i r_i^T X r_i.  The oracle evaluates that estimator
exactly from the eigen-decomposition H = V diag(eps) V^T: with c_i = V^T r_i the Chebyshev
moments are mu_k = (1/s) sum_i sum_n c_in^2 C_k(x_n).

Sec. II.D (analytic free-energy derivative): the exact derivative of the polynomial estimator
Omega^ = (1/s) sum_i r_i^T q(H^) r_i, q = sum_k g_k beta_k C_k, with the spectral bounds held
fixed, is the Daleckii-Krein form  dOmega^/dH = (2/W) V (Gamma o (C C^T / s)) V^T  with
Gamma_mn the divided difference of q at (x_m, x_n).

Jackson damping factors g_k are not part of the paper; they are the standard kernel-polynomial
factors of Weisse, Wellein, Alvermann & Fehske, Rev. Mod. Phys. 78, 275 (2006), Eq. (71).
"""
from __future__ import annotations

import numpy as np
import scipy.fft

from . import physics

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state: np.ndarray) -> np.ndarray:
    """The SplitMix64 output function (mix64 of java.util.SplittableRandom; Steele, Lea &
    Flood, OOPSLA 2014) applied to a uint64 state array."""
    z = state.astype(np.uint64)
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def probes(n_rows: int, s: int, seed: int) -> np.ndarray:
    """Rademacher probe block R (n_rows x s) of +-1.

    Entry (i, j) is the (x + 1)-th output of a SplitMix64 stream seeded with ``seed``, where the
    counter is x = i * 2^32 + j; the sign is -1 when the top bit of the output is set.
    """
    with np.errstate(over="ignore"):
        i = np.arange(n_rows, dtype=np.uint64)[:, None]
        j = np.arange(s, dtype=np.uint64)[None, :]
        x = (i << np.uint64(32)) | j
        state = np.uint64(seed) + (x + np.uint64(1)) * _GAMMA
        v = splitmix64(state)
    return np.where((v >> np.uint64(63)) == 1, -1.0, 1.0)


def n_nodes(p: int) -> int:
    """Quadrature nodes used for p coefficients."""
    return max(4 * p, 256)


def nodes(M: int):
    t = np.pi * (np.arange(M) + 0.5) / M
    return t, np.cos(t)


def coefficients(h_values: np.ndarray, p: int) -> np.ndarray:
    """alpha_k, k < p, of the function sampled at the M Chebyshev-Gauss nodes x_j = cos t_j.

    alpha_k = (2 - delta_k0)/M * sum_j h(x_j) cos(k t_j); the sum is a type-II DCT.
    """
    M = h_values.shape[-1]
    y = scipy.fft.dct(h_values, type=2, axis=-1)[..., :p]     # 2 sum_j h_j cos(pi k (2j+1)/2M)
    a = y / M
    a[..., 0] *= 0.5
    return a


def coefficients_direct(h_values: np.ndarray, p: int) -> np.ndarray:
    """Same as ``coefficients`` by the explicit O(pM) sum (small cases)."""
    M = h_values.shape[-1]
    t, _ = nodes(M)
    k = np.arange(p)[:, None]
    a = (2.0 / M) * (np.cos(k * t[None, :]) @ h_values)
    a[0] *= 0.5
    return a


def energy_at(x, emin, emax):
    return emin * (1.0 - x) / 2.0 + emax * (1.0 + x) / 2.0


def fd_coefficients(p, emin, emax, mu, T):
    """(alpha[f], alpha[eps f], beta[g]) on p terms."""
    M = n_nodes(p)
    _, x = nodes(M)
    e = energy_at(x, emin, emax)
    f = physics.fermi(e, mu, T)
    g = physics.free_energy_fn(e, mu, T)
    return coefficients(f, p), coefficients(e * f, p), coefficients(g, p)


def jackson(p: int) -> np.ndarray:
    """Jackson damping factors g_k, k < p (g_0 = 1)."""
    k = np.arange(p)
    q = np.pi / (p + 1)
    return ((p - k + 1) * np.cos(q * k) + np.sin(q * k) / np.tan(q)) / (p + 1)


def damping(p: int, use_jackson: bool) -> np.ndarray:
    return jackson(p) if use_jackson else np.ones(p)


def probe_columns(n_rows: int, cols, seed: int) -> np.ndarray:
    """Columns ``cols`` of the probe block ``probes(n_rows, s, seed)`` (any s > max(cols)),
    generated directly from the same counter definition, for blocks too large to hold whole."""
    with np.errstate(over="ignore"):
        i = np.arange(n_rows, dtype=np.uint64)[:, None]
        j = np.asarray(cols, dtype=np.uint64)[None, :]
        x = (i << np.uint64(32)) | j
        state = np.uint64(seed) + (x + np.uint64(1)) * _GAMMA
        v = splitmix64(state)
    return np.where((v >> np.uint64(63)) == 1, -1.0, 1.0)


def cheb_T(x: np.ndarray, p: int) -> np.ndarray:
    """C_k(x) = cos(k arccos x) for k < p (rows) at points x (columns); |x| <= 1."""
    th = np.arccos(np.clip(x, -1.0, 1.0))
    return np.cos(np.arange(p)[:, None] * th[None, :])


def mapped(eps, emin, emax):
    return (2.0 * eps - (emax + emin)) / (emax - emin)


def probe_weights(V: np.ndarray, R: np.ndarray) -> np.ndarray:
    """w_n = (1/s) sum_i (V^T r_i)_n^2."""
    C = V.T @ R
    return (C * C).sum(axis=1) / R.shape[1]


def exact_moments(eps, V, R, emin, emax, p):
    """mu_k = (1/s) sum_i r_i^T C_k(H^) r_i, k < p, exactly (through the eigenpairs)."""
    w = probe_weights(V, R)
    return cheb_T(mapped(eps, emin, emax), p) @ w


def exact_probe_moments(eps, V, R, emin, emax, p):
    """mu_k^(i) = r_i^T C_k(H^) r_i for k < p (rows) and each probe i (columns), exactly: with
    c_i = V^T r_i, mu_k^(i) = sum_n c_in^2 C_k(x_n).  Their mean over i is exact_moments; their
    spread is the sampling error of Sec. II.C.2."""
    C = V.T @ R
    return cheb_T(mapped(eps, emin, emax), p) @ (C * C)


def recurrence_probe_moments(H, R, emin, emax, p):
    """mu_k^(i) = r_i^T C_k(H^) r_i for k < p (rows) and the probes in the columns of R, by the
    three-term recurrence of Eq. poly_PQ in FP64: y_0 = r, y_1 = H^ r, y_{k+1} = 2 H^ y_k - y_{k-1}.
    H is anything with a matrix product (dense or SciPy sparse); for clusters too large for
    the eigen-decomposition."""
    R = np.asarray(R, dtype=np.float64)
    W, c = emax - emin, emax + emin
    hat = lambda Y: (2.0 * (H @ Y) - c * Y) / W
    out = np.zeros((p, R.shape[1]))
    y0 = R
    out[0] = np.sum(R * y0, axis=0)
    if p > 1:
        y1 = hat(y0)
        out[1] = np.sum(R * y1, axis=0)
        for k in range(2, p):
            y0, y1 = y1, 2.0 * hat(y1) - y0
            out[k] = np.sum(R * y1, axis=0)
    return out


def estimator_observables(moments, emin, emax, mu, T, use_jackson=False):
    """(Omega^, E^, N^) = sum_k g_k c_k mu_k with c = beta[g], alpha[eps f], alpha[f]."""
    p = len(moments)
    af, aef, bg = fd_coefficients(p, emin, emax, mu, T)
    gk = damping(p, use_jackson)
    return (float(np.dot(gk * bg, moments)), float(np.dot(gk * aef, moments)),
            float(np.dot(gk * af, moments)))


def estimator_mu(moments, emin, emax, n_electrons, T, use_jackson=False,
                 rel_tol=1e-13, max_iter=200):
    """mu^ with N^(mu) = n_electrons by bisection on [emin, emax] (midpoint of final bracket)."""
    p = len(moments)
    gk = damping(p, use_jackson)
    M = n_nodes(p)
    _, x = nodes(M)
    e = energy_at(x, emin, emax)
    lo, hi = emin, emax
    W = emax - emin
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        n_mid = float(np.dot(gk * coefficients(physics.fermi(e, mid, T), p), moments))
        if n_mid < n_electrons:
            lo = mid
        else:
            hi = mid
        if hi - lo < rel_tol * W:
            break
    return 0.5 * (lo + hi)


def poly_values(coef: np.ndarray, x: np.ndarray) -> np.ndarray:
    """q(x) = sum_k coef_k C_k(x)."""
    return coef @ cheb_T(x, len(coef))


def poly_derivative(coef: np.ndarray, x: np.ndarray) -> np.ndarray:
    """q'(x) = sum_k k coef_k U_{k-1}(x), with U_{k-1}(cos t) = sin(k t)/sin t."""
    p = len(coef)
    th = np.arccos(np.clip(x, -1.0, 1.0))
    k = np.arange(p)[:, None]
    s = np.sin(th)[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        U = np.where(np.abs(s) > 1e-12, np.sin(k * th[None, :]) / s,
                     k * np.where(np.cos(th)[None, :] > 0, 1.0, (-1.0) ** (k + 1)))
    return (coef * np.arange(p)) @ U


def divided_differences(coef: np.ndarray, x: np.ndarray, close: float = 1e-6,
                        max_nodes: int = 8) -> np.ndarray:
    """Gamma_mn = (q(x_m) - q(x_n))/(x_m - x_n).

    For |x_m - x_n| < close the difference quotient loses digits, so the mean-value form
    int_0^1 q'(x_n + t (x_m - x_n)) dt is used instead, by Gauss-Legendre quadrature with
    min(p/2 + 1, max_nodes) nodes: exact for p <= 2 max_nodes - 1, otherwise in error by
    O(|x_m - x_n|^(2 max_nodes) max|q^(2 max_nodes + 1)|), far below rounding for |dx| < 1e-6."""
    q = poly_values(coef, x)
    dx = x[:, None] - x[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        G = (q[:, None] - q[None, :]) / dx
    mi, ni = np.nonzero(np.abs(dx) < close)
    if mi.size:
        nq = max(1, min((len(coef) + 1) // 2 + 1, max_nodes))
        t, w = np.polynomial.legendre.leggauss(nq)
        t = 0.5 * (t + 1.0)
        w = 0.5 * w
        xm, xn = x[mi], x[ni]
        vals = np.zeros(mi.size)
        for tq, wq in zip(t, w):
            vals += wq * poly_derivative(coef, xn + tq * (xm - xn))
        G[mi, ni] = vals
    return G


def estimator_gradient(eps, V, R, emin, emax, mu, T, use_jackson=False, p=None):
    """dOmega^/dH (dense, symmetric) of the p-term estimator at fixed bounds (Sec. II.D)."""
    _, _, bg = fd_coefficients(p, emin, emax, mu, T)
    coef = damping(p, use_jackson) * bg
    x = mapped(eps, emin, emax)
    Gam = divided_differences(coef, x)
    C = V.T @ R
    K = (C @ C.T) / R.shape[1]
    W = emax - emin
    return (2.0 / W) * (V @ (Gam * K) @ V.T)


def hutchinson_sigma(A: np.ndarray, s: int) -> float:
    """Standard error of (1/s) sum_i r_i^T A r_i for Rademacher probes: Var = 2 sum_{j!=k} A_jk^2
    per probe (the element-wise deviation matrix E = 1 - delta of Sec. II.C.2), sigma = sqrt(Var/s)."""
    off = A - np.diag(np.diag(A))
    return float(np.sqrt(2.0 * np.sum(off * off) / s))

