"""Exact finite-temperature observables from dense diagonalisation -- oracle, test-only.

Follows Sec. II.A of arXiv 1812.05264 with S = I:

* g(x) = -2T ln(1 + exp(-(x - mu)/T)) and f(x) = g'(x) = 2 / (1 + exp((x - mu)/T))
  (spin factor 2, Eq. free_energy_function);
* F = Omega = tr g(H) = sum_i g(eps_i) (Eq. free_energy);
* P = dF/dH = sum_i f(eps_i) phi_i phi_i^T (Eq. density_matrix);
* N = tr P, E = tr[H P];
* dF/dlambda = tr[P dH/dlambda] (Eq. observable), forces F_c = -dOmega/dR_c.

The chemical potential for a given electron count is found by bisection.
"""
from __future__ import annotations

import numpy as np


def fermi(eps, mu, T):
    """f(eps) = 2 / (1 + exp((eps - mu)/T)), evaluated without overflow."""
    z = (np.asarray(eps, dtype=np.float64) - mu) / T
    out = np.empty_like(z)
    pos = z > 0
    ez = np.exp(-z[pos])
    out[pos] = 2.0 * ez / (1.0 + ez)
    out[~pos] = 2.0 / (1.0 + np.exp(z[~pos]))
    return out


def free_energy_fn(eps, mu, T):
    """g(eps) = -2T ln(1 + exp(-(eps - mu)/T)) with a stable softplus."""
    u = -(np.asarray(eps, dtype=np.float64) - mu) / T
    sp = np.maximum(u, 0.0) + np.log1p(np.exp(-np.abs(u)))
    return -2.0 * T * sp


def eigh(H):
    w, V = np.linalg.eigh(H)
    return w, V


def chemical_potential(eps, n_electrons, T, tol=1e-13, max_iter=400):
    """mu with sum_i f(eps_i; mu, T) = n_electrons, by bisection."""
    lo = float(np.min(eps)) - 40.0 * T
    hi = float(np.max(eps)) + 40.0 * T
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        if fermi(eps, mid, T).sum() < n_electrons:
            lo = mid
        else:
            hi = mid
        if hi - lo < tol * max(1.0, abs(mid)):
            break
    return 0.5 * (lo + hi)


def observables(eps, mu, T):
    """(Omega, E, N) = (sum g, sum eps f, sum f)."""
    f = fermi(eps, mu, T)
    return float(free_energy_fn(eps, mu, T).sum()), float((eps * f).sum()), float(f.sum())


def density_matrix(eps, V, mu, T):
    f = fermi(eps, mu, T)
    return (V * f[None, :]) @ V.T


def forces_from_blocks(X, a, b, dH, n_atoms, n_orb):
    """F_c = -sum_{blocks} <X_ab, dH_ab/dR_c> for a matrix X = dOmega/dH (Eq. observable).

    ``dH[k, c]`` is dH_ab/dd_c for the directed pair (a[k], b[k]) with d = R_b - R_a, so
    dH_ab/dR_b = +dH and dH_ab/dR_a = -dH.  Every directed pair is summed separately.
    """
    F = np.zeros((n_atoms, 3))
    o = n_orb
    for k in range(len(a)):
        aa, bb = a[k], b[k]
        Xab = X[o * aa:o * aa + o, o * bb:o * bb + o]
        for c in range(3):
            t = float(np.sum(Xab * dH[k, c]))
            F[bb, c] -= t
            F[aa, c] += t
    return F
