"""Multi-colour probe ensemble -- oracle, test-only.

Sec. II.C.3 (hybrid approximation): the n basis functions are split into q colours such that
two functions of one colour sit farther apart than a colouring radius r_max.  One sample R_i of
the ensemble has q columns; column k is nonzero exactly on the functions of colour k, where its
entries have unit modulus and random phase.  The mean of R_i R_i^T is I, and the element-wise
deviation E_jk is 1 when c(j) = c(k) with j != k and 0 otherwise, so the sampling error of
Eq. sampling_error only sees the matrix elements between distinct functions of one colour.

Sec. II.E (implementation details): atom colours come from the Welsh-Powell vertex colouring (Welsh &
Powell, The Computer Journal 10, 85 (1967)) of the graph whose vertices are the atoms and whose
edges join atoms closer than the colouring radius; each of an atom's n_orb orbitals then takes a
colour of its own, so one atom colour stands for n_orb function colours.

Welsh-Powell: list the vertices by non-increasing degree; give the first colour to the first
vertex of the list and then, going down the list, to every vertex not adjacent to one that
already has it; repeat with the next colour on the vertices still uncoloured.

Readings (the paper states none of these details):
* An edge joins atoms a, b when |r_a - r_b|^2 <= r_max^2 (the squared distance rounded as in
  ``neighbors``), so that two atoms of one colour are strictly farther apart than r_max, as the
  ensemble's condition asks.  A periodic box uses the minimum image.
* Vertices of equal degree keep their index order in the list.
* Function (a, o) of atom a and orbital o has colour c(a) * n_orb + o; q = n_orb * q_atoms.
* Real Rademacher signs stand in for the complex random phase (the same E).  The sign of
  function j in sample i is the plain probe entry R[j, i] of ``chebyshev.probes`` (counter
  (j, i)), placed in column i * q + c(j); every other entry of that row is zero.
* The estimator divides by the number of samples s, not by the s * q columns:
  tr X ~ (1/s) sum_i tr(R_i^T X R_i).
"""
from __future__ import annotations

import numpy as np

from . import chebyshev as ch
from . import neighbors


def color_graph(pos: np.ndarray, r_color: float, box=None):
    """CSR (row_ptr, col) of the colouring graph: atom pairs with r^2 <= r_color^2, self
    excluded, columns ascending."""
    rp, col = neighbors.neighbor_csr(pos, r_color, box)
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    keep = col != rows
    col2 = col[keep]
    counts = np.bincount(rows[keep], minlength=n)
    rp2 = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rp2[1:])
    return rp2, col2.astype(np.int64)


def welsh_powell_order(row_ptr: np.ndarray) -> np.ndarray:
    """Vertices by non-increasing degree, equal degrees in index order."""
    deg = np.diff(row_ptr)
    return np.lexsort((np.arange(len(deg)), -deg))


def welsh_powell(row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Colour of every vertex (0, 1, ...), by one colour class at a time over the Welsh-Powell
    list.  Pure-Python loops: small graphs only."""
    n = len(row_ptr) - 1
    order = welsh_powell_order(row_ptr)
    color = np.full(n, -1, dtype=np.int64)
    k = 0
    while (color < 0).any():
        for v in order:
            if color[v] >= 0:
                continue
            nb = col[row_ptr[v]:row_ptr[v + 1]]
            if not np.any(color[nb] == k):
                color[v] = k
        k += 1
    return color


def atom_colors(pos: np.ndarray, r_color: float, box=None) -> np.ndarray:
    """Welsh-Powell colours of the atoms at colouring radius r_color."""
    rp, col = color_graph(pos, r_color, box)
    return welsh_powell(rp, col)


def function_colors(atom_color: np.ndarray, n_orb: int) -> np.ndarray:
    """Colour of each basis function, c(a) * n_orb + o, rows in atom-major order."""
    return (np.asarray(atom_color, dtype=np.int64)[:, None] * n_orb
            + np.arange(n_orb, dtype=np.int64)[None, :]).reshape(-1)


def colored_probes(fcolor: np.ndarray, q: int, R: np.ndarray) -> np.ndarray:
    """The s samples of the ensemble side by side, n x (s * q): column i * q + k holds
    R[j, i] on the functions j of colour k and zero elsewhere."""
    n, s = R.shape
    out = np.zeros((n, s * q))
    rows = np.arange(n)
    for i in range(s):
        out[rows, i * q + fcolor] = R[:, i]
    return out


def exact_colored_moments(eps, V, Rc, n_samples, emin, emax, p):
    """mu_k = (1/s) sum_i tr(R_i^T C_k(H^) R_i), k < p, exactly through the eigenpairs
    (Eq. random_density with the multi-colour R_i)."""
    C = V.T @ Rc
    w = (C * C).sum(axis=1) / n_samples
    return ch.cheb_T(ch.mapped(eps, emin, emax), p) @ w


def colored_estimator_gradient(eps, V, Rc, n_samples, emin, emax, mu, T, p,
                               use_jackson=False):
    """dOmega^/dH of the multi-colour estimator at fixed bounds: the Daleckii-Krein form of
    Sec. II.D with the probe outer products summed over all columns and divided by s."""
    _, _, bg = ch.fd_coefficients(p, emin, emax, mu, T)
    coef = ch.damping(p, use_jackson) * bg
    Gam = ch.divided_differences(coef, ch.mapped(eps, emin, emax))
    C = V.T @ Rc
    K = (C @ C.T) / n_samples
    return (2.0 / (emax - emin)) * (V @ (Gam * K) @ V.T)


def deviation_matrix(fcolor: np.ndarray) -> np.ndarray:
    """E of the multi-colour ensemble: 1 where c(j) = c(k) and j != k, else 0."""
    E = (fcolor[:, None] == fcolor[None, :]).astype(float)
    np.fill_diagonal(E, 0.0)
    return E


def colored_sigma(A: np.ndarray, fcolor: np.ndarray, n_samples: int) -> float:
    """Standard error of (1/s) sum_i tr(R_i^T A R_i) for symmetric A with real signs:
    Var = 2 ||A o E||_F^2 per sample (Eq. sampling_error with the multi-colour E; the factor 2
    is that of real signs), sigma = sqrt(Var/s)."""
    AE = A * deviation_matrix(fcolor)
    return float(np.sqrt(2.0 * np.sum(AE * AE) / n_samples))
