"""Local approximation of the sampled density and energy-density matrices -- oracle, test-only.

Sec. II.C.1 with S = I.  The localized mask M_L(r) joins basis functions whose centres are at
most r apart.  For function i, L_i holds the columns of I of the functions in row i of
M_L(r_max); the local problem is H_i = L_i^T H L_i, with P_i = f(H_i) and Q_i = H_i f(H_i).
Eq. local_density keeps only column i of each local result:
[P~_L]_{:, i} = L_i P_i L_i^T e_i (and likewise for Q), and the output is that matrix restricted
to the pattern M.  The columns come from different local problems, so the result is not
symmetric.

All orbitals of an atom share its centre, hence its region: the oracle solves one dense local
problem per atom (``eigh``) and keeps the columns of that atom's own functions.  With a
Chebyshev order ``p`` and bounds, f is replaced by its p-term expansion p_f on [emin, emax]
(Sec. II.B.1), evaluated on the local eigenvalues.
"""
from __future__ import annotations

import numpy as np

from . import chebyshev as ch
from . import neighbors, physics


def local_density(H, pos, n_orb, r_max, mu, T, mask=None, box=None, poly=None):
    """(P~_L, Q~_L), dense.  ``mask`` (bool, n x n) restricts the result to M; ``poly`` =
    (emin, emax, p) takes the p-term Chebyshev expansion of f instead of f itself."""
    pos = np.asarray(pos, dtype=np.float64)
    n_atoms = pos.shape[0]
    n = n_atoms * n_orb
    rp, col = neighbors.neighbor_csr(pos, r_max, box)
    Pt = np.zeros((n, n))
    Qt = np.zeros((n, n))
    orb = np.arange(n_orb)
    for a in range(n_atoms):
        region = col[rp[a]:rp[a + 1]]                       # atoms within r_max, a included
        idx = (region[:, None] * n_orb + orb[None, :]).reshape(-1)
        Hi = H[np.ix_(idx, idx)]
        w, V = np.linalg.eigh(Hi)
        if poly is None:
            fw = physics.fermi(w, mu, T)
        else:
            emin, emax, p = poly
            af, _, _ = ch.fd_coefficients(p, emin, emax, mu, T)
            fw = ch.poly_values(af, ch.mapped(w, emin, emax))
        own = np.searchsorted(region, a) * n_orb + orb      # a's functions inside the region
        Vo = V[own, :]                                      # rows of a's functions
        Pt[np.ix_(idx, a * n_orb + orb)] = (V * fw) @ Vo.T
        Qt[np.ix_(idx, a * n_orb + orb)] = (V * (w * fw)) @ Vo.T
    if mask is not None:
        Pt = Pt * mask
        Qt = Qt * mask
    return Pt, Qt
