"""Dense (and, for large clusters, sparse) Hamiltonians for the oracle (test-only).

Two models, both orthogonal (S = I, Sec. II.A):

* SK: 9x9 blocks from ``slater_koster.block`` for every neighbour pair a != b (d = R_b - R_a)
  and the diagonal on-site block diag(es, ep x3, ed x5).
* table: blocks looked up by the (minimum-image) displacement vector of each neighbour pair,
  and a per-site on-site diagonal (the simple-cubic test model of Sec. IV and its 9-orbital
  periodic variant).
"""
from __future__ import annotations

import numpy as np

from . import neighbors, slater_koster


def pairs(row_ptr, col):
    """Directed pairs (a, b) of a CSR pattern."""
    n = len(row_ptr) - 1
    a = np.repeat(np.arange(n), np.diff(row_ptr))
    return a, np.asarray(col, dtype=np.int64)


def bond_vectors(pos, a, b, box=None):
    return neighbors.min_image(pos[b] - pos[a], box)


def dense_sk(pos, row_ptr, col, V, r0, decay, onsite_spd, box=None):
    """Dense SK Hamiltonian (9N x 9N)."""
    n = pos.shape[0]
    H = np.zeros((9 * n, 9 * n))
    a, b = pairs(row_ptr, col)
    off = a != b
    blocks = slater_koster.block(bond_vectors(pos, a[off], b[off], box), V, r0, decay)
    for aa, bb, blk in zip(a[off], b[off], blocks):
        H[9 * aa:9 * aa + 9, 9 * bb:9 * bb + 9] = blk
    ons = slater_koster.onsite_block(*onsite_spd)
    for i in range(n):
        H[9 * i:9 * i + 9, 9 * i:9 * i + 9] = ons
    return H


def sparse_sk(pos, row_ptr, col, V, r0, decay, onsite_spd, box=None):
    """The SK Hamiltonian of ``dense_sk`` as a SciPy BSR matrix with 9 x 9 blocks, for clusters
    whose dense matrix does not fit in memory."""
    import scipy.sparse as sp
    n = pos.shape[0]
    a, b = pairs(row_ptr, col)
    off = a != b
    data = np.zeros((len(a), 9, 9))
    data[off] = slater_koster.block(bond_vectors(pos, a[off], b[off], box), V, r0, decay)
    data[~off] = slater_koster.onsite_block(*onsite_spd)
    return sp.bsr_matrix((data, np.asarray(col, dtype=np.int64), np.asarray(row_ptr, dtype=np.int64)),
                         shape=(9 * n, 9 * n))


def table_lookup(d, disp, tol=1e-6):
    """Index into ``disp`` of each displacement d (exact up to tol); -1 if absent."""
    diff = np.abs(d[:, None, :] - disp[None, :, :]).max(axis=2)
    idx = np.argmin(diff, axis=1)
    idx[diff[np.arange(d.shape[0]), idx] > tol] = -1
    return idx


def dense_table(pos, row_ptr, col, n_orb, disp, blocks, onsite_site=None, box=None):
    """Dense Hamiltonian of a lattice-table model (n_orb N x n_orb N)."""
    n = pos.shape[0]
    b_ = n_orb
    H = np.zeros((b_ * n, b_ * n))
    a, b = pairs(row_ptr, col)
    off = a != b
    d = bond_vectors(pos, a[off], b[off], box)
    idx = table_lookup(d, np.asarray(disp, float))
    if np.any(idx < 0):
        raise ValueError("a neighbour displacement is not in the table")
    blocks = np.asarray(blocks, float).reshape(-1, b_, b_)
    for aa, bb, k in zip(a[off], b[off], idx):
        H[b_ * aa:b_ * aa + b_, b_ * bb:b_ * bb + b_] += blocks[k]
    if onsite_site is not None:
        ons = np.asarray(onsite_site, float).reshape(n, -1)
        for i in range(n):
            H[b_ * i:b_ * i + b_, b_ * i:b_ * i + b_] += np.diag(np.broadcast_to(ons[i], (b_,)))
    return H


def sk_bond_grads(pos, row_ptr, col, V, r0, decay, box=None):
    """(a, b, dH_ab/dd) for every off-diagonal directed pair, d = R_b - R_a."""
    a, b = pairs(row_ptr, col)
    off = a != b
    a, b = a[off], b[off]
    g = slater_koster.block_grad(bond_vectors(pos, a, b, box), V, r0, decay)
    return a, b, g
