"""Pins for the oracle's local approximation of M o P and M o Q (Sec. II.C.1, Eq. local_density;
CPU only): a three-site chain worked by hand, the whole-cluster limit, the polynomial variant,
the symmetry of a translation- and inversion-invariant lattice, and the decay of the
localization error with the radius."""
import numpy as np
import pytest

import workloads as wl
from oracle import chebyshev as ch, direct as di, hamiltonian, local as lo, neighbors, physics


def test_three_site_chain_by_hand():
    t, mu, T = -1.0, 0.3, 0.2
    pos = np.zeros((3, 3))
    pos[:, 0] = [0.0, 1.0, 2.0]
    H = t * (np.eye(3, k=1) + np.eye(3, k=-1))
    f = lambda e: physics.fermi(np.array([e]), mu, T)[0]
    P, Q = lo.local_density(H, pos, 1, 1.0, mu, T)
    # column 0 from the dimer {0, 1}: eigenvalues +-t, vectors (1, +-1)/sqrt 2
    assert P[0, 0] == pytest.approx((f(t) + f(-t)) / 2, rel=1e-13)
    assert P[1, 0] == pytest.approx((f(t) - f(-t)) / 2, rel=1e-13)
    assert P[2, 0] == 0.0
    assert Q[0, 0] == pytest.approx(t * (f(t) - f(-t)) / 2, rel=1e-13)
    assert Q[1, 0] == pytest.approx(t * (f(t) + f(-t)) / 2, rel=1e-13)
    # column 1 from the whole chain: eigenvalues sqrt2 t, 0, -sqrt2 t with vectors
    # (1, sqrt2, 1)/2, (1, 0, -1)/sqrt2, (1, -sqrt2, 1)/2
    r2 = np.sqrt(2.0)
    assert P[1, 1] == pytest.approx((f(r2 * t) + f(-r2 * t)) / 2, rel=1e-13)
    assert P[0, 1] == pytest.approx(r2 / 4 * (f(r2 * t) - f(-r2 * t)), rel=1e-13)
    assert P[2, 1] == pytest.approx(P[0, 1], rel=1e-13)
    # column 2 mirrors column 0
    assert P[2, 2] == pytest.approx(P[0, 0], rel=1e-13) and P[1, 2] == pytest.approx(P[1, 0], rel=1e-13)
    # one column per local problem: not symmetric
    assert abs(P[0, 1] - P[1, 0]) > 1e-3


def _small_sk(n, jitter=0.05, seed=2):
    V = wl.sk_integrals(5264)
    pos = wl.fcc_sphere(n, jitter=jitter, seed=seed)
    rp, col = neighbors.neighbor_csr(pos, wl.SK_CUTOFF)
    H = hamiltonian.dense_sk(pos, rp, col, V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)
    return pos, rp, col, H


def test_radius_beyond_the_cluster_is_the_exact_density_matrix():
    pos, rp, col, H = _small_sk(13)
    w, V = np.linalg.eigh(H)
    mu, T = float(np.median(w)), 0.3
    P, Q = lo.local_density(H, pos, 9, 50.0, mu, T)
    Pex = physics.density_matrix(w, V, mu, T)
    assert np.allclose(P, Pex, atol=1e-12)
    assert np.allclose(Q, H @ Pex, atol=1e-11)
    M = di.block_mask(rp, col, 9)
    Pm, _ = lo.local_density(H, pos, 9, 50.0, mu, T, mask=M)
    assert np.array_equal(Pm, P * M)


def test_polynomial_variant():
    """With the p-term expansion: beyond the cluster it is p_f(H^) itself; for large p at a
    warm T it matches the exact-f local result."""
    pos, rp, col, H = _small_sk(13)
    w, V = np.linalg.eigh(H)
    emin, emax, mu, T = w.min() - 1.0, w.max() + 1.0, float(np.median(w)), 0.8
    P, _ = lo.local_density(H, pos, 9, 50.0, mu, T, poly=(emin, emax, 60))
    pf = di.fermi_polynomial(w, emin, emax, mu, T, 60)
    assert np.allclose(P, (V * pf) @ V.T, atol=1e-12)
    p = int(np.ceil((emax - emin) / T * np.log(1e12) / 6.4)) + 20
    P1, Q1 = lo.local_density(H, pos, 9, 4.0, mu, T, poly=(emin, emax, p))
    P2, Q2 = lo.local_density(H, pos, 9, 4.0, mu, T)
    assert np.abs(P1 - P2).max() < 1e-9 and np.abs(Q1 - Q2).max() < 1e-8


def test_translation_and_inversion_invariant_lattice_gives_a_symmetric_result():
    L = 6
    pos, box = wl.sc_lattice(L)
    rp, col = neighbors.neighbor_csr(pos, 1.0, box)
    disp = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    H = hamiltonian.dense_table(pos, rp, col, 1, disp, -np.ones(6), box=box)
    P, Q = lo.local_density(H, pos, 1, 2.0, 0.1, 0.5, box=box)
    assert np.allclose(P, P.T, atol=1e-13) and np.allclose(Q, Q.T, atol=1e-13)
    # every site's local problem is the same: equal diagonals
    assert np.ptp(np.diag(P)) < 1e-13


def test_localization_error_falls_with_the_radius():
    """Eq. local_homogeneous_bound: ||M o (P - P~_L)||_F falls roughly like exp(-gamma r_max)."""
    pos, rp, col, H = _small_sk(79, jitter=0.05, seed=4)
    w, V = np.linalg.eigh(H)
    mu, T = float(np.quantile(w, 11 / 18)), 1.0
    Pex = physics.density_matrix(w, V, mu, T)
    M = di.block_mask(rp, col, 9)
    errs = []
    for r in (4.0, 5.2, 6.4, 7.6):
        P, _ = lo.local_density(H, pos, 9, r, mu, T, mask=M)
        errs.append(np.linalg.norm((P - Pex) * M))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.2 * errs[0], errs
