"""Pins for the oracle's direct estimates of M o P~ and M o Q~ (Eq. poly_PQ, Eq. random_density;
CPU only).

The eigen route of the oracle is checked against the paper's own vector recurrence on the
probes and against the dense matrix recurrence on H^; its traces against the moment route
(N^ and a Chebyshev product identity); its mean and element-wise variance by enumerating every
sign vector; its limit against the exact density matrix and forces."""
import numpy as np
import pytest
from scipy.linalg import hadamard

import workloads as wl
from oracle import chebyshev as ch, direct as di, hamiltonian, neighbors, physics


def _small_sk(n, jitter=0.05):
    V = wl.sk_integrals(5264)
    pos = wl.fcc_sphere(n, jitter=jitter, seed=2)
    rp, col = neighbors.neighbor_csr(pos, wl.SK_CUTOFF)
    H = hamiltonian.dense_sk(pos, rp, col, V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)
    return pos, rp, col, V, H


def _setup(n_atoms=13, s=6, p=80, T=0.5):
    pos, rp, col, Vsk, H = _small_sk(n_atoms)
    w, V = np.linalg.eigh(H)
    emin, emax = w.min() - 1.0, w.max() + 1.0
    mu = float(np.median(w))
    R = ch.probes(H.shape[0], s, 21)
    return pos, rp, col, Vsk, H, w, V, emin, emax, mu, T, p, R


def test_eigen_route_equals_the_probe_recurrence():
    """P~ from the eigenpairs equals (1/s) sum_k alpha_k y_k R^T with y_k run by the three-term
    recurrence on the probes, as Eq. poly_PQ prescribes; Q~ = H times it."""
    _, _, _, _, H, w, V, emin, emax, mu, T, p, R = _setup()
    Pt, Qt = di.direct_density(w, V, R, emin, emax, mu, T, p)
    af, _, _ = ch.fd_coefficients(p, emin, emax, mu, T)
    Hh = (2 * H - (emax + emin) * np.eye(H.shape[0])) / (emax - emin)
    y0, y1 = R, Hh @ R
    X = af[0] * y0 + af[1] * y1
    for k in range(2, p):
        y0, y1 = y1, 2 * Hh @ y1 - y0
        X += af[k] * y1
    s = R.shape[1]
    assert np.allclose(Pt, X @ R.T / s, rtol=1e-10, atol=1e-11)
    assert np.allclose(Qt, H @ X @ R.T / s, rtol=1e-10, atol=1e-10)
    assert not np.allclose(Pt, Pt.T, atol=1e-6)             # nonsymmetric for finite s


def test_hadamard_probes_give_the_polynomial_matrix():
    """(1/n) R R^T = I for a Sylvester-Hadamard R: P~ = p_f(H^), computed here by the dense
    matrix recurrence."""
    _, _, _, _, H = _small_sk(8)
    H = H[:64, :64]
    w, V = np.linalg.eigh(H)
    emin, emax, mu, T, p = w.min() - 0.5, w.max() + 0.5, float(np.median(w)), 0.4, 70
    Pt, Qt = di.direct_density(w, V, hadamard(64).astype(float), emin, emax, mu, T, p)
    af, _, _ = ch.fd_coefficients(p, emin, emax, mu, T)
    Hh = (2 * H - (emax + emin) * np.eye(64)) / (emax - emin)
    T0, T1 = np.eye(64), Hh
    F = af[0] * T0 + af[1] * T1
    for k in range(2, p):
        T0, T1 = T1, 2 * Hh @ T1 - T0
        F += af[k] * T1
    assert np.allclose(Pt, F, atol=1e-11)
    assert np.allclose(Qt, H @ F, atol=1e-10)


def test_traces_match_the_moment_route():
    """tr P~ = N^ = sum_k alpha_k mu_k; tr Q~ = sum_k alpha_k [(W/4)(mu_{k+1} + mu_{|k-1|})
    + (c/2) mu_k], from H = (W H^ + c)/2 and H^ C_k = (C_{k+1} + C_{|k-1|})/2."""
    _, _, _, _, H, w, V, emin, emax, mu, T, p, R = _setup()
    Pt, Qt = di.direct_density(w, V, R, emin, emax, mu, T, p)
    mom = ch.exact_moments(w, V, R, emin, emax, p + 1)
    _, _, N = ch.estimator_observables(mom[:p], emin, emax, mu, T)
    assert np.trace(Pt) == pytest.approx(N, rel=1e-12)
    af, _, _ = ch.fd_coefficients(p, emin, emax, mu, T)
    W, c = emax - emin, emax + emin
    k = np.arange(p)
    trQ = np.sum(af * (W / 4 * (mom[k + 1] + mom[np.abs(k - 1)]) + c / 2 * mom[k]))
    assert np.trace(Qt) == pytest.approx(trQ, rel=1e-11)


def test_mean_and_elementwise_variance_over_every_sign_vector():
    rng = np.random.default_rng(31)
    n = 10
    B = rng.normal(size=(n, n))
    H = B + B.T
    w, V = np.linalg.eigh(H)
    emin, emax, mu, T, p = w.min() - 0.2, w.max() + 0.2, 0.3, 0.6, 40
    signs = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1) * -2.0 + 1.0
    R = signs.T
    Pt, _ = di.direct_density(w, V, R, emin, emax, mu, T, p)
    X = V @ np.diag(di.fermi_polynomial(w, emin, emax, mu, T, p)) @ V.T
    assert np.allclose(Pt, X, atol=1e-12)                   # unbiased
    per = np.einsum("jm,mi,li->ijl", X, R, R)               # X r_i r_i^T for every sign vector
    assert np.allclose(per.var(axis=0), di.direct_density_sigma(X, 1) ** 2, rtol=1e-10, atol=1e-13)
    assert np.allclose(di.direct_density_sigma(X, 25), di.direct_density_sigma(X, 1) / 5, rtol=1e-14)


def test_limit_is_the_exact_density_matrix_and_its_forces():
    """With Hadamard probes and p large for a warm T, M o P~ is M o P to the polynomial error,
    and forces from it (Eq. observable) are the exact Hellmann-Feynman forces."""
    pos, rp, col, Vsk, H = _small_sk(7, jitter=0.08)
    n = H.shape[0]                                           # 63 functions
    Hp = np.zeros((64, 64))
    Hp[:n, :n] = H
    Hp[n, n] = 0.0                                           # one decoupled padding function
    w, V = np.linalg.eigh(Hp)
    emin, emax, T = w.min() - 1.0, w.max() + 1.0, 1.0
    mu = float(np.median(w))
    p = int(np.ceil((emax - emin) / T * np.log(1e12) / 6.4)) + 20
    Pt, _ = di.direct_density(w, V, hadamard(64).astype(float), emin, emax, mu, T, p)
    P = physics.density_matrix(w, V, mu, T)
    M = di.block_mask(rp, col, 9)
    assert np.abs((Pt[:n, :n] - P[:n, :n]) * M).max() < 1e-9
    a, b, dH = hamiltonian.sk_bond_grads(pos, rp, col, Vsk, wl.SK_R0, wl.SK_DECAY)
    F_direct = physics.forces_from_blocks(Pt[:n, :n] * M, a, b, dH, 7, 9)
    F_exact = physics.forces_from_blocks(P[:n, :n], a, b, dH, 7, 9)
    assert np.abs(F_direct - F_exact).max() < 1e-8


def test_forces_see_only_the_symmetric_part():
    """tr(P~ D) = tr(sym(P~) D) for symmetric dH: the nonsymmetric estimate and its symmetric
    part give the same forces."""
    pos, rp, col, Vsk, H, w, V, emin, emax, mu, T, p, R = _setup()
    Pt, _ = di.direct_density(w, V, R, emin, emax, mu, T, p)
    M = di.block_mask(rp, col, 9)
    a, b, dH = hamiltonian.sk_bond_grads(pos, rp, col, Vsk, wl.SK_R0, wl.SK_DECAY)
    F1 = physics.forces_from_blocks(Pt * M, a, b, dH, 13, 9)
    F2 = physics.forces_from_blocks(0.5 * (Pt + Pt.T) * M, a, b, dH, 13, 9)
    assert np.allclose(F1, F2, rtol=1e-12, atol=1e-12)


def test_block_mask_of_a_chain_by_hand():
    pos = np.zeros((3, 3))
    pos[:, 0] = [0.0, 2.5, 5.0]
    rp, col = neighbors.neighbor_csr(pos, 2.5)              # each atom, itself and the next ones
    M = di.block_mask(rp, col, 2)
    A = np.array([[1, 1, 0], [1, 1, 1], [0, 1, 1]], dtype=bool)
    ref = np.repeat(np.repeat(A, 2, axis=0), 2, axis=1)
    assert np.array_equal(M, ref)
    assert M.sum() == len(col) * 4
