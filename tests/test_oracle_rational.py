"""Pins for the oracle's rational approximation of the Fermi function and its CGLS solves
(Sec. II.B.2, Eq. rational_fit, Eq. rational_PQ with S = I; CPU only).

The continued-fraction poles and residues are checked against the Fermi function itself
(exponential convergence in the number of pole pairs), its symmetry f(mu) = 1, and the
Matsubara frequencies (2n + 1) pi that its first poles approach; CGLS against a dense solve; the
pole-by-pole application of Eq. rational_PQ against the eigen route; the rational estimate of
the density matrix against the exact one as the poles converge.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import chebyshev as ch, direct as di, hamiltonian, neighbors, physics
from oracle import rational as ra


def test_continued_fraction_reproduces_the_fermi_function():
    x = np.linspace(-30.0, 30.0, 2001)
    exact = 1.0 / (1.0 + np.exp(x))
    errs = []
    for n in (3, 6, 9, 12):
        z, R = ra.cfe_poles(n)
        approx = 0.5 + np.real((R[None, :] * (1 / (x[:, None] - 1j * z) + 1 / (x[:, None] + 1j * z))).sum(1))
        errs.append(np.abs(approx - exact).max())
    assert errs[-1] < 1e-12
    # exponential: every 3 more pairs gain more than two orders of magnitude until rounding
    assert all(e1 < 1e-2 * e0 for e0, e1 in zip(errs[:-1], errs[1:-1]))


def test_poles_residues_and_symmetry():
    z, R = ra.cfe_poles(20)
    assert np.all(z > 0) and np.all(np.diff(z) > 0) and np.all(R < 0)
    # the first poles approach the Matsubara frequencies (2n + 1) pi of 1/(1 + e^u)
    assert np.allclose(z[:4], (2 * np.arange(4) + 1) * np.pi, rtol=1e-10)
    # and their residues the Matsubara residue -1 of 1/(1 + e^u) at u = i (2n+1) pi
    assert np.allclose(R[:4], -1.0, rtol=1e-8)
    mu, T = 1.3, 0.07
    assert ra.fermi_rational(np.array([mu]), mu, T, 20)[0] == pytest.approx(1.0, abs=1e-14)
    # f(mu + d) + f(mu - d) = 2 (particle-hole symmetry of the Fermi function)
    d = np.linspace(0.01, 2.0, 50)
    fp = ra.fermi_rational(mu + d, mu, T, 20)
    fm = ra.fermi_rational(mu - d, mu, T, 20)
    assert np.allclose(fp + fm, 2.0, atol=1e-13)
    assert np.allclose(fp, physics.fermi(mu + d, mu, T), atol=1e-12)


def test_cgls_solves_a_complex_shifted_system():
    rng = np.random.default_rng(3)
    A0 = rng.standard_normal((40, 40))
    H = A0 + A0.T
    z = 0.3 + 0.2j
    b = rng.standard_normal((40, 3)).astype(np.complex128)
    x, res, it = ra.cgls(lambda v: H @ v - z * v, lambda v: H @ v - np.conj(z) * v, b, tol=1e-13)
    ref = np.linalg.solve(H - z * np.eye(40), b)
    assert np.all(res < 1e-12) and it <= 400
    assert np.abs(x - ref).max() < 1e-9 * np.abs(ref).max()
    # a warm start at the solution needs no iteration
    _, _, it0 = ra.cgls(lambda v: H @ v - z * v, lambda v: H @ v - np.conj(z) * v, b, x0=ref, tol=1e-9)
    assert it0 == 0


def _small_sk(n=13, jitter=0.05):
    V = wl.sk_integrals(5264)
    pos = wl.fcc_sphere(n, jitter=jitter, seed=2)
    rp, col = neighbors.neighbor_csr(pos, wl.SK_CUTOFF)
    H = hamiltonian.dense_sk(pos, rp, col, V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)
    return rp, col, H


def test_pole_by_pole_cgls_equals_the_eigen_route():
    rp, col, H = _small_sk()
    w, V = np.linalg.eigh(H)
    mu, T, n_pairs = float(np.median(w)), 0.4, 16
    R = ch.probes(H.shape[0], 6, 5)
    X = ra.rational_apply(H, R, mu, T, n_pairs, tol=1e-13)
    Pt, Qt = ra.rational_density(w, V, R, mu, T, n_pairs)
    s = R.shape[1]
    assert np.allclose(X @ R.T / s, Pt, atol=1e-10 * np.abs(Pt).max())
    assert np.allclose(H @ X @ R.T / s, Qt, atol=1e-10 * np.abs(Qt).max())


def test_rational_estimate_converges_to_the_exact_probe_estimate():
    """With enough pole pairs, f_r(H) R R^T / s is the probe estimate of the exact P (the same
    probes through f itself): the error falls with the pairs and the trace gives N."""
    rp, col, H = _small_sk()
    w, V = np.linalg.eigh(H)
    mu, T = float(np.median(w)), 0.3
    R = ch.probes(H.shape[0], 8, 11)
    X_exact = V @ (physics.fermi(w, mu, T)[:, None] * (V.T @ R))
    P_exact = X_exact @ R.T / 8
    errs = [np.abs(ra.rational_density(w, V, R, mu, T, n)[0] - P_exact).max() for n in (6, 12, 24)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-10
    Pt = ra.rational_density(w, V, R, mu, T, 24)[0]
    assert np.trace(Pt) == pytest.approx(np.trace(P_exact), rel=1e-12)
    # a wrong sign of the residues, or residues without the factor T, break the match (planted
    # mistakes); conjugating the poles does not, since the residues are real
    zeta, wts = ra.fermi_poles(mu, T, 24)
    bad = 1.0 + 2.0 * np.real((-wts[None, :] / (w[:, None] - zeta[None, :])).sum(1))
    assert np.abs(bad - physics.fermi(w, mu, T)).max() > 0.5
    bad2 = 1.0 + 2.0 * np.real((wts[None, :] / T / (w[:, None] - zeta[None, :])).sum(1))
    assert np.abs(bad2 - physics.fermi(w, mu, T)).max() > 0.5
    assert np.all(np.abs(np.imag(wts)) == 0)
