"""Pins for the oracle's exact finite-temperature physics (CPU only)."""
import numpy as np
import pytest

import workloads as wl
from oracle import hamiltonian, neighbors, physics

V = wl.sk_integrals(5264)


def _sk_cluster(n=13, jitter=0.05, seed=3):
    pos = wl.fcc_sphere(n, jitter=jitter, seed=seed)
    rp, col = neighbors.neighbor_csr(pos, wl.SK_CUTOFF)
    return pos, rp, col


def _H(pos, rp, col):
    return hamiltonian.dense_sk(pos, rp, col, V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)


def test_fermi_and_g_relations():
    e = np.linspace(-30, 30, 2001)
    mu, T = 0.3, 0.7
    f = physics.fermi(e, mu, T)
    g = physics.free_energy_fn(e, mu, T)
    assert np.all((f >= 0) & (f <= 2))
    assert f[e < mu - 40 * T].min() == pytest.approx(2.0)
    # f = g' (central differences)
    h = 1e-5
    fd = (physics.free_energy_fn(e + h, mu, T) - physics.free_energy_fn(e - h, mu, T)) / (2 * h)
    assert np.allclose(fd, f, atol=1e-8)
    # g -> 2 (eps - mu) far below mu, -> 0 far above
    assert g[0] == pytest.approx(2 * (e[0] - mu))
    assert abs(g[-1]) < 1e-15


def test_trace_P_equals_electron_count():
    pos, rp, col = _sk_cluster()
    w, Vv = physics.eigh(_H(pos, rp, col))
    ne = 11.0 * pos.shape[0]
    mu = physics.chemical_potential(w, ne, 0.5)
    P = physics.density_matrix(w, Vv, mu, 0.5)
    assert np.trace(P) == pytest.approx(ne, abs=1e-9)


def test_idempotency_at_low_temperature():
    """(P/2)^2 -> P/2 as T -> 0 when the chemical potential sits in a gap (spin factor 2)."""
    rng = np.random.default_rng(0)
    A = rng.normal(size=(12, 12))
    H = A + A.T
    w, Vv = physics.eigh(H)
    mu = 0.5 * (w[5] + w[6])
    for T, tol in [(0.5, None), (0.01, 1e-10)]:
        P = physics.density_matrix(w, Vv, mu, T)
        err = np.abs((P / 2) @ (P / 2) - P / 2).max()
        if tol is not None:
            assert err < tol
    assert np.trace(physics.density_matrix(w, Vv, mu, 0.01)) == pytest.approx(12.0, abs=1e-10)


def test_thermodynamic_identities():
    pos, rp, col = _sk_cluster()
    w, _ = physics.eigh(_H(pos, rp, col))
    T = 0.5
    mu = physics.chemical_potential(w, 11.0 * pos.shape[0], T)
    Om, E, N = physics.observables(w, mu, T)
    h = 1e-5
    dOm_dmu = (physics.observables(w, mu + h, T)[0] - physics.observables(w, mu - h, T)[0]) / (2 * h)
    assert -dOm_dmu == pytest.approx(N, rel=1e-8)
    # Omega = E - mu N - T S with S the spin-degenerate Fermi-Dirac entropy
    ft = physics.fermi(w, mu, T) / 2
    ft = np.clip(ft, 1e-300, 1 - 1e-16)
    S = -2 * np.sum(ft * np.log(ft) + (1 - ft) * np.log1p(-ft))
    assert Om == pytest.approx(E - mu * N - T * S, rel=1e-10, abs=1e-9)
    dOm_dT = (physics.observables(w, mu, T + h)[0] - physics.observables(w, mu, T - h)[0]) / (2 * h)
    assert -dOm_dT == pytest.approx(S, rel=1e-6)


def test_single_atom_and_dimer():
    pos = np.zeros((1, 3))
    rp, col = neighbors.neighbor_csr(pos, 4.0)
    w = np.linalg.eigvalsh(_H(pos, rp, col))
    assert np.allclose(w, sorted([5, 10, 10, 10, 0, 0, 0, 0, 0]))
    # dimer along z: the pi and delta channels decouple into 2x2 problems with closed forms
    r = 2.55
    pos = np.array([[0, 0, 0], [0, 0, r]], float)
    rp, col = neighbors.neighbor_csr(pos, 4.0)
    w = np.sort(np.linalg.eigvalsh(_H(pos, rp, col)))
    ddd = V[9]
    # the delta channel (dxy, dx2-y2 on both atoms) is two decoupled 2x2 problems ed +- dd_delta
    expect = [0 + ddd, 0 - ddd, 0 + ddd, 0 - ddd]
    sub = w.copy()
    for v in expect:
        k = np.argmin(np.abs(sub - v))
        assert abs(sub[k] - v) < 1e-12
        sub = np.delete(sub, k)


def _omega_fixed_mu(pos, rp, col, mu, T):
    w = np.linalg.eigvalsh(_H(pos, rp, col))
    return physics.observables(w, mu, T)[0]


def test_forces_sum_torque_and_finite_differences():
    pos, rp, col = _sk_cluster(n=13)
    T = 0.5
    w, Vv = physics.eigh(_H(pos, rp, col))
    ne = 11.0 * pos.shape[0]
    mu = physics.chemical_potential(w, ne, T)
    P = physics.density_matrix(w, Vv, mu, T)
    a, b, dH = hamiltonian.sk_bond_grads(pos, rp, col, V, wl.SK_R0, wl.SK_DECAY)
    F = physics.forces_from_blocks(P, a, b, dH, pos.shape[0], 9)
    assert np.abs(F.sum(0)).max() < 1e-10                     # translation invariance
    assert np.abs(np.cross(pos, F).sum(0)).max() < 1e-9       # rotation invariance (open cluster)
    h = 1e-4
    for atom, c in [(0, 0), (3, 2), (7, 1)]:
        pp, pm = pos.copy(), pos.copy()
        pp[atom, c] += h
        pm[atom, c] -= h
        fd = -(_omega_fixed_mu(pp, rp, col, mu, T) - _omega_fixed_mu(pm, rp, col, mu, T)) / (2 * h)
        assert F[atom, c] == pytest.approx(fd, abs=1e-6)
        # and the Helmholtz free energy A = Omega + mu N at fixed electron count
        def A(p_):
            ww = np.linalg.eigvalsh(_H(p_, rp, col))
            m_ = physics.chemical_potential(ww, ne, T)
            om, _, n_ = physics.observables(ww, m_, T)
            return om + m_ * n_
        fdA = -(A(pp) - A(pm)) / (2 * h)
        assert F[atom, c] == pytest.approx(fdA, abs=1e-6)
