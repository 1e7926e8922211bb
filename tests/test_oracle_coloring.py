"""Pins for the oracle's multi-colour probe ensemble (Sec. II.C.3 and Sec. II.E; CPU only).

The colouring is pinned by colourings worked out by hand, by the first-fit restatement of the
Welsh-Powell procedure, by the Welsh-Powell bound and by brute-force distances; the ensemble by
enumerating every sign vector of a small system (exact mean, deviation matrix and variance), by
the special cases where it reduces to the exact trace or to plain Rademacher probes, and by
finite differences of the coloured estimator."""
import numpy as np
import pytest

import workloads as wl
from oracle import chebyshev as ch, coloring as co, hamiltonian, neighbors


def _chain(n, step):
    pos = np.zeros((n, 3))
    pos[:, 0] = step * np.arange(n)
    return pos


def test_chain_colourings_worked_by_hand():
    # step 2.5 (exact in binary): at r = 2.5 each atom's neighbours are the next ones along the
    # chain (the pair at exactly r is an edge).  Degrees 1,2,2,2,2,1; list 1,2,3,4,0,5.
    # First colour: 1, 3, 5; second: 2, 4, 0.
    pos = _chain(6, 2.5)
    assert co.atom_colors(pos, 2.5).tolist() == [1, 0, 1, 0, 1, 0]
    # just below the spacing there are no edges: one colour
    assert co.atom_colors(pos, 2.4999).tolist() == [0] * 6
    # at r = 5.0 second neighbours join.  Degrees 2,3,4,4,3,2; list 2,3,1,4,0,5.
    # First colour: 2, 5; second: 3, 0; third: 1, 4.
    assert co.atom_colors(pos, 5.0).tolist() == [1, 2, 0, 1, 2, 0]


def test_pentagon_is_an_odd_cycle_with_three_colours():
    t = 2 * np.pi * np.arange(5) / 5
    pos = np.stack([np.cos(t), np.sin(t), np.zeros(5)], axis=1)
    # side 2 sin(pi/5) = 1.18 < 1.5 < diagonal 2 sin(2 pi/5) = 1.90: the graph is a 5-cycle.
    # All degrees 2, list 0..4; first colour 0, 2; second 1, 3; third 4.
    assert co.atom_colors(pos, 1.5).tolist() == [0, 1, 0, 1, 2]
    # above the diagonal every pair is an edge: five colours
    assert sorted(co.atom_colors(pos, 2.0).tolist()) == [0, 1, 2, 3, 4]


@pytest.mark.parametrize("n,r", [(120, 3.0), (200, 6.0), (79, 9.5)])
def test_colouring_is_first_fit_in_degree_order_valid_and_within_the_bound(n, r):
    pos = wl.fcc_sphere(n, jitter=0.05, seed=3)
    rp, col = co.color_graph(pos, r)
    c = co.atom_colors(pos, r)
    # Welsh-Powell gives each listed vertex the smallest colour none of its earlier-listed
    # neighbours has (first-fit greedy in the same order)
    order = co.welsh_powell_order(rp)
    seen = np.zeros(n, bool)
    ff = np.full(n, -1)
    for v in order:
        nb = col[rp[v]:rp[v + 1]]
        used = {int(ff[u]) for u in nb if seen[u]}
        k = 0
        while k in used:
            k += 1
        ff[v] = k
        seen[v] = True
    assert np.array_equal(c, ff)
    # two atoms of one colour are farther apart than r (brute force over all pairs)
    d2 = ((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1)
    same = (c[:, None] == c[None, :]) & ~np.eye(n, dtype=bool)
    assert (d2[same] > r * r).all()
    # the colouring graph is exactly the pairs within r
    A = np.zeros((n, n), bool)
    A[np.repeat(np.arange(n), np.diff(rp)), col] = True
    assert np.array_equal(A, (d2 <= r * r) & ~np.eye(n, dtype=bool))
    # Welsh-Powell bound: q <= max_i min(d_i + 1, i) over the degrees in non-increasing order
    d = np.sort(np.diff(rp))[::-1]
    q = int(c.max()) + 1
    assert q <= max(min(int(d[i]) + 1, i + 1) for i in range(n))
    # each colour class is maximal among the later colours: a vertex of colour k has a
    # neighbour of every colour j < k
    for v in range(n):
        nbc = set(c[col[rp[v]:rp[v + 1]]].tolist())
        assert set(range(c[v])) <= nbc


def test_function_colours():
    fc = co.function_colors(np.array([1, 0, 1]), 9)
    assert fc.tolist() == list(range(9, 18)) + list(range(0, 9)) + list(range(9, 18))


def _three_atom_ensemble():
    # a 3-atom chain coloured [1, 0, 1], three orbitals each: 9 functions, q = 6
    ac = co.atom_colors(_chain(3, 2.5), 2.5)
    assert ac.tolist() == [1, 0, 1]
    fc = co.function_colors(ac, 3)
    n = 9
    signs = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1) * -2.0 + 1.0
    return fc, 6, signs.T          # every sign vector, one sample each


def test_ensemble_mean_and_deviation_over_every_sign_vector():
    fc, q, R = _three_atom_ensemble()
    n, s = R.shape
    Rc = co.colored_probes(fc, q, R)
    assert Rc.shape == (n, s * q)
    # each function is nonzero in exactly one column of a sample, the column of its colour
    nz = Rc.reshape(n, s, q) != 0
    assert (nz.sum(axis=2) == 1).all()
    assert (np.argmax(nz, axis=2) == fc[:, None]).all()
    # mean of R_i R_i^T is I; mean of (R_i R_i^T - I)^2 is E (1 on distinct functions of one
    # colour, 0 elsewhere)
    outer = np.einsum("jiq,kiq->ijk", Rc.reshape(n, s, q), Rc.reshape(n, s, q))
    assert np.array_equal(outer.mean(axis=0), np.eye(n))
    dev = ((outer - np.eye(n)) ** 2).mean(axis=0)
    E = co.deviation_matrix(fc)
    assert np.array_equal(dev, E)
    for j in range(n):
        for k in range(n):
            assert E[j, k] == (1.0 if (fc[j] == fc[k] and j != k) else 0.0)


def test_coloured_estimator_unbiased_with_the_stated_variance():
    fc, q, R = _three_atom_ensemble()
    n, s = R.shape
    rng = np.random.default_rng(12)
    A = rng.normal(size=(n, n))
    A = A + A.T
    Rc = co.colored_probes(fc, q, R).reshape(n, s, q)
    est = np.einsum("jiq,jk,kiq->i", Rc, A, Rc)            # tr(R_i^T A R_i) per sample
    assert est.mean() == pytest.approx(np.trace(A), rel=1e-13)
    assert est.var() == pytest.approx(co.colored_sigma(A, fc, 1) ** 2, rel=1e-12)
    # with s samples the standard error shrinks by sqrt(s)
    assert co.colored_sigma(A, fc, 16) == pytest.approx(co.colored_sigma(A, fc, 1) / 4, rel=1e-15)
    # and the moments through the eigenpairs, over all samples, are the exact traces
    w, V = np.linalg.eigh(A)
    emin, emax = w.min() - 0.1, w.max() + 0.1
    mom = co.exact_colored_moments(w, V, co.colored_probes(fc, q, R), s, emin, emax, 16)
    ref = ch.cheb_T(ch.mapped(w, emin, emax), 16).sum(axis=1)
    assert np.allclose(mom, ref, rtol=1e-12, atol=1e-10)


def _small_sk(n, jitter=0.05):
    V = wl.sk_integrals(5264)
    pos = wl.fcc_sphere(n, jitter=jitter, seed=2)
    rp, col = neighbors.neighbor_csr(pos, wl.SK_CUTOFF)
    return pos, hamiltonian.dense_sk(pos, rp, col, V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)


def test_radius_beyond_the_cluster_gives_the_exact_trace_from_one_sample():
    pos, H = _small_sk(13)
    ac = co.atom_colors(pos, 100.0)
    assert sorted(ac.tolist()) == list(range(13))          # every atom its own colour
    fc = co.function_colors(ac, 9)
    w, V = np.linalg.eigh(H)
    emin, emax, p = w.min() - 1.0, w.max() + 1.0, 40
    Rc = co.colored_probes(fc, 13 * 9, ch.probes(H.shape[0], 1, 77))
    mom = co.exact_colored_moments(w, V, Rc, 1, emin, emax, p)
    ref = ch.cheb_T(ch.mapped(w, emin, emax), p).sum(axis=1)
    assert np.allclose(mom, ref, rtol=1e-12, atol=1e-9)


def test_one_colour_and_one_orbital_is_the_plain_rademacher_ensemble():
    rng = np.random.default_rng(3)
    B = rng.normal(size=(40, 40))
    H = B + B.T
    pos = wl.fcc_sphere(40, seed=1)
    ac = co.atom_colors(pos, 1.0)                          # below the nearest-neighbour distance
    assert (ac == 0).all()
    R = ch.probes(40, 6, 9)
    Rc = co.colored_probes(co.function_colors(ac, 1), 1, R)
    assert np.array_equal(Rc, R)
    w, V = np.linalg.eigh(H)
    emin, emax = w.min() - 0.5, w.max() + 0.5
    assert np.allclose(co.exact_colored_moments(w, V, Rc, 6, emin, emax, 30),
                       ch.exact_moments(w, V, R, emin, emax, 30), rtol=1e-13, atol=1e-12)
    G1 = co.colored_estimator_gradient(w, V, Rc, 6, emin, emax, 0.1, 0.4, 30)
    G2 = ch.estimator_gradient(w, V, R, emin, emax, 0.1, 0.4, p=30)
    assert np.allclose(G1, G2, rtol=1e-13, atol=1e-13)


def test_coloured_estimator_gradient_matches_finite_differences():
    pos, H = _small_sk(6)
    n = H.shape[0]
    fc = co.function_colors(co.atom_colors(pos, wl.FCC_A / np.sqrt(2) * 1.1), 9)
    q = int(fc.max()) + 1
    Rc = co.colored_probes(fc, q, ch.probes(n, 2, 5))
    w, V = np.linalg.eigh(H)
    emin, emax, T, p = w.min() - 1.0, w.max() + 1.0, 0.5, 60
    mu = float(np.median(w))
    G = co.colored_estimator_gradient(w, V, Rc, 2, emin, emax, mu, T, p)
    assert np.allclose(G, G.T, atol=1e-12)

    def omega_hat(Hx):
        ww, VV = np.linalg.eigh(Hx)
        mom = co.exact_colored_moments(ww, VV, Rc, 2, emin, emax, p)
        return ch.estimator_observables(mom, emin, emax, mu, T)[0]
    rng = np.random.default_rng(6)
    for _ in range(3):
        D = rng.normal(size=(n, n))
        D = D + D.T
        h = 1e-5
        fd = (omega_hat(H + h * D) - omega_hat(H - h * D)) / (2 * h)
        assert np.sum(G * D) == pytest.approx(fd, rel=1e-6, abs=1e-8)
