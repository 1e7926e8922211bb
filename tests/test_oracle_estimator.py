"""Pins for the oracle's Chebyshev coefficients and the exact random-probe estimator (CPU only)."""
import os

import numpy as np
import pytest
from scipy.linalg import hadamard

import workloads as wl
from oracle import bloch, chebyshev as ch, hamiltonian, neighbors, physics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    st = np.uint64(1234567)
    out = []
    with np.errstate(over="ignore"):
        for _ in range(5):
            st = st + np.uint64(0x9E3779B97F4A7C15)
            out.append(int(ch.splitmix64(np.array([st]))[0]))
    assert out == vals


def test_probes_are_rademacher_and_balanced():
    R = ch.probes(4096, 64, 7)
    assert set(np.unique(R)) == {-1.0, 1.0}
    assert abs(R.mean()) < 4 / np.sqrt(R.size)
    # prefix property: fewer probes are the first columns of more probes
    assert np.array_equal(ch.probes(100, 8, 7), R[:100, :8])
    # (1/s) R^T R ~ I
    G = R.T @ R / 4096
    assert np.abs(G - np.eye(64)).max() < 6 / np.sqrt(4096)
    # single columns of a large block come from the same counters
    assert np.array_equal(ch.probe_columns(4096, [0, 37, 63], 7), R[:, [0, 37, 63]])


@pytest.mark.parametrize("m", [0, 1, 5, 17])
def test_coefficients_of_a_chebyshev_polynomial(m):
    p = 32
    M = ch.n_nodes(p)
    t, x = ch.nodes(M)
    a = ch.coefficients(np.cos(m * t), p)
    e = np.zeros(p)
    e[m] = 1.0
    assert np.allclose(a, e, atol=1e-14)


def test_dct_equals_direct_sum_and_node_count_converges():
    p = 40
    M = ch.n_nodes(p)
    _, x = ch.nodes(M)
    f = physics.fermi(ch.energy_at(x, -3.0, 5.0), 0.4, 0.3)
    assert np.allclose(ch.coefficients(f, p), ch.coefficients_direct(f, p), atol=1e-14)
    _, x2 = ch.nodes(2 * M)
    f2 = physics.fermi(ch.energy_at(x2, -3.0, 5.0), 0.4, 0.3)
    assert np.allclose(ch.coefficients(f, p), ch.coefficients(f2, p), atol=1e-14)


def test_expansion_error_follows_the_paper_model():
    """max |f^ - sum alpha_k C_k| falls like exp(-6.4 p T / W) (Sec. II.B.1), within a factor."""
    emin, emax, T, mu = -10.0, 10.0, 0.5, 0.3
    xs = np.linspace(-1, 1, 4001)
    for p in (100, 200):
        af, _, _ = ch.fd_coefficients(p, emin, emax, mu, T)
        err = np.abs(ch.poly_values(af, xs) - physics.fermi(ch.energy_at(xs, emin, emax), mu, T)).max()
        model = np.exp(-6.4 * p * T / (emax - emin))
        assert model / 30 < err < model * 30


def test_jackson_factors():
    p = 50
    g = ch.jackson(p)
    assert g[0] == pytest.approx(1.0)
    assert np.all(np.diff(g) < 0) and g[-1] > 0
    # damped expansion of a positive (step-like) function stays positive
    af, _, _ = ch.fd_coefficients(p, -1.0, 1.0, 0.0, 0.01)
    vals = ch.poly_values(g * af, np.linspace(-1, 1, 2001))
    assert vals.min() > -1e-12
    # a constant is reproduced exactly
    M = ch.n_nodes(p)
    a = ch.coefficients(np.full(M, 3.0), p)
    assert np.allclose(ch.poly_values(g * a, np.linspace(-1, 1, 11)), 3.0)


def _small_sk(n=13, jitter=0.05):
    V = wl.sk_integrals(5264)
    pos = wl.fcc_sphere(n, jitter=jitter, seed=2)
    rp, col = neighbors.neighbor_csr(pos, wl.SK_CUTOFF)
    H = hamiltonian.dense_sk(pos, rp, col, V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)
    return pos, rp, col, V, H


def test_moments_match_dense_matrix_recurrence():
    """Eigen route mu_k = sum_n w_n C_k(x_n) vs the matrix recurrence on H^ itself."""
    _, _, _, _, H = _small_sk()
    w, Vv = np.linalg.eigh(H)
    emin, emax = w.min() - 1.0, w.max() + 1.0
    R = ch.probes(H.shape[0], 8, 11)
    p = 30
    mu = ch.exact_moments(w, Vv, R, emin, emax, p)
    Hh = (2 * H - (emax + emin) * np.eye(H.shape[0])) / (emax - emin)
    Y0, Y1 = R, Hh @ R
    ref = [np.sum(R * Y0) / 8, np.sum(R * Y1) / 8]
    for _ in range(2, p):
        Y0, Y1 = Y1, 2 * Hh @ Y1 - Y0
        ref.append(np.sum(R * Y1) / 8)
    assert np.allclose(mu, ref, rtol=1e-11, atol=1e-9)
    assert mu[0] == pytest.approx(H.shape[0])              # Rademacher: r^T r = n exactly


def test_probe_moments_match_dense_recurrence_per_probe():
    """Each probe's moments from the eigen route against r_i . y_k of the matrix recurrence run on
    that probe alone; their mean is exact_moments and mu_0 is n for every +-1 probe."""
    _, _, _, _, H = _small_sk()
    w, Vv = np.linalg.eigh(H)
    emin, emax = w.min() - 1.0, w.max() + 1.0
    s, p = 6, 25
    R = ch.probes(H.shape[0], s, 23)
    per = ch.exact_probe_moments(w, Vv, R, emin, emax, p)
    assert per.shape == (p, s)
    Hh = (2 * H - (emax + emin) * np.eye(H.shape[0])) / (emax - emin)
    for i in range(s):
        r = R[:, i]
        y0, y1 = r, Hh @ r
        ref = [r @ y0, r @ y1]
        for _ in range(2, p):
            y0, y1 = y1, 2 * Hh @ y1 - y0
            ref.append(r @ y1)
        assert np.allclose(per[:, i], ref, rtol=1e-11, atol=1e-9)
    assert np.all(per[0] == pytest.approx(H.shape[0]))
    assert np.allclose(per.mean(axis=1), ch.exact_moments(w, Vv, R, emin, emax, p), rtol=1e-13, atol=1e-10)


def test_probe_spread_gives_the_hutchinson_error():
    """The standard deviation over probes of the single-probe estimates, / sqrt(s), estimates the
    exact standard error 2 sum_{j!=k} A_jk^2 / s of the trace estimate (Sec. II.C.2)."""
    pos, rp, col, V, H = _small_sk(n=55, jitter=0.0)
    w, Vv = np.linalg.eigh(H)
    T, p, s = 0.5, 300, 2048
    mu = physics.chemical_potential(w, 11.0 * pos.shape[0], T)
    emin, emax = w.min() - 0.5, w.max() + 0.5
    _, _, bg = ch.fd_coefficients(p, emin, emax, mu, T)
    R = ch.probes(H.shape[0], s, 91)
    per = ch.exact_probe_moments(w, Vv, R, emin, emax, p)
    omega_i = bg @ per                       # one estimate per probe
    se = omega_i.std(ddof=1) / np.sqrt(s)
    A = Vv @ np.diag(ch.poly_values(bg, ch.mapped(w, emin, emax))) @ Vv.T
    assert se == pytest.approx(ch.hutchinson_sigma(A, s), rel=0.1)


def test_estimator_exact_for_diagonal_H():
    """Diagonal H: r_j^2 = 1 makes the probe estimate exact for any s."""
    rng = np.random.default_rng(5)
    d = rng.uniform(-2, 3, size=50)
    Vv = np.eye(50)
    R = ch.probes(50, 3, 1)
    emin, emax, T, mu, p = -3.0, 4.0, 0.2, 0.5, 120
    mom = ch.exact_moments(d, Vv, R, emin, emax, p)
    Om, E, N = ch.estimator_observables(mom, emin, emax, mu, T)
    af, aef, bg = ch.fd_coefficients(p, emin, emax, mu, T)
    x = ch.mapped(d, emin, emax)
    assert Om == pytest.approx(ch.poly_values(bg, x).sum(), rel=1e-12)
    assert N == pytest.approx(ch.poly_values(af, x).sum(), rel=1e-12)
    # and p is large enough here that it matches the exact physics closely
    assert N == pytest.approx(physics.fermi(d, mu, T).sum(), abs=1e-6)


def test_estimator_exact_with_hadamard_probes():
    """(1/n) R R^T = I for a Sylvester-Hadamard R: estimator = exact polynomial trace."""
    _, _, _, _, H = _small_sk(n=8)
    H = H[:64, :64]
    w, Vv = np.linalg.eigh(H)
    R = hadamard(64).astype(float)
    emin, emax, p = w.min() - 0.5, w.max() + 0.5, 60
    mom = ch.exact_moments(w, Vv, R, emin, emax, p)
    ref = ch.cheb_T(ch.mapped(w, emin, emax), p).sum(axis=1)
    assert np.allclose(mom, ref, rtol=1e-12, atol=1e-10)


def test_estimator_unbiased_over_all_sign_vectors():
    """Brute force: the average over all 2^n sign vectors equals the exact trace."""
    rng = np.random.default_rng(8)
    A = rng.normal(size=(10, 10))
    H = A + A.T
    w, Vv = np.linalg.eigh(H)
    n = 10
    signs = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1) * -2.0 + 1.0
    R = signs.T
    emin, emax = w.min() - 0.1, w.max() + 0.1
    mom = ch.exact_moments(w, Vv, R, emin, emax, 20)
    ref = ch.cheb_T(ch.mapped(w, emin, emax), 20).sum(axis=1)
    assert np.allclose(mom, ref, rtol=1e-12, atol=1e-10)


def test_divided_difference_identity_behind_the_adjoint():
    """(C_k(x) - C_k(y))/(x - y) = sum_{j<k} (2 - delta_j0) C_j(x) U_{k-1-j}(y): the identity
    that makes the Clenshaw adjoint of Sec. II.D equal to the Daleckii-Krein gradient."""
    rng = np.random.default_rng(2)
    for k in range(1, 12):
        x, y = rng.uniform(-1, 1, 2)
        lhs = (np.cos(k * np.arccos(x)) - np.cos(k * np.arccos(y))) / (x - y)
        ty = np.arccos(y)
        U = lambda m: np.sin((m + 1) * ty) / np.sin(ty)
        rhs = sum((2.0 - (j == 0)) * np.cos(j * np.arccos(x)) * U(k - 1 - j) for j in range(k))
        assert lhs == pytest.approx(rhs, rel=1e-11, abs=1e-11)


def test_divided_differences_close_and_equal_points():
    coef = np.random.default_rng(4).normal(size=40) / np.arange(1, 41)
    x = np.array([0.3, 0.3, 0.3 + 1e-9, -0.8, 0.99999])
    G = ch.divided_differences(coef, x)
    h = 1e-6
    d03 = (ch.poly_values(coef, np.array([0.3 + h])) - ch.poly_values(coef, np.array([0.3 - h]))) / (2 * h)
    assert G[0, 1] == pytest.approx(d03[0], rel=1e-7)
    assert G[0, 2] == pytest.approx(d03[0], rel=1e-7)
    q = ch.poly_values(coef, x)
    assert G[0, 3] == pytest.approx((q[0] - q[3]) / (x[0] - x[3]), rel=1e-12)
    assert np.allclose(G, G.T)


def test_estimator_gradient_matches_finite_differences():
    _, _, _, _, H = _small_sk(n=4)
    n = H.shape[0]
    w, Vv = np.linalg.eigh(H)
    emin, emax, T, p = w.min() - 1.0, w.max() + 1.0, 0.5, 60
    R = ch.probes(n, 5, 3)
    mu = float(np.median(w))
    G = ch.estimator_gradient(w, Vv, R, emin, emax, mu, T, p=p)
    assert np.allclose(G, G.T, atol=1e-12)

    def omega_hat(Hx):
        ww, VV = np.linalg.eigh(Hx)
        return ch.estimator_observables(ch.exact_moments(ww, VV, R, emin, emax, p),
                                        emin, emax, mu, T)[0]
    rng = np.random.default_rng(1)
    for _ in range(3):
        D = rng.normal(size=(n, n))
        D = D + D.T
        h = 1e-5
        fd = (omega_hat(H + h * D) - omega_hat(H - h * D)) / (2 * h)
        assert np.sum(G * D) == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_estimator_forces_match_finite_differences():
    pos, rp, col, V, H = _small_sk(n=6)
    n = H.shape[0]
    w, Vv = np.linalg.eigh(H)
    emin, emax, T, p = w.min() - 2.0, w.max() + 2.0, 0.5, 80
    R = ch.probes(n, 4, 9)
    mu = float(np.median(w))
    G = ch.estimator_gradient(w, Vv, R, emin, emax, mu, T, p=p)
    a, b, dH = hamiltonian.sk_bond_grads(pos, rp, col, V, wl.SK_R0, wl.SK_DECAY)
    F = physics.forces_from_blocks(G, a, b, dH, pos.shape[0], 9)
    assert np.abs(F.sum(0)).max() < 1e-9

    def omega_hat(p_):
        Hx = hamiltonian.dense_sk(p_, rp, col, V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)
        ww, VV = np.linalg.eigh(Hx)
        return ch.estimator_observables(ch.exact_moments(ww, VV, R, emin, emax, p),
                                        emin, emax, mu, T)[0]
    h = 1e-5
    for atom, c in [(0, 0), (2, 1), (5, 2)]:
        pp, pm = pos.copy(), pos.copy()
        pp[atom, c] += h
        pm[atom, c] -= h
        fd = -(omega_hat(pp) - omega_hat(pm)) / (2 * h)
        assert F[atom, c] == pytest.approx(fd, abs=2e-7)


def test_estimator_vs_exact_physics_zscore_and_rate():
    """|O^ - O_exact - bias_poly| <= 4 sigma with sigma from the Hutchinson variance
    (Eq. sampling_error); the error shrinks like s^-1/2."""
    pos, rp, col, V, H = _small_sk(n=55, jitter=0.0)
    w, Vv = np.linalg.eigh(H)
    T = 0.5
    ne = 11.0 * pos.shape[0]
    mu = physics.chemical_potential(w, ne, T)
    emin, emax = w.min() - 0.5, w.max() + 0.5
    p = 300
    af, aef, bg = ch.fd_coefficients(p, emin, emax, mu, T)
    x = ch.mapped(w, emin, emax)
    exact = physics.observables(w, mu, T)
    poly = (ch.poly_values(bg, x).sum(), ch.poly_values(aef, x).sum(), ch.poly_values(af, x).sum())
    mats = [Vv @ np.diag(ch.poly_values(c, x)) @ Vv.T for c in (bg, aef, af)]
    sig_ratio = []
    for s in (32, 128, 512):
        R = ch.probes(H.shape[0], s, 77)
        est = ch.estimator_observables(ch.exact_moments(w, Vv, R, emin, emax, p), emin, emax, mu, T)
        for q in range(3):
            sigma = ch.hutchinson_sigma(mats[q], s)
            bias = poly[q] - exact[q]
            assert abs(est[q] - exact[q] - bias) <= 4 * sigma
        sig_ratio.append(ch.hutchinson_sigma(mats[0], s))
    assert sig_ratio[0] / sig_ratio[2] == pytest.approx(4.0)
    # the polynomial bias itself is tiny at this p
    assert abs(poly[2] - exact[2]) < 1e-6


def test_bloch_oracle_reproduces_real_space():
    """Bloch bands and the probe estimator on a periodic 9-orbital lattice vs dense real space."""
    L = 3
    dirs, h = wl.lattice9_blocks(3)
    pos, box = wl.sc_lattice(L)
    disp = np.concatenate([dirs, -dirs])
    blocks = np.concatenate([h, np.transpose(h, (0, 2, 1))])
    # L = 3 would alias +-d bonds onto one neighbour; check on L = 4 instead
    L = 4
    pos, box = wl.sc_lattice(L)
    rp, col = neighbors.neighbor_csr(pos, 1.5, box)
    H = hamiltonian.dense_table(pos, rp, col, 9, disp, blocks, None, box)
    w = np.linalg.eigvalsh(H)
    wk, U = bloch.bands(L, disp, blocks)
    assert np.allclose(np.sort(wk.ravel()), w, atol=1e-11)
    R = ch.probes(H.shape[0], 3, 5)
    wr, Vr = np.linalg.eigh(H)
    emin, emax = w.min() - 0.1, w.max() + 0.1
    m_real = ch.exact_moments(wr, Vr, R, emin, emax, 12)
    wts = bloch.estimator_weights(L, R, U)
    m_bloch = ch.cheb_T(ch.mapped(wk.ravel(), emin, emax), 12) @ wts.ravel()
    assert np.allclose(m_real, m_bloch, rtol=1e-10, atol=1e-8)


def test_sparse_hamiltonian_equals_the_dense_one():
    pos, rp, col, V, H = _small_sk(n=30, jitter=0.08)
    Hs = hamiltonian.sparse_sk(pos, rp, col, V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)
    assert Hs.blocksize == (9, 9) and Hs.nnz == len(col) * 81
    assert np.array_equal(Hs.toarray(), H)


def test_recurrence_probe_moments_equal_the_eigen_route():
    """The FP64 three-term recurrence on the probes (the route the oracle takes for clusters too
    large to diagonalise) against the eigen route, on sparse and dense H."""
    pos, rp, col, V, H = _small_sk(n=19)
    Hs = hamiltonian.sparse_sk(pos, rp, col, V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)
    w, Vv = np.linalg.eigh(H)
    emin, emax, p = w.min() - 0.7, w.max() + 0.3, 50
    R = ch.probes(H.shape[0], 7, 19)
    ref = ch.exact_probe_moments(w, Vv, R, emin, emax, p)
    for M in (Hs, H):
        got = ch.recurrence_probe_moments(M, R, emin, emax, p)
        assert np.abs(got - ref).max() < 1e-11 * H.shape[0]
    assert np.array_equal(got[0], np.full(7, float(H.shape[0])))     # r^T r = n
    # each probe runs on its own: one column alone gives its moments (to rounding order)
    assert np.allclose(ch.recurrence_probe_moments(Hs, R[:, 2:3], emin, emax, p)[:, 0],
                       ch.recurrence_probe_moments(Hs, R, emin, emax, p)[:, 2],
                       rtol=0, atol=1e-12 * H.shape[0])
