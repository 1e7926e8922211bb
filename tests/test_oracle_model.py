"""Pins for the oracle's Slater-Koster blocks and Hamiltonian assembly (CPU only)."""
import numpy as np
import pytest

import workloads as wl
from oracle import hamiltonian, neighbors, slater_koster as sk

V = np.arange(1.0, 11.0) * np.array([1, -1, 1, 1, -1, 1, -1, 1, -1, 1])   # distinct values
SSS, SPS, SDS, PPS, PPP, PDS, PDP, DDS, DDP, DDD = V
R0, DEC = 2.55, 2.0


def _blk(d):
    return sk.block(np.array([d], float), V, R0, DEC)[0]


def test_bond_along_z_hand_values():
    r = 2.55                                      # radial factor exactly 1
    E = _blk([0, 0, r])
    assert E[0, 0] == pytest.approx(SSS)
    assert E[0, 3] == pytest.approx(SPS) and E[3, 0] == pytest.approx(-SPS)
    assert E[3, 3] == pytest.approx(PPS)
    assert E[1, 1] == pytest.approx(PPP) and E[2, 2] == pytest.approx(PPP)
    assert E[0, 8] == pytest.approx(SDS)
    assert E[3, 8] == pytest.approx(PDS) and E[8, 3] == pytest.approx(-PDS)
    assert E[1, 6] == pytest.approx(PDP) and E[2, 5] == pytest.approx(PDP)
    assert E[8, 8] == pytest.approx(DDS)
    assert E[5, 5] == pytest.approx(DDP) and E[6, 6] == pytest.approx(DDP)
    assert E[4, 4] == pytest.approx(DDD) and E[7, 7] == pytest.approx(DDD)
    # everything else vanishes along z
    mask = np.ones((9, 9), bool)
    for (a, b) in [(0, 0), (0, 3), (3, 0), (3, 3), (1, 1), (2, 2), (0, 8), (8, 0), (3, 8), (8, 3),
                   (1, 6), (6, 1), (2, 5), (5, 2), (8, 8), (5, 5), (6, 6), (4, 4), (7, 7)]:
        mask[a, b] = False
    assert np.abs(E[mask]).max() < 1e-14


def test_bond_along_111():
    r = 2.55
    d = np.array([1.0, 1.0, 1.0]) * r / np.sqrt(3)
    E = _blk(d)
    c = 1 / np.sqrt(3)
    assert E[0, 1] == pytest.approx(c * SPS)
    assert E[1, 1] == pytest.approx(PPS / 3 + 2 * PPP / 3)
    assert E[1, 2] == pytest.approx((PPS - PPP) / 3)
    assert E[0, 4] == pytest.approx(np.sqrt(3) / 3 * SDS)
    assert E[0, 7] == pytest.approx(0.0, abs=1e-14) and E[0, 8] == pytest.approx(0.0, abs=1e-14)
    # dxy-dxy: 3/9 dds + (2/3 - 4/9) ddp + (1/3 + 1/9) ddd
    assert E[4, 4] == pytest.approx(DDS / 3 + 2 * DDP / 9 + 4 * DDD / 9)


def test_radial_factor():
    E1 = _blk([0, 0, 2.55])
    E2 = _blk([0, 0, 3.0])
    assert np.allclose(E2, E1 * np.exp(-2.0 * (3.0 / 2.55 - 1.0)))


def test_reverse_bond_is_transpose():
    rng = np.random.default_rng(0)
    d = rng.normal(size=(20, 3)) * 2
    Ef = sk.block(d, V, R0, DEC)
    Eb = sk.block(-d, V, R0, DEC)
    assert np.allclose(Eb, np.transpose(Ef, (0, 2, 1)), atol=1e-13)


def _orbital_funcs(P):
    x, y, z = P[:, 0], P[:, 1], P[:, 2]
    s3 = np.sqrt(3)
    return np.stack([np.ones_like(x), x, y, z, s3 * x * y, s3 * y * z, s3 * z * x,
                     0.5 * s3 * (x * x - y * y), z * z - 0.5 * (x * x + y * y)], axis=1)


def _rep(Rot):
    """D with phi_i(Rot r) = sum_k D_ik phi_k(r), fitted on random points (exact span)."""
    rng = np.random.default_rng(1)
    P = rng.normal(size=(40, 3))
    A = _orbital_funcs(P)
    B = _orbital_funcs(P @ Rot.T)
    Dt, *_ = np.linalg.lstsq(A, B, rcond=None)
    return Dt.T


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_rotation_covariance(seed):
    """A rotated dimer has the block D H D^T: fails on any sign or index slip in the table."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    D = _rep(Q)
    assert np.allclose(D @ D.T, np.eye(9), atol=1e-10)
    d = rng.normal(size=3) * 2.0
    lhs = _blk(Q @ d)
    rhs = D @ _blk(d) @ D.T
    assert np.allclose(lhs, rhs, atol=1e-11)


def test_complex_step_gradient_matches_fd():
    rng = np.random.default_rng(3)
    d = rng.normal(size=(5, 3)) * 2 + 1
    g = sk.block_grad(d, V, R0, DEC)
    h = 1e-6
    for c in range(3):
        dp, dm = d.copy(), d.copy()
        dp[:, c] += h
        dm[:, c] -= h
        fd = (sk.block(dp, V, R0, DEC) - sk.block(dm, V, R0, DEC)) / (2 * h)
        assert np.allclose(g[:, c], fd, atol=1e-7)


def test_dense_sk_symmetric_and_onsite():
    pos = wl.fcc_sphere(19)
    rp, col = neighbors.neighbor_csr(pos, 4.0)
    H = hamiltonian.dense_sk(pos, rp, col, V, R0, DEC, (5.0, 10.0, 0.0))
    assert np.allclose(H, H.T, atol=1e-13)
    assert np.allclose(np.diag(H)[:9], [5, 10, 10, 10, 0, 0, 0, 0, 0])


def test_dense_table_sc_open_spectrum_closed_form():
    """Open L^3 simple-cubic cluster, hopping t: eps = 2t sum_i cos(pi m_i/(L+1))."""
    L, t = 5, -1.0
    wk = wl.sc_disorder(L=L, t=t, w=0.0)
    rp, col = neighbors.neighbor_csr(wk.positions, wk.cutoff)
    H = hamiltonian.dense_table(wk.positions, rp, col, 1, wk.disp, wk.blocks, None)
    ev = np.linalg.eigvalsh(H)
    c = np.cos(np.pi * np.arange(1, L + 1) / (L + 1))
    ex = np.sort((2 * t * (c[:, None, None] + c[None, :, None] + c[None, None, :])).ravel())
    assert np.allclose(ev, ex, atol=1e-12)


def test_dense_table_sc_periodic_spectrum_closed_form():
    """Periodic L^3 simple-cubic lattice: eps = 2t sum_i cos(2 pi m_i/L)."""
    L, t = 4, -1.0
    pos, box = wl.sc_lattice(L)
    disp = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    rp, col = neighbors.neighbor_csr(pos, 1.0, box)
    H = hamiltonian.dense_table(pos, rp, col, 1, disp, np.full((6, 1, 1), t), None, box)
    ev = np.linalg.eigvalsh(H)
    c = np.cos(2 * np.pi * np.arange(L) / L)
    ex = np.sort((2 * t * (c[:, None, None] + c[None, :, None] + c[None, None, :])).ravel())
    assert np.allclose(ev, ex, atol=1e-12)
