"""Pins for the oracle's neighbour search and the seeded workload geometry (CPU only)."""
import numpy as np
import pytest

import workloads as wl
from oracle import hamiltonian, neighbors


def _sc_expected(L, periodic):
    """Nearest-neighbour pattern of an L^3 simple-cubic lattice from integer index arithmetic."""
    rows = []
    for i in range(L):
        for j in range(L):
            for k in range(L):
                nb = {(i * L + j) * L + k}
                for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    a, b, c = i + d[0], j + d[1], k + d[2]
                    if periodic:
                        a, b, c = a % L, b % L, c % L
                    elif not (0 <= a < L and 0 <= b < L and 0 <= c < L):
                        continue
                    nb.add((a * L + b) * L + c)
                rows.append(sorted(nb))
    return rows


@pytest.mark.parametrize("periodic", [False, True])
def test_sc_pattern_matches_index_arithmetic(periodic):
    L = 5
    pos = wl.sc_cluster(L)
    box = [float(L)] * 3 if periodic else None
    rp, col = neighbors.neighbor_csr(pos, 1.0, box)
    exp = _sc_expected(L, periodic)
    got = [list(col[rp[i]:rp[i + 1]]) for i in range(L ** 3)]
    assert got == exp


def test_sc_periodic_nnn_count():
    L = 4
    pos = wl.sc_cluster(L)
    rp, _ = neighbors.neighbor_csr(pos, 1.5, [4.0] * 3)
    assert np.all(np.diff(rp) == 19)          # self + 6 NN + 12 NNN


def test_fcc_sphere_shells_and_counts():
    pos = wl.fcc_sphere(1000)
    assert pos.shape == (1000, 3)
    assert np.allclose(pos[0], 0.0)
    r = np.sqrt((pos ** 2).sum(1))
    assert np.all(np.diff(r) >= -1e-12)               # sorted by radius
    rp, col = neighbors.neighbor_csr(pos, wl.SK_CUTOFF)
    cnt = np.diff(rp)
    assert cnt[0] == 19 and cnt.max() == 19           # self + 12 (2.553 A) + 6 (3.61 A)
    # symmetric pattern, each row sorted and containing its own index
    pairs = set(zip(np.repeat(np.arange(1000), cnt), col))
    assert all((b, a) in pairs for a, b in pairs)
    for i in range(1000):
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c


def test_fcc_nearest_neighbour_distance():
    pos = wl.fcc_sphere(200)
    d = np.sqrt(((pos[1:] - pos[0]) ** 2).sum(1))
    assert abs(d.min() - wl.FCC_A / np.sqrt(2)) < 1e-12


def test_inclusive_cutoff_and_rounding():
    # r^2 = 1 exactly for unit-spaced integer points: the pair at exactly the cutoff is kept
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0000000000000002, 0.0]])
    rp, col = neighbors.neighbor_csr(pos, 1.0)
    assert list(col[rp[0]:rp[1]]) == [0, 1]


def test_lattice9_blocks_gershgorin_scale():
    dirs, h = wl.lattice9_blocks(7, half_width=5.0)
    rows = sum(np.abs(h[d]).sum(1) + np.abs(h[d].T).sum(1) for d in range(9))
    assert abs(rows.max() - 5.0) < 1e-12


def test_lattice9_workload_has_a_ten_ev_bloch_band():
    """The periodic 9-orbital workload's blocks are scaled by a stored constant to a 10 eV band:
    the Bloch eigenvalues of the scaled model on the 48^3 k-grid span exactly 10 eV, and the
    constant is the unscaled width (the blocks are linear in it)."""
    from oracle import bloch
    wk = wl.sc9_periodic(L=48, n_probes=8)
    w, _ = bloch.bands(48, wk.disp, wk.blocks)
    assert abs((w.max() - w.min()) - 10.0) < 1e-9
    dirs, h1 = wl.lattice9_blocks(4848, scale=1.0)
    _, h10 = wl.lattice9_blocks(4848, band_width=10.0)
    assert np.allclose(h10, h1 * 10.0 / wl.lattice9_width(4848), rtol=1e-15, atol=0)


def test_batched_sizes_in_range():
    spec = wl.batched_clusters(64, 100, 5000, (0.025, 0.1, 0.5), seed=64)
    assert spec.sizes.min() >= 100 and spec.sizes.max() <= 5000
    assert set(np.unique(spec.kTs)) <= {0.025, 0.1, 0.5}
    assert all(p.shape == (n, 3) for p, n in zip(spec.positions, spec.sizes))


def test_morton_order_is_a_permutation_that_keeps_neighbours_close():
    pos = wl.fcc_sphere(2000, seed=1)
    perm = wl.morton_order(pos, wl.FCC_A)
    assert np.array_equal(np.sort(perm), np.arange(2000))
    # the same cluster: the reordered atoms are the original atoms
    a = wl.fcc_cu(2000, kT=0.1, n_probes=8, atom_order="morton").positions
    b = wl.fcc_cu(2000, kT=0.1, n_probes=8).positions
    assert np.array_equal(a[np.lexsort(a.T[::-1])], b[np.lexsort(b.T[::-1])])
    # Z-order keeps bonded atoms closer in index than the radial listing does
    rp, col = neighbors.neighbor_csr(a, 2.6)
    rows = np.repeat(np.arange(2000), np.diff(rp))
    rpb, colb = neighbors.neighbor_csr(b, 2.6)
    rowsb = np.repeat(np.arange(2000), np.diff(rpb))
    assert np.median(np.abs(rows - col)) < np.median(np.abs(rowsb - colb))


def test_lattice9_hermitian_table_gives_a_symmetric_h():
    """h_{-d} = h_d^T: the periodic 9-orbital lattice built from the table is symmetric."""
    wk = wl.sc9_periodic(L=4, n_probes=8)
    rp, col = neighbors.neighbor_csr(wk.positions, wk.cutoff, wk.box)
    H = hamiltonian.dense_table(wk.positions, rp, col, 9, wk.disp, wk.blocks, wk.onsite_site, wk.box)
    assert np.array_equal(H, H.T)
    assert len(col) == 64 * 19                              # 1 + 6 + 12 neighbours per site


def test_batched_clusters_are_log_uniform_with_every_temperature():
    spec = wl.batched_clusters(64, 100, 5000, (0.025, 0.1, 0.5), seed=64)
    lg = np.log(spec.sizes)
    # log-uniform on [log 100, log 5000]: mean 6.21, sd 1.13; 64 draws stay within 4 sigma/8
    assert abs(lg.mean() - 0.5 * (np.log(100) + np.log(5000))) < 4 * 1.13 / 8
    assert set(np.unique(spec.kTs)) == {0.025, 0.1, 0.5}
    assert len(set(spec.seeds.tolist())) == 64
    # the same seed gives the same batch
    again = wl.batched_clusters(64, 100, 5000, (0.025, 0.1, 0.5), seed=64)
    assert np.array_equal(spec.sizes, again.sizes) and np.array_equal(spec.kTs, again.kTs)
    assert all(np.array_equal(p, q) for p, q in zip(spec.positions, again.positions))
