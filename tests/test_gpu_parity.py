"""Parity of the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (stated per test): neighbour pattern bit-exact; FP64-mode energies within 1e-6
eV/atom of the oracle's exact value of the same estimator, mixed mode within 1e-4 eV/atom;
forces within 1e-3 eV/A (mixed) and 1e-6 eV/A (FP64).
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import chebyshev as och
from oracle import neighbors as onb

from gpu_common import (blocks_of, oracle_H, oracle_estimator, oracle_estimator_forces,
                        small_fcc)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1812_05264_gb300 import build
    build.build()
    from paper_1812_05264_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context()
    yield c
    c.close()           # give the device memory back before the next module


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


# ---- a1 neighbour list: bit-exact ---------------------------------------------------------

@pytest.mark.parametrize("case", ["fcc1000", "fcc_jitter", "sc_open", "sc_periodic", "edge", "dense"])
def test_neighbors_bit_exact(api, ctx, case):
    box = None
    if case == "fcc1000":
        pos, rc = wl.fcc_sphere(1000), 4.0
    elif case == "dense":
        # more pairs per atom than the binding's first column capacity: counted, then rebuilt
        pos, rc = wl.fcc_sphere(60, jitter=0.05, seed=9), 12.0
    elif case == "fcc_jitter":
        pos, rc = wl.fcc_sphere(700, jitter=0.05, seed=3), 4.0
    elif case == "sc_open":
        pos, rc = wl.sc_cluster(10), 1.0
    elif case == "sc_periodic":
        pos, box = wl.sc_lattice(7)
        rc = 1.5
    else:
        # points at exactly the cutoff, one ulp inside and outside, coincident points
        rc = 1.0
        pos = np.array([[0, 0, 0], [1, 0, 0], [0, 1.0000000000000002, 0], [0, 0, 0.9999999999999999],
                        [0, 0, 0], [3, 3, 3], [3.6, 3, 3]], float)
    rp, col = onb.neighbor_csr(pos, rc, box)
    g = api.build_neighbors(ctx, _dev(pos), rc, box)
    assert g.nnzb == len(col)
    assert np.array_equal(g.row_ptr.cpu().numpy(), rp.astype(np.int32))
    assert np.array_equal(g.col.cpu().numpy(), col)


def test_neighbors_single_atom_and_empty(api, ctx):
    g = api.build_neighbors(ctx, _dev(np.zeros((1, 3))), 2.0)
    assert g.nnzb == 1 and g.col.cpu().tolist() == [0]
    g0 = api.build_neighbors(ctx, torch.zeros((0, 3), dtype=torch.float64, device="cuda"), 2.0)
    assert g0.nnzb == 0


@pytest.mark.parametrize("case", ["fcc500_r6", "sc_periodic_r2"])
def test_atom_colours_equal_the_oracle(api, ctx, case):
    """Multi-colour ensemble preprocessing (Sec. II.E): the device neighbour list at the colouring
    radius, coloured by the library's Welsh-Powell pass, colour for colour the oracle's."""
    from oracle import coloring as oco
    box = None
    if case == "fcc500_r6":
        pos, r = wl.fcc_sphere(500, jitter=0.05, seed=5), 6.0
    else:
        pos, box = wl.sc_lattice(8)
        r = 2.0
    c, q = api.atom_colors(ctx, _dev(pos), r, box)
    ref = oco.atom_colors(pos, r, box)
    assert np.array_equal(c, ref) and q == int(ref.max()) + 1


# ---- a2 assembly ----------------------------------------------------------------------------

def test_assemble_sk_matches_oracle(api, ctx):
    wk = small_fcc(60, jitter=0.08)
    rp, col, H = oracle_H(wk)
    s = api.Solver(wk, ctx)
    g = api.build_neighbors(ctx, _dev(wk.positions), wk.cutoff)
    Hg = api.assemble_H(ctx, s.model, _dev(wk.positions), g)
    ref = blocks_of(H, rp, col, 9)
    assert np.allclose(Hg.val.cpu().numpy(), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("which", ["sc1", "lattice9"])
def test_assemble_table_matches_oracle(api, ctx, which):
    wk = wl.sc_disorder(L=6) if which == "sc1" else wl.sc9_periodic(L=4, n_probes=8)
    rp, col, H = oracle_H(wk)
    s = api.Solver(wk, ctx)
    g = api.build_neighbors(ctx, _dev(wk.positions), wk.cutoff, s.box)
    Hg = api.assemble_H(ctx, s.model, _dev(wk.positions), g, s.box)
    assert np.allclose(Hg.val.cpu().numpy(), blocks_of(H, rp, col, wk.n_orb), rtol=0, atol=1e-14)


# ---- a3 bounds, a4 coefficients ------------------------------------------------------------

@pytest.mark.parametrize("which", ["fcc", "sc1"])
def test_spectral_bounds_enclose_spectrum(api, ctx, which):
    wk = small_fcc(80) if which == "fcc" else wl.sc_disorder(L=8)
    _, _, H = oracle_H(wk)
    w = np.linalg.eigvalsh(H)
    s = api.Solver(wk, ctx)
    g = api.build_neighbors(ctx, _dev(wk.positions), wk.cutoff)
    Hg = api.assemble_H(ctx, s.model, _dev(wk.positions), g)
    emin, emax = api.spectral_bounds(ctx, Hg, steps=64, margin=0.01)
    assert emin < w.min() and emax > w.max()
    assert (emax - emin) < 1.1 * (w.max() - w.min())


@pytest.mark.parametrize("fn", [0, 1, 2])
@pytest.mark.parametrize("jackson", [False, True])
def test_coefficients_match_oracle(api, ctx, fn, jackson):
    p, emin, emax, mu, T = 300, -12.0, 25.0, 3.3, 0.2
    c = api.chebyshev_coefficients(ctx, fn, p, emin, emax, mu, T, jackson).cpu().numpy()
    af, aef, bg = och.fd_coefficients(p, emin, emax, mu, T)
    ref = [af, aef, bg][fn] * och.damping(p, jackson)
    assert np.allclose(c, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))


# ---- a5-a8 moments and observables ----------------------------------------------------------

def _gpu_run(api, ctx, wk, p, fp64, direct=False, bounds=None):
    s = api.Solver(wk, ctx)
    pos = _dev(wk.positions)
    res = s.energies(pos, order=p, fp64=fp64, bounds=bounds, direct=direct)
    return s, pos, res


@pytest.mark.parametrize("direct", [False, True])
def test_moments_fp64_match_exact_estimator(api, ctx, direct):
    wk = small_fcc(50, n_probes=16)
    rp, col, H = oracle_H(wk)
    s, pos, res = _gpu_run(api, ctx, wk, 151, fp64=True, direct=direct)
    est = oracle_estimator(wk, H, res.emin, res.emax, 151)
    n = H.shape[0]
    assert np.allclose(res.moments.cpu().numpy(), est["moments"], rtol=0, atol=1e-11 * n)


def test_sc_cluster_energies_fp64(api, ctx):
    """Simple-cubic 10^3 open cluster, 1 orbital, Jackson damping, 32 probes, p = 200."""
    wk = wl.sc_disorder(L=10)
    rp, col, H = oracle_H(wk)
    s, pos, res = _gpu_run(api, ctx, wk, wk.order, fp64=True)
    est = oracle_estimator(wk, H, res.emin, res.emax, wk.order)
    n = wk.n_atoms
    assert np.allclose(res.moments.cpu().numpy(), est["moments"], rtol=0, atol=1e-11 * n)
    assert abs(res.mu - est["mu"]) < 1e-9
    for key in ("Omega", "E", "N"):
        assert abs(getattr(res, key) - est[key]) / n < 1e-6, key


@pytest.mark.parametrize("fp64,tol", [(True, 1e-6), (False, 1e-4)])
def test_fcc_energies_vs_oracle(api, ctx, fp64, tol):
    wk = small_fcc(120, kT=0.5, n_probes=32)
    rp, col, H = oracle_H(wk)
    s, pos, res = _gpu_run(api, ctx, wk, 220, fp64=fp64)
    est = oracle_estimator(wk, H, res.emin, res.emax, 220)
    n = wk.n_atoms
    for key in ("Omega", "E", "N"):
        assert abs(getattr(res, key) - est[key]) / n < tol, key
    assert abs(res.mu - est["mu"]) < 100 * tol


def test_fermi_level_from_oracle_moments(api, ctx):
    """a8 alone: same moments in, same mu / Omega / E / N out (FP64, 1e-10 relative)."""
    wk = small_fcc(40)
    rp, col, H = oracle_H(wk)
    w = np.linalg.eigvalsh(H)
    emin, emax = w.min() - 0.5, w.max() + 0.5
    est = oracle_estimator(wk, H, emin, emax, 180)
    mom = _dev(est["moments"])
    mu, Om, E, N = api.fermi_level(ctx, mom, emin, emax, wk.n_electrons, wk.kT)
    assert mu == pytest.approx(est["mu"], abs=1e-10)
    assert Om == pytest.approx(est["Omega"], rel=1e-10)
    assert E == pytest.approx(est["E"], rel=1e-10)
    assert N == pytest.approx(est["N"], rel=1e-10)
    # fixed chemical potential
    mu0 = est["mu"] + 0.3
    _, Om2, E2, N2 = api.fermi_level(ctx, mom, emin, emax, None, wk.kT, mu=mu0)
    ref = och.estimator_observables(est["moments"], emin, emax, mu0, wk.kT)
    assert np.allclose([Om2, E2, N2], ref, rtol=1e-10)


# ---- a9-a10 density matrix and forces -------------------------------------------------------

@pytest.mark.parametrize("fp64,ftol", [(True, 1e-6), (False, 1e-3)])
def test_density_and_forces_vs_oracle(api, ctx, fp64, ftol):
    wk = small_fcc(30, kT=0.5, n_probes=8)
    p = 120
    rp, col, H = oracle_H(wk)
    s, pos, res = _gpu_run(api, ctx, wk, p, fp64=fp64)
    est = oracle_estimator(wk, H, res.emin, res.emax, p)
    Gd, F = oracle_estimator_forces(wk, rp, col, est, res.emin, res.emax, p)
    # use the oracle's mu so that G and F are compared at the same point
    G, Fg = api.density_and_forces(ctx, res.H, s.model, pos, None, res.emin, res.emax,
                                   wk.probe_seed, wk.n_probes, p, est["mu"], wk.kT, False, fp64)
    Gref = blocks_of(Gd, rp, col, 9)
    gscale = np.abs(Gref).max()
    assert np.abs(G.cpu().numpy() - Gref).max() < (1e-9 if fp64 else 2e-4) * gscale
    assert np.abs(Fg.cpu().numpy() - F).max() < ftol
    assert np.abs(Fg.cpu().numpy().sum(0)).max() < 1e-9


def test_checkpointed_adjoint_equals_stored(api, ctx):
    """Replaying segments from checkpoints gives the same G as keeping every panel."""
    wk = small_fcc(30, n_probes=8)
    p = 90
    s, pos, res = _gpu_run(api, ctx, wk, p, fp64=True)
    args = (ctx, res.H, s.model, pos, None, res.emin, res.emax, wk.probe_seed, wk.n_probes, p,
            res.mu, wk.kT, False, True)
    G1, F1 = api.density_and_forces(*args)
    panel = wk.n_atoms * 9 * wk.n_probes * 8
    G2, F2 = api.density_and_forces(*args, max_panel_bytes=40 * panel)
    assert torch.equal(G1, G2) and torch.equal(F1, F2)


def test_autograd_free_energy(api, ctx):
    wk = small_fcc(25, n_probes=8, order=100)
    s = api.Solver(wk, ctx)
    pos = _dev(wk.positions).requires_grad_(True)
    A = api.FreeEnergy.apply(pos, s)
    A.backward()
    res = s.energies(_dev(wk.positions), order=100)
    r2 = s.forces(_dev(wk.positions), res)
    assert torch.allclose(pos.grad, -r2.forces)


def test_autograd_forces_match_central_finite_differences(api, ctx):
    """Forces from the adjoint kernel through torch.autograd against central differences
    (dx = 1e-4 A) of A^ = Omega^ + mu^ N_e on 8 random atoms.  FP64 recurrence; the spectral
    bounds, probes and order are held fixed, as in the analytic derivative (Sec. II.D).  No pair
    distance of the jittered fcc cluster is near the 4.0 A cutoff (shells at 3.61 and 4.42 A), so
    the pattern does not change under the displacements."""
    wk = small_fcc(60, n_probes=16, order=150, kT=0.5)
    s = api.Solver(wk, ctx)
    pos0 = _dev(wk.positions)
    r0 = s.energies(pos0, fp64=True)
    bounds = (r0.emin - 0.5, r0.emax + 0.5)
    pos = pos0.clone().requires_grad_(True)
    A = api.FreeEnergy.apply(pos, s, bounds)
    A.backward()
    grad = pos.grad.cpu().numpy()
    ne = wk.n_electrons

    def a_hat(p):
        r = s.energies(p, fp64=True, bounds=bounds)
        return r.Omega + r.mu * ne

    rng = np.random.default_rng(1812)
    h = 1e-4
    for a in rng.choice(wk.n_atoms, 8, replace=False):
        for c in range(3):
            pp, pm = pos0.clone(), pos0.clone()
            pp[a, c] += h
            pm[a, c] -= h
            fd = (a_hat(pp) - a_hat(pm)) / (2 * h)
            assert grad[a, c] == pytest.approx(fd, abs=1e-5, rel=1e-5)


# ---- error paths ------------------------------------------------------------------------------

def test_too_narrow_bounds_raise_spectrum_error(api, ctx):
    from paper_1812_05264_gb300._lib import TBK_ERR_SPECTRUM, TbkError
    wk = small_fcc(30)
    s = api.Solver(wk, ctx)
    pos = _dev(wk.positions)
    g = api.build_neighbors(ctx, pos, wk.cutoff)
    H = api.assemble_H(ctx, s.model, pos, g)
    emin, emax = api.spectral_bounds(ctx, H)
    mid, half = 0.5 * (emin + emax), 0.3 * (emax - emin)
    with pytest.raises(TbkError) as e:
        api.chebyshev_moments(ctx, H, mid - half, mid + half, 1, 8, 400, fp64=True)
    assert e.value.code == TBK_ERR_SPECTRUM


def test_argument_errors(api, ctx):
    from paper_1812_05264_gb300._lib import TBK_ERR_ARG, TBK_ERR_NOCONV, TbkError
    wk = small_fcc(20)
    s = api.Solver(wk, ctx)
    pos = _dev(wk.positions)
    g = api.build_neighbors(ctx, pos, wk.cutoff)
    H = api.assemble_H(ctx, s.model, pos, g)
    with pytest.raises(TbkError) as e:
        api.chebyshev_moments(ctx, H, -1.0, 1.0, 1, 6, 10)          # probes not a multiple of 4
    assert e.value.code == TBK_ERR_ARG
    with pytest.raises(TbkError) as e:
        api.chebyshev_moments(ctx, H, 1.0, -1.0, 1, 8, 10)          # emax < emin
    assert e.value.code == TBK_ERR_ARG
    emin, emax = api.spectral_bounds(ctx, H)
    mom = api.chebyshev_moments(ctx, H, emin, emax, 1, 8, 50, fp64=True)
    with pytest.raises(TbkError) as e:
        api.fermi_level(ctx, mom, emin, emax, 1e9, 0.5)               # more electrons than states
    assert e.value.code == TBK_ERR_NOCONV
    # the context stays usable after errors
    mom2 = api.chebyshev_moments(ctx, H, emin, emax, 1, 8, 50, fp64=True)
    assert torch.equal(mom, mom2)


# ---- the TMA-fed step kernel (mixed precision, 9x9 blocks, probes a multiple of 128) ----------

@pytest.mark.parametrize("s", [128, 256, 512, 1024])
def test_tma_step_kernel_matches_plain_kernel_and_oracle(api, ctx, s):
    wk = small_fcc(90, n_probes=s, jitter=0.05)
    rp, col, H = oracle_H(wk)
    sv = api.Solver(wk, ctx)
    pos = _dev(wk.positions)
    g = api.build_neighbors(ctx, pos, wk.cutoff)
    Hg = api.assemble_H(ctx, sv.model, pos, g)
    emin, emax = api.spectral_bounds(ctx, Hg)
    p = 101
    m_tma = api.chebyshev_moments(ctx, Hg, emin, emax, wk.probe_seed, s, p)
    m_plain = api.chebyshev_moments(ctx, Hg, emin, emax, wk.probe_seed, s, p, plain=True)
    n = H.shape[0]
    # same FMA order per element: agreement to rounding of the partial-sum grouping
    assert np.allclose(m_tma.cpu().numpy(), m_plain.cpu().numpy(), rtol=0, atol=1e-9 * n)
    est = oracle_estimator(wk, H, emin, emax, p)
    assert np.abs(m_tma.cpu().numpy() - est["moments"]).max() < 2e-5 * n
    d_tma = api.chebyshev_moments(ctx, Hg, emin, emax, wk.probe_seed, s, p, direct=True)
    assert np.abs(d_tma.cpu().numpy() - est["moments"]).max() < 2e-5 * n


@pytest.mark.parametrize("s", [128, 256, 512])
def test_fused_clenshaw_outer_product_kernel(api, ctx, s):
    """The TMA-fed backward step with the fused y_j b_{j+1}^T term vs the plain kernels and the
    oracle's estimator forces (mixed precision: 1e-3 eV/A)."""
    wk = small_fcc(40, n_probes=s, kT=0.5)
    p = 80
    rp, col, H = oracle_H(wk)
    s_, pos, res = _gpu_run(api, ctx, wk, p, fp64=False)
    est = oracle_estimator(wk, H, res.emin, res.emax, p)
    args = (ctx, res.H, s_.model, pos, None, res.emin, res.emax, wk.probe_seed, wk.n_probes, p,
            est["mu"], wk.kT, False, False)
    G1, F1 = api.density_and_forces(*args)
    G2, F2 = api.density_and_forces(*args, plain=True)
    gmax = G2.abs().max().item()
    assert torch.allclose(G1, G2, rtol=0, atol=2e-5 * gmax)
    assert torch.allclose(F1, F2, rtol=0, atol=1e-4)
    _, F = oracle_estimator_forces(wk, rp, col, est, res.emin, res.emax, p)
    assert np.abs(F1.cpu().numpy() - F).max() < 1e-3


# ---- the tensor-core step (tcgen05, TF32 split three ways) ------------------------------------

@pytest.mark.parametrize("s", [128, 256, 512])
def test_tensor_core_step_matches_fp32_kernels_and_oracle(api, ctx, s):
    wk = small_fcc(90, n_probes=s, jitter=0.05)
    rp, col, H = oracle_H(wk)
    sv = api.Solver(wk, ctx)
    pos = _dev(wk.positions)
    g = api.build_neighbors(ctx, pos, wk.cutoff)
    Hg = api.assemble_H(ctx, sv.model, pos, g)
    emin, emax = api.spectral_bounds(ctx, Hg)
    p = 101
    m_tc = api.chebyshev_moments(ctx, Hg, emin, emax, wk.probe_seed, s, p, tensor_cores=True)
    m_fp32 = api.chebyshev_moments(ctx, Hg, emin, emax, wk.probe_seed, s, p)
    n = H.shape[0]
    est = oracle_estimator(wk, H, emin, emax, p)
    assert np.abs(m_tc.cpu().numpy() - est["moments"]).max() < 2e-5 * n
    assert np.abs(m_tc.cpu().numpy() - m_fp32.cpu().numpy()).max() < 2e-5 * n
    mu, Om, E, N = api.fermi_level(ctx, m_tc, emin, emax, wk.n_electrons, wk.kT)
    assert abs(Om - est["Omega"]) / wk.n_atoms < 1e-4
    assert abs(E - est["E"]) / wk.n_atoms < 1e-4


@pytest.mark.parametrize("s", [128, 512])
def test_doubled_adjoint_checkpoints_and_orders(api, ctx, s):
    """The fused (doubled-moment) adjoint at 128 and 512 probes: segment replays equal storing
    every panel, and odd and even orders (down to p = 2 and 3) match the oracle's estimator G
    (every entry within 2e-5 of max G) and forces."""
    wk = small_fcc(30, n_probes=s, kT=0.5)
    rp, col, H = oracle_H(wk)
    for p in (2, 3, 37, 90):
        s_, pos, res = _gpu_run(api, ctx, wk, p, fp64=False)
        est = oracle_estimator(wk, H, res.emin, res.emax, p)
        args = (ctx, res.H, s_.model, pos, None, res.emin, res.emax, wk.probe_seed, s, p,
                est["mu"], wk.kT, False, False)
        G1, F1 = api.density_and_forces(*args)
        Gd, F = oracle_estimator_forces(wk, rp, col, est, res.emin, res.emax, p)
        Gref = blocks_of(Gd, rp, col, 9)
        assert np.abs(G1.cpu().numpy() - Gref).max() < 2e-5 * np.abs(Gref).max(), p
        assert np.abs(F1.cpu().numpy() - F).max() < 1e-3, p
        if p >= 37:
            # below the p/2 + 8 panels of the all-stored plan, above the checkpoint plan's need
            panel = wk.n_atoms * 9 * s * 4
            G2, F2 = api.density_and_forces(*args, max_panel_bytes=(24 if p == 37 else 30) * panel)
            assert torch.equal(G1, G2) and torch.equal(F1, F2), p


# ---- energies and forces in one call ---------------------------------------------------------

@pytest.mark.parametrize("s,p,fp64,budget", [(128, 90, False, 0), (256, 37, False, 24), (128, 61, True, 0),
                                             (16, 40, False, 0)])
def test_energies_and_forces_one_call_equals_separate_calls(api, ctx, s, p, fp64, budget):
    """The combined entry point takes its moments from the adjoint's own forward sweep (or, for the
    shapes the fused kernels do not take, runs the separate calls): every output is bit-identical
    to moments + Fermi level + density and forces, and matches the oracle."""
    wk = small_fcc(40, n_probes=s, kT=0.5)
    rp, col, H = oracle_H(wk)
    sv, pos, res = _gpu_run(api, ctx, wk, p, fp64=fp64)
    mpb = budget * wk.n_atoms * 9 * s * 4
    sv.forces(pos, res, fp64=fp64, want_G=True, max_panel_bytes=mpb)
    r2 = sv.energies_and_forces(pos, order=p, fp64=fp64, bounds=(res.emin, res.emax), want_G=True,
                                max_panel_bytes=mpb)
    assert torch.equal(res.moments, r2.moments)
    assert (res.mu, res.Omega, res.E, res.N) == (r2.mu, r2.Omega, r2.E, r2.N)
    assert torch.equal(res.G, r2.G) and torch.equal(res.forces, r2.forces)
    est = oracle_estimator(wk, H, res.emin, res.emax, p)
    tol = 1e-6 if fp64 else 1e-4
    assert abs(r2.Omega - est["Omega"]) / wk.n_atoms < tol
    _, F = oracle_estimator_forces(wk, rp, col, est, res.emin, res.emax, p)
    assert np.abs(r2.forces.cpu().numpy() - F).max() < (1e-6 if fp64 else 1e-3)


def test_energies_and_forces_rejects_bad_arguments(api, ctx):
    from paper_1812_05264_gb300._lib import TbkError
    wk = small_fcc(20, n_probes=128)
    sv, pos, res = _gpu_run(api, ctx, wk, 20, fp64=False)
    with pytest.raises(TbkError):
        api.energies_and_forces(ctx, res.H, sv.model, pos, None, res.emin, res.emax, 1, 128, 20,
                                wk.n_electrons, -1.0)
    with pytest.raises(TbkError):  # no Fermi level inside the bounds
        api.energies_and_forces(ctx, res.H, sv.model, pos, None, res.emin, res.emax, 1, 128, 20,
                                1e9, wk.kT)


def test_kernel_timer_counts_the_recurrence_launches(api, ctx):
    wk = small_fcc(40, n_probes=128)
    sv, pos, res = _gpu_run(api, ctx, wk, 30, fp64=False)
    fams = ("step", "backward", "window")
    # K = 15: 15 moment steps + 15 forward steps; fused: 14 adjoint steps and the y_0 outer
    # product; windowed: 14 adjoint steps, windows 1..4 .. 13..14 and y_0
    for windowed, want in ((False, {"step": 30, "backward": 15, "window": 0}),
                           (True, {"step": 30, "backward": 14, "window": 5})):
        ctx.time_kernels(*fams)
        api.chebyshev_moments(ctx, res.H, res.emin, res.emax, wk.probe_seed, 128, 30, False)
        api.density_and_forces(ctx, res.H, sv.model, pos, None, res.emin, res.emax, wk.probe_seed,
                               128, 30, res.mu, wk.kT, False, False, windowed=windowed)
        got = {f: ctx.kernel_time(f) for f in fams}
        ctx.time_kernels()
        assert {f: n for f, (ms, n) in got.items()} == want, got
        assert all(ms > 0.0 for ms, n in got.values() if n > 0)


@pytest.mark.parametrize("s,p", [(128, 61), (512, 40)])
def test_windowed_outer_products_match_fused(api, ctx, s, p):
    """The outer products summed over windows of steps by their own kernel give the fused kernel's
    G up to FP32 summation order; replaying segments does not change a bit."""
    wk = small_fcc(36, n_probes=s, kT=0.5)
    rp, col, H = oracle_H(wk)
    sv, pos, res = _gpu_run(api, ctx, wk, p, fp64=False)
    args = (ctx, res.H, sv.model, pos, None, res.emin, res.emax, wk.probe_seed, s, p, res.mu,
            wk.kT, False, False)
    G1, F1 = api.density_and_forces(*args)
    G2, F2 = api.density_and_forces(*args, windowed=True)
    gmax = G1.abs().max().item()
    assert torch.allclose(G1, G2, rtol=0, atol=2e-6 * gmax)
    assert torch.allclose(F1, F2, rtol=0, atol=1e-5)
    panel = wk.n_atoms * 9 * s * 4
    # one panel below the all-stored plan (p/2 + 8 panels): segments are replayed
    G3, F3 = api.density_and_forces(*args, windowed=True, max_panel_bytes=(p // 2 + 7) * panel)
    assert torch.equal(G2, G3) and torch.equal(F2, F3)
    est = oracle_estimator(wk, H, res.emin, res.emax, p)
    _, F = oracle_estimator_forces(wk, rp, col, est, res.emin, res.emax, p)
    assert np.abs(F2.cpu().numpy() - F).max() < 1e-3


@pytest.mark.parametrize("s,fp64,direct", [(16, True, False), (16, True, True), (128, False, False),
                                            (512, False, True), (512, False, False)])
def test_probe_moments_vs_oracle(api, ctx, s, fp64, direct):
    """a7 per probe: r_i^T C_k(H^) r_i for every probe against the oracle's exact values (plain,
    self-fed and TMA-fed steps); the sweep's summed moments equal tbk_chebyshev_moments, the mean
    over the probes equals them to rounding, and a second call repeats every bit."""
    wk = small_fcc(40, n_probes=s)
    rp, col, H = oracle_H(wk)
    sv, pos, res = _gpu_run(api, ctx, wk, 20, fp64=fp64)
    p, n = 61, H.shape[0]
    args = (ctx, res.H, res.emin, res.emax, wk.probe_seed, s, p)
    mom, per = api.chebyshev_probe_moments(*args, fp64=fp64, direct=direct)
    assert per.shape == (p, s)
    assert torch.equal(mom, api.chebyshev_moments(*args, fp64=fp64, direct=direct))
    w, V = np.linalg.eigh(H)
    exact = och.exact_probe_moments(w, V, och.probes(n, s, wk.probe_seed), res.emin, res.emax, p)
    assert np.abs(per.cpu().numpy() - exact).max() < (1e-11 if fp64 else 2e-5) * n
    assert np.allclose(per.mean(dim=1).cpu().numpy(), mom.cpu().numpy(), rtol=0,
                       atol=(1e-12 if fp64 else 1e-6) * n)
    _, again = api.chebyshev_probe_moments(*args, fp64=fp64, direct=direct)
    assert torch.equal(per, again)


def test_row_without_its_diagonal_block_is_rejected(api, ctx):
    """H^ = (2H - (emax + emin) I) / W keeps its shift on the diagonal blocks, so a pattern in which
    an atom's row stores no block at all is refused with TBK_ERR_ARG by every call that maps H
    (the self-fed 128-probe kernels among those that run on it first skip the empty row and stay
    in bounds), and the context then computes as before."""
    from paper_1812_05264_gb300 import _lib as L
    wk = small_fcc(30, n_probes=128, kT=0.5)
    sv, pos, res = _gpu_run(api, ctx, wk, 20, fp64=False)
    p = 41
    m0 = api.chebyshev_moments(ctx, res.H, res.emin, res.emax, wk.probe_seed, 128, p)
    j, g = 7, res.H.graph
    rpc, colc, val = g.row_ptr.cpu().long(), g.col.cpu().long(), res.H.val.cpu()
    rows = torch.repeat_interleave(torch.arange(g.n_atoms), rpc[1:] - rpc[:-1])
    keep = (rows != j) & (colc != j)
    counts = torch.bincount(rows[keep], minlength=g.n_atoms)
    assert counts[j] == 0
    rp2 = torch.cat([torch.zeros(1, dtype=torch.long), counts.cumsum(0)]).int()
    H2 = api.BSR(api.Graph(g.n_atoms, int(keep.sum()), rp2.cuda(), colc[keep].int().cuda()), 9,
                 val[keep].contiguous().cuda())
    e0, e1 = res.emin, res.emax
    calls = [
        lambda: api.chebyshev_moments(ctx, H2, e0, e1, wk.probe_seed, 128, p),
        lambda: api.chebyshev_moments(ctx, H2, e0, e1, wk.probe_seed, 128, p, plain=True),
        lambda: api.density_and_forces(ctx, H2, None, None, None, e0, e1, wk.probe_seed, 128, p,
                                       res.mu, wk.kT, want_forces=False, windowed=True),
        lambda: api.density_and_forces(ctx, H2, None, None, None, e0, e1, wk.probe_seed, 128, p,
                                       res.mu, wk.kT, want_forces=False, windowed=False),
        lambda: api.batched_moments(ctx, [res.H, H2], [e0, e0], [e1, e1], [1, 2], 128, [p, p]),
    ]
    for call in calls:
        with pytest.raises(L.TbkError) as e:
            call()
        assert e.value.code == L.TBK_ERR_ARG and "diagonal" in str(e.value)
    m1 = api.chebyshev_moments(ctx, res.H, res.emin, res.emax, wk.probe_seed, 128, p)
    assert torch.equal(m0, m1)


@pytest.mark.parametrize("s", [128, 512])
def test_bounded_wait_reports_timeout_and_context_recovers(api, ctx, s):
    """A recurrence step whose producer copies nothing (the self-fed single-warp kernel at 128
    probes, the producer-warp kernel with four consumer warps at 512): the consumers' waits give
    up after their wall-time limit, the call returns TBK_ERR_TIMEOUT, nothing faults, and the same
    context then computes the same moments as before."""
    from paper_1812_05264_gb300 import _lib as L
    wk = small_fcc(40, n_probes=s)
    sv, pos, res = _gpu_run(api, ctx, wk, 30, fp64=False)
    args = (ctx, res.H, res.emin, res.emax, wk.probe_seed, s, 30, False)
    m0 = api.chebyshev_moments(*args)
    L.call("tbk_test_stall_next_step", ctx.handle)
    with pytest.raises(L.TbkError) as e:
        api.chebyshev_moments(*args)
    assert e.value.code == L.TBK_ERR_TIMEOUT
    m1 = api.chebyshev_moments(*args)
    assert torch.equal(m0, m1)


def test_autotune_choice_keeps_the_results(api):
    """tbk_autotune times the step's probe chunk and the adjoint's schedule and keeps its choice
    for this operator shape in the context: moments, G and forces stay those of the default
    choice up to FP32 summation order, and within the oracle's tolerances."""
    ctx2 = api.Context()  # a context of its own, so that no other test sees the choice
    wk = small_fcc(60, n_probes=512, kT=0.5)
    rp, col, H = oracle_H(wk)
    sv, pos, res = _gpu_run(api, ctx2, wk, 40, fp64=False)
    args = (ctx2, res.H, sv.model, pos, None, res.emin, res.emax, wk.probe_seed, 512, 40, res.mu, wk.kT,
            False, False)
    m0 = api.chebyshev_moments(ctx2, res.H, res.emin, res.emax, wk.probe_seed, 512, 40, False)
    G0, F0 = api.density_and_forces(*args)
    chunk, sched = api.autotune(ctx2, res.H, res.emin, res.emax, 512)
    assert chunk in (128, 256, 512) and sched in ("fused", "windowed", "tensor")
    m1 = api.chebyshev_moments(ctx2, res.H, res.emin, res.emax, wk.probe_seed, 512, 40, False)
    G1, F1 = api.density_and_forces(*args)
    n = H.shape[0]
    assert torch.allclose(m0, m1, rtol=0, atol=1e-9 * n)
    assert torch.allclose(G0, G1, rtol=0, atol=2e-6 * G0.abs().max().item())
    assert torch.allclose(F0, F1, rtol=0, atol=1e-5)
    est = oracle_estimator(wk, H, res.emin, res.emax, 40)
    _, F = oracle_estimator_forces(wk, rp, col, est, res.emin, res.emax, 40)
    assert np.abs(F1.cpu().numpy() - F).max() < 1e-3
    ctx2.close()


@pytest.mark.parametrize("s", [128, 256, 512])
def test_every_step_kernel_forms_the_same_panels(api, ctx, s):
    """The plain, self-fed (128-probe tasks) and TMA-fed (256/512) FP32 step kernels sum each
    row's blocks in stored order and each block's columns l = 0..8 in order, so they form the
    same y_k to the bit: the per-probe moments, computed from the panels by the same reduction,
    are equal bit for bit (doubled and direct)."""
    wk = small_fcc(60, n_probes=s, jitter=0.05)
    sv, pos, res = _gpu_run(api, ctx, wk, 20, fp64=False)
    args = (ctx, res.H, res.emin, res.emax, wk.probe_seed, s, 57)
    for direct in (False, True):
        _, per = api.chebyshev_probe_moments(*args, direct=direct)
        _, per_plain = api.chebyshev_probe_moments(*args, direct=direct, plain=True)
        assert torch.equal(per, per_plain), direct


def test_fused_adjoint_bounded_wait_reports_timeout_and_context_recovers(api, ctx):
    """The fused adjoint step (producer warp, four consumer warps, 512 probes) whose producer copies
    nothing: its consumers give up after their wall-time limit, the adjoint call returns
    TBK_ERR_TIMEOUT, nothing faults, and the same context then computes the same G and forces."""
    from paper_1812_05264_gb300 import _lib as L
    wk = small_fcc(40, n_probes=512)
    sv, pos, res = _gpu_run(api, ctx, wk, 30, fp64=False)
    args = (ctx, res.H, sv.model, pos, None, res.emin, res.emax, wk.probe_seed, 512, 30, res.mu, wk.kT,
            False, False)
    G0, F0 = api.density_and_forces(*args, windowed="fused")
    L.call("tbk_test_stall_next_adjoint", ctx.handle)
    with pytest.raises(L.TbkError) as e:
        api.density_and_forces(*args, windowed="fused")
    assert e.value.code == L.TBK_ERR_TIMEOUT
    G1, F1 = api.density_and_forces(*args, windowed="fused")
    assert torch.equal(G0, G1) and torch.equal(F0, F1)


@pytest.mark.parametrize("s", [128, 512])
def test_isolated_atoms_and_separate_clusters(api, ctx, s):
    """Degenerate rows: atoms with no neighbour (their rows store only the diagonal block) and two
    clusters far apart in one operator, through the TMA-fed step (single-warp kernel at 128 probes,
    producer-warp kernel at 512) and the fused adjoint step, against the oracle's estimator:
    moments within 2e-5 n, every G entry within 2e-5 of max G, forces within 1e-3 eV/A."""
    wk = small_fcc(24, n_probes=s, kT=0.5)
    far = wl.fcc_sphere(13, jitter=0.05, seed=3) + np.array([40.0, 0.0, 0.0])
    iso = np.array([[0.0, 40.0, 0.0], [0.0, 0.0, 40.0], [-40.0, 0.0, 0.0]])
    wk.positions = np.vstack([wk.positions, far, iso])
    wk.n_electrons = 11.0 * wk.n_atoms
    p = 60
    rp, col, H = oracle_H(wk)
    assert np.diff(rp).min() == 1 and np.diff(rp)[-3:].max() == 1
    sv, pos, res = _gpu_run(api, ctx, wk, p, fp64=False)
    est = oracle_estimator(wk, H, res.emin, res.emax, p)
    n = H.shape[0]
    assert np.abs(res.moments.cpu().numpy() - est["moments"]).max() < 2e-5 * n
    Gd, Fo = oracle_estimator_forces(wk, rp, col, est, res.emin, res.emax, p)
    G, F = api.density_and_forces(ctx, res.H, sv.model, pos, None, res.emin, res.emax, wk.probe_seed, s, p,
                                  est["mu"], wk.kT, False, False, windowed="fused")
    Gref = blocks_of(Gd, rp, col, 9)
    assert np.abs(G.cpu().numpy() - Gref).max() < 2e-5 * np.abs(Gref).max()
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-3
    # an isolated atom feels no force
    assert np.abs(F.cpu().numpy()[-3:]).max() < 1e-9


@pytest.mark.parametrize("s,sched", [(128, "fused"), (512, "fused"), (512, "windowed")])
def test_jackson_damping_through_the_benchmarked_kernels(api, ctx, s, sched):
    """Jackson-damped coefficients through the mixed one-call path (TMA-fed step, doubled moments,
    fused or windowed adjoint): mu, Omega, E, N within 1e-4 eV/atom, every G entry within 2e-5 of
    max G and forces within 1e-3 eV/A of the oracle's damped estimator."""
    wk = small_fcc(30, n_probes=s, kT=0.5)
    wk.jackson = True
    p = 90
    rp, col, H = oracle_H(wk)
    sv, pos, res = _gpu_run(api, ctx, wk, 20, fp64=False)
    mom, obs, G, F = api.energies_and_forces(ctx, res.H, sv.model, pos, None, res.emin, res.emax, wk.probe_seed,
                                             s, p, wk.n_electrons, wk.kT, True, False, want_G=True,
                                             windowed=sched)
    est = oracle_estimator(wk, H, res.emin, res.emax, p)
    n = wk.n_atoms
    mu, Om, E, N = obs
    assert abs(mu - est["mu"]) < 1e-4
    for got, key in ((Om, "Omega"), (E, "E"), (N, "N")):
        assert abs(got - est[key]) / n < 1e-4, key
    Gd, Fo = oracle_estimator_forces(wk, rp, col, dict(est, mu=mu), res.emin, res.emax, p)
    Gref = blocks_of(Gd, rp, col, 9)
    assert np.abs(G.cpu().numpy() - Gref).max() < 2e-5 * np.abs(Gref).max()
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-3
