"""Periodic 9-orbital simple-cubic lattice (lattice-table model): energies in mixed and FP64 mode
against the oracle's exact estimator, the sampled density matrix against the Daleckii-Krein
gradient, and the Bloch oracle against exact physics."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import bloch, chebyshev as och, physics

from gpu_common import blocks_of, oracle_H, oracle_estimator

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


@pytest.fixture(scope="module")
def lattice(api, ctx):
    wk = wl.sc9_periodic(L=6, kT=0.05, n_probes=128, order=None)
    rp, col, H = oracle_H(wk)
    s = api.Solver(wk, ctx)
    pos = torch.as_tensor(wk.positions, dtype=torch.float64, device="cuda")
    return wk, rp, col, H, s, pos


@pytest.mark.parametrize("fp64,tol", [(True, 1e-6), (False, 1e-4)])
def test_periodic_energies_vs_oracle(api, ctx, lattice, fp64, tol):
    wk, rp, col, H, s, pos = lattice
    res = s.energies(pos, fp64=fp64)
    est = oracle_estimator(wk, H, res.emin, res.emax, res.order)
    n = wk.n_atoms
    for key in ("Omega", "E", "N"):
        assert abs(getattr(res, key) - est[key]) / n < tol, key
    w = np.linalg.eigvalsh(H)
    assert res.emin < w.min() and res.emax > w.max()


def test_periodic_density_matrix_vs_oracle(api, ctx, lattice):
    wk, rp, col, H, s, pos = lattice
    res = s.energies(pos, order=120, fp64=True)
    est = oracle_estimator(wk, H, res.emin, res.emax, 120)
    G, _ = api.density_and_forces(ctx, res.H, None, None, s.box, res.emin, res.emax, wk.probe_seed,
                                  wk.n_probes, 120, est["mu"], wk.kT, False, True, want_forces=False)
    Gd = och.estimator_gradient(est["w"], est["V"], est["R"], res.emin, res.emax, est["mu"], wk.kT,
                                p=120)
    ref = blocks_of(Gd, rp, col, 9)
    assert np.abs(G.cpu().numpy() - ref).max() < 1e-9 * np.abs(ref).max()


def test_bloch_oracle_estimator_on_the_gpu_probes(api, ctx, lattice):
    """The Bloch route (48^3-capable) reproduces the dense estimator on the GPU's probes."""
    wk, rp, col, H, s, pos = lattice
    res = s.energies(pos, order=150, fp64=True)
    L = 6
    wk_b, U = bloch.bands(L, wk.disp, wk.blocks)
    R = och.probes(H.shape[0], wk.n_probes, wk.probe_seed)
    wts = bloch.estimator_weights(L, R, U)
    mom = och.cheb_T(och.mapped(wk_b.ravel(), res.emin, res.emax), 150) @ wts.ravel()
    n = H.shape[0]
    assert np.abs(res.moments.cpu().numpy() - mom).max() < 1e-10 * n
    # and the exact physics of the lattice lies within the sampling error of the estimate
    mu = physics.chemical_potential(wk_b.ravel(), wk.n_electrons, wk.kT)
    Om, E, N = physics.observables(wk_b.ravel(), mu, wk.kT)
    assert abs(N - wk.n_electrons) < 1e-8


@pytest.mark.parametrize("s", [128, 512])
def test_periodic_density_matrix_mixed_fused_kernel(api, ctx, s):
    """The benchmarked precision and kernels on the periodic lattice: G from the fused adjoint
    step (FP32 panels, 128 and 512 probes, blocks wrapping across the cell) against the oracle's
    Daleckii-Krein gradient of the same estimator, every entry within 2e-5 of max G."""
    wk = wl.sc9_periodic(L=6, kT=0.05, n_probes=s, order=None)
    rp, col, H = oracle_H(wk)
    sv = api.Solver(wk, ctx)
    pos = torch.as_tensor(wk.positions, dtype=torch.float64, device="cuda")
    p = 120
    res = sv.energies(pos, order=p, fp64=False)
    est = oracle_estimator(wk, H, res.emin, res.emax, p)
    G, _ = api.density_and_forces(ctx, res.H, None, None, sv.box, res.emin, res.emax, wk.probe_seed, s, p,
                                  est["mu"], wk.kT, False, False, want_forces=False, windowed="fused")
    Gd = och.estimator_gradient(est["w"], est["V"], est["R"], res.emin, res.emax, est["mu"], wk.kT, p=p)
    ref = blocks_of(Gd, rp, col, 9)
    assert np.abs(G.cpu().numpy() - ref).max() < 2e-5 * np.abs(ref).max()
