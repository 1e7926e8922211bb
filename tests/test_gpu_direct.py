"""f2: the direct random estimates M o P~ and M o Q~ (Eq. poly_PQ with S = I, Eq. random_density)
on the GPU, through the C ABI, against the oracle (oracle/direct.py) on the same probes, order,
bounds, mu and kT.

Tolerances: every block entry within 1e-10 (FP64) or 2e-5 (mixed) of max|P~| (likewise Q~); the
forces from the symmetric part within 1e-6 (FP64) / 1e-3 (mixed) eV/A.  Independent of the
oracle: the trace of P~ equals the moment route's N^(mu) (tbk_chebyshev_moments +
tbk_fermi_level at fixed mu), to 1e-9 relative in FP64.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import chebyshev as och, direct as odi, hamiltonian as oham, physics as oph

from gpu_common import blocks_of, oracle_H

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
    c.close()


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _operator(api, ctx, wk, box=None):
    model = api.Model.from_workload(wk, torch.device("cuda"))
    pos = _dev(wk.positions)
    g = api.build_neighbors(ctx, pos, wk.cutoff, box)
    H = api.assemble_H(ctx, model, pos, g, box)
    emin, emax = api.spectral_bounds(ctx, H)
    return model, pos, H, emin, emax


@pytest.mark.parametrize("s,fp64", [(128, False), (512, False), (16, False), (16, True), (128, True)])
def test_direct_density_vs_oracle(api, ctx, s, fp64):
    wk = wl.fcc_cu(40, kT=0.5, n_probes=s, seed=5264, probe_seed=313, jitter=0.05)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    p = 120
    w, V = np.linalg.eigh(Hd)
    mu = float(np.median(w))
    P, Q, F = api.direct_density(ctx, H, model, pos, None, emin, emax, wk.probe_seed, s, p, mu, wk.kT,
                                 fp64=fp64, want_forces=True)
    R = och.probes(Hd.shape[0], s, wk.probe_seed)
    Pt, Qt = odi.direct_density(w, V, R, emin, emax, mu, wk.kT, p)
    tol = 1e-10 if fp64 else 2e-5
    for got, ref in ((P, Pt), (Q, Qt)):
        rb = blocks_of(ref, rp, col, 9)
        err = np.abs(got.cpu().numpy() - rb).max() / np.abs(rb).max()
        assert err < tol, err
    Ps = blocks_of(0.5 * (Pt + Pt.T), rp, col, 9)
    G = np.zeros_like(Pt)
    for a in range(wk.n_atoms):
        for k in range(rp[a], rp[a + 1]):
            b = col[k]
            G[9 * a:9 * a + 9, 9 * b:9 * b + 9] = Ps[k]
    a_, b_, dH = oham.sk_bond_grads(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY)
    Fo = oph.forces_from_blocks(G, a_, b_, dH, wk.n_atoms, 9)
    assert np.abs(F.cpu().numpy() - Fo).max() < (1e-6 if fp64 else 1e-3)


def test_trace_of_the_direct_density_is_the_moment_route_count(api, ctx):
    """tr P~ = (1/s) sum_i r_i^T p_f(H^) r_i = N^(mu): the diagonal entries of the diagonal blocks
    against the Chebyshev moments and the Fermi-level call at the same mu (FP64)."""
    wk = wl.fcc_cu(60, kT=0.3, n_probes=32, seed=5264, probe_seed=99, jitter=0.05)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    p = 150
    mom = api.chebyshev_moments(ctx, H, emin, emax, wk.probe_seed, 32, p, fp64=True)
    mu0, _, _, _ = api.fermi_level(ctx, mom, emin, emax, wk.n_electrons, wk.kT)
    _, _, _, N = api.fermi_level(ctx, mom, emin, emax, None, wk.kT, mu=mu0)
    P, _, _ = api.direct_density(ctx, H, None, None, None, emin, emax, wk.probe_seed, 32, p, mu0, wk.kT,
                                 fp64=True, want_Q=False)
    rp = H.graph.row_ptr.cpu().numpy()
    col = H.graph.col.cpu().numpy()
    Pn = P.cpu().numpy()
    tr = sum(np.trace(Pn[k]) for a in range(wk.n_atoms) for k in range(rp[a], rp[a + 1]) if col[k] == a)
    assert abs(tr - N) < 1e-9 * abs(N)
    assert abs(N - wk.n_electrons) < 1e-6 * wk.n_electrons


def test_direct_density_one_orbital_lattice(api, ctx):
    """1 x 1 blocks (the simple-cubic cluster, Jackson damping) in FP64 and mixed precision."""
    wk = wl.sc_disorder(L=6, n_probes=16)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    w, V = np.linalg.eigh(Hd)
    mu, p = 0.0, 100
    R = och.probes(Hd.shape[0], 16, wk.probe_seed)
    Pt, Qt = odi.direct_density(w, V, R, emin, emax, mu, wk.kT, p, use_jackson=True)
    for fp64, tol in ((True, 1e-10), (False, 2e-5)):
        P, Q, _ = api.direct_density(ctx, H, None, None, None, emin, emax, wk.probe_seed, 16, p, mu, wk.kT,
                                     jackson=True, fp64=fp64)
        for got, ref in ((P, Pt), (Q, Qt)):
            rb = blocks_of(ref, rp, col, 1)
            assert np.abs(got.cpu().numpy() - rb).max() < tol * np.abs(rb).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_direct_density_lowest_orders(api, ctx, p):
    """The degenerate orders of the Clenshaw form: X = alpha_0 R (p = 1), alpha_0 R + alpha_1 H^ R
    (p = 2), and the first step with a b_{k+2} (p = 3), FP64 against the oracle."""
    wk = wl.fcc_cu(20, kT=0.5, n_probes=8, seed=5264, probe_seed=314, jitter=0.05)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    w, V = np.linalg.eigh(Hd)
    mu = float(np.median(w))
    P, Q, _ = api.direct_density(ctx, H, None, None, None, emin, emax, wk.probe_seed, 8, p, mu, wk.kT, fp64=True)
    R = och.probes(Hd.shape[0], 8, wk.probe_seed)
    Pt, Qt = odi.direct_density(w, V, R, emin, emax, mu, wk.kT, p)
    for got, ref in ((P, Pt), (Q, Qt)):
        rb = blocks_of(ref, rp, col, 9)
        assert np.abs(got.cpu().numpy() - rb).max() < 1e-10 * max(1.0, np.abs(rb).max())
