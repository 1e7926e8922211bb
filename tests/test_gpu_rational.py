"""f4: the rational approximation with CGLS solves (Sec. II.B.2, Eq. rational_fit, Eq. rational_PQ
with S = I, Eq. random_density) on the GPU, through the C ABI, against the oracle
(oracle/rational.py: the same continued-fraction poles, evaluated through the eigenpairs).

Tolerances: CGLS to a relative residual of 1e-12 per probe column; every block entry of P~ and
Q~ within 1e-8 of the largest; forces within 1e-6 eV/A.  Independent of the oracle: with enough
pole pairs the rational estimate and the Chebyshev direct estimate (same probes, high order)
approximate the same f(H) R R^T / s, and agree to 1e-7 of the largest entry.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import chebyshev as och, hamiltonian as oham, physics as oph, rational as ora

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


def _operator(api, ctx, wk):
    model = api.Model.from_workload(wk, torch.device("cuda"))
    pos = _dev(wk.positions)
    g = api.build_neighbors(ctx, pos, wk.cutoff)
    H = api.assemble_H(ctx, model, pos, g)
    emin, emax = api.spectral_bounds(ctx, H)
    return model, pos, H, emin, emax


@pytest.mark.parametrize("n_pairs,s", [(8, 8), (24, 16)])
def test_rational_density_vs_oracle(api, ctx, n_pairs, s):
    wk = wl.fcc_cu(30, kT=0.5, n_probes=s, seed=5264, probe_seed=71, jitter=0.05)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    w, V = np.linalg.eigh(Hd)
    mu = float(np.median(w))
    P, Q, F, (iters, res) = api.rational_density(ctx, H, model, pos, None, wk.probe_seed, s, mu, wk.kT,
                                                 n_pairs, tol=1e-12, want_forces=True)
    assert res < 1e-12 and iters > 0
    R = och.probes(Hd.shape[0], s, wk.probe_seed)
    Pt, Qt = ora.rational_density(w, V, R, mu, wk.kT, n_pairs)
    for got, ref in ((P, Pt), (Q, Qt)):
        rb = blocks_of(ref, rp, col, 9)
        err = np.abs(got.cpu().numpy() - rb).max() / np.abs(rb).max()
        assert err < 1e-8, err
    Ps = blocks_of(0.5 * (Pt + Pt.T), rp, col, 9)
    G = np.zeros_like(Pt)
    for a in range(wk.n_atoms):
        for k in range(rp[a], rp[a + 1]):
            G[9 * a:9 * a + 9, 9 * col[k]:9 * col[k] + 9] = Ps[k]
    a_, b_, dH = oham.sk_bond_grads(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY)
    Fo = oph.forces_from_blocks(G, a_, b_, dH, wk.n_atoms, 9)
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-6


def test_rational_and_chebyshev_estimates_agree(api, ctx):
    """Both approximate f(H) R R^T / s on the same probes: 40 pole pairs against 1,200 Chebyshev
    terms at kT = 0.5 eV."""
    wk = wl.fcc_cu(30, kT=0.5, n_probes=8, seed=5264, probe_seed=72, jitter=0.05)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    mu = 0.5 * (emin + emax)
    Pr, Qr, _, _ = api.rational_density(ctx, H, None, None, None, wk.probe_seed, 8, mu, wk.kT, 40, tol=1e-12)
    Pc, Qc, _ = api.direct_density(ctx, H, None, None, None, emin, emax, wk.probe_seed, 8, 1200, mu, wk.kT,
                                   fp64=True)
    for a, b in ((Pr, Pc), (Qr, Qc)):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.abs(a - b).max() < 1e-7 * np.abs(b).max()


def test_rational_reports_a_solve_that_stops_early(api, ctx):
    from paper_1812_05264_gb300._lib import TBK_ERR_NOCONV, TBK_ERR_ARG, TbkError
    wk = wl.fcc_cu(20, kT=0.5, n_probes=8, seed=5264, probe_seed=73)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    with pytest.raises(TbkError) as e:
        api.rational_density(ctx, H, None, None, None, 1, 8, 0.0, wk.kT, 8, tol=1e-12, max_iter=2)
    assert e.value.code == TBK_ERR_NOCONV
    with pytest.raises(TbkError) as e:
        api.rational_density(ctx, H, None, None, None, 1, 6, 0.0, wk.kT, 8)   # probes not a multiple of 4
    assert e.value.code == TBK_ERR_ARG
    P, _, _, (it, res) = api.rational_density(ctx, H, None, None, None, 1, 8, 0.0, wk.kT, 8, want_Q=False)
    assert res < 1e-10 and torch.isfinite(P).all()


def test_rational_single_pole_pair(api, ctx):
    """n_pairs = 1: f_r(x) = 1 + 2 Re w_1/(x - zeta_1), the coarsest expansion, FP64 against the
    oracle's eigen route."""
    wk = wl.fcc_cu(15, kT=0.5, n_probes=4, seed=5264, probe_seed=74, jitter=0.05)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    w, V = np.linalg.eigh(Hd)
    mu = float(np.median(w))
    P, Q, _, (it, res) = api.rational_density(ctx, H, None, None, None, wk.probe_seed, 4, mu, wk.kT, 1, tol=1e-12)
    R = och.probes(Hd.shape[0], 4, wk.probe_seed)
    Pt, Qt = ora.rational_density(w, V, R, mu, wk.kT, 1)
    for got, ref in ((P, Pt), (Q, Qt)):
        rb = blocks_of(ref, rp, col, 9)
        assert np.abs(got.cpu().numpy() - rb).max() < 1e-8 * np.abs(rb).max()
