"""f3: the local approximation M o P~_L, M o Q~_L (Sec. II.C.1, Eq. local_density, S = I) on the
GPU, through the C ABI, against the oracle (oracle/local.py, its p-term polynomial variant on the
same bounds, mu and kT).

Tolerances: every block entry within 1e-10 (FP64) or 2e-5 (mixed) of max|P~_L| (likewise Q~_L).
Independent of the oracle: with r_max beyond the cluster every region is the whole cluster, so
P~_L is the polynomial p_f(H^) itself and Q~_L = H p_f(H^), checked against the dense three-term
matrix recurrence on H^ (FP64).
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import chebyshev as och, direct as odi, local as olo

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


@pytest.mark.parametrize("r_max,fp64", [(4.5, True), (6.0, True), (6.0, False), (4.0, False)])
def test_local_density_vs_oracle(api, ctx, r_max, fp64):
    wk = wl.fcc_cu(60, kT=0.5, n_probes=8, seed=5264, probe_seed=1, jitter=0.05)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    p = 100
    w = np.linalg.eigvalsh(Hd)
    mu = float(np.median(w))
    P, Q = api.local_density(ctx, H, pos, None, r_max, emin, emax, p, mu, wk.kT, fp64=fp64)
    mask = odi.block_mask(rp, col, 9)
    Pt, Qt = olo.local_density(Hd, wk.positions, 9, r_max, mu, wk.kT, mask=mask, poly=(emin, emax, p))
    tol = 1e-10 if fp64 else 2e-5
    for got, ref in ((P, Pt), (Q, Qt)):
        rb = blocks_of(ref, rp, col, 9)
        err = np.abs(got.cpu().numpy() - rb).max() / np.abs(rb).max()
        assert err < tol, err


def test_local_density_radius_beyond_the_cluster_is_the_polynomial(api, ctx):
    """Every region is the whole cluster: P~_L = p_f(H^) and Q~_L = H p_f(H^) on the pattern, here
    by the dense three-term matrix recurrence on H^ (FP64)."""
    wk = wl.fcc_cu(20, kT=0.5, n_probes=8, seed=5264, probe_seed=1, jitter=0.05)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    p, mu = 80, 3.0
    P, Q = api.local_density(ctx, H, pos, None, 100.0, emin, emax, p, mu, wk.kT, fp64=True)
    af, _, _ = och.fd_coefficients(p, emin, emax, mu, wk.kT)
    n = Hd.shape[0]
    Hh = (2 * Hd - (emax + emin) * np.eye(n)) / (emax - emin)
    T0, T1 = np.eye(n), Hh.copy()
    Pf = af[0] * T0 + af[1] * T1
    for k in range(2, p):
        T0, T1 = T1, 2 * Hh @ T1 - T0
        Pf += af[k] * T1
    for got, ref in ((P, Pf), (Q, Hd @ Pf)):
        rb = blocks_of(ref, rp, col, 9)
        assert np.abs(got.cpu().numpy() - rb).max() < 1e-10 * np.abs(rb).max()


def test_local_density_one_orbital_cluster(api, ctx):
    """1 x 1 blocks (the open simple-cubic cluster), FP64."""
    wk = wl.sc_disorder(L=5, n_probes=8)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    p, mu, r_max = 90, 0.1, 2.0
    P, Q = api.local_density(ctx, H, pos, None, r_max, emin, emax, p, mu, wk.kT, fp64=True)
    mask = odi.block_mask(rp, col, 1)
    Pt, Qt = olo.local_density(Hd, wk.positions, 1, r_max, mu, wk.kT, mask=mask, poly=(emin, emax, p))
    for got, ref in ((P, Pt), (Q, Qt)):
        rb = blocks_of(ref, rp, col, 1)
        assert np.abs(got.cpu().numpy() - rb).max() < 1e-10 * np.abs(rb).max()


def test_local_density_rejects_a_radius_below_the_cutoff(api, ctx):
    from paper_1812_05264_gb300._lib import TBK_ERR_ARG, TbkError
    wk = wl.fcc_cu(30, kT=0.5, n_probes=8, seed=5264, probe_seed=1)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    with pytest.raises(TbkError) as e:
        api.local_density(ctx, H, pos, None, 3.0, emin, emax, 40, 2.0, wk.kT)
    assert e.value.code == TBK_ERR_ARG


def test_local_density_single_atom(api, ctx):
    """One atom: its region is itself, so P~_L is p_f of its 9 x 9 on-site block (FP64)."""
    wk = wl.fcc_cu(1, kT=0.5, n_probes=8, seed=5264, probe_seed=1)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    p, mu = 60, 4.0
    P, Q = api.local_density(ctx, H, pos, None, 5.0, emin, emax, p, mu, wk.kT, fp64=True)
    w, V = np.linalg.eigh(Hd)
    af, _, _ = och.fd_coefficients(p, emin, emax, mu, wk.kT)
    pf = och.poly_values(af, och.mapped(w, emin, emax))
    Pref = (V * pf) @ V.T
    assert np.abs(P.cpu().numpy()[0] - Pref).max() < 1e-12
    assert np.abs(Q.cpu().numpy()[0] - Hd @ Pref).max() < 1e-11
