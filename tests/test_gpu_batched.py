"""a11: a batch of clusters of uneven size and temperature in one launch per recurrence step,
against the single-cluster path (same kernels, same probes) and the oracle."""
import numpy as np
import pytest
import torch

import workloads as wl

from gpu_common import oracle_H, oracle_estimator

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1812_05264_gb300 import build
    build.build()
    from paper_1812_05264_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def ctx(api):
    return api.Context()


def _batch(api, ctx, sizes, kTs, s=128):
    out = []
    for i, (n, kT) in enumerate(zip(sizes, kTs)):
        wk = wl.fcc_cu(n, kT=kT, n_probes=s, jitter=0.05, seed=5264, probe_seed=700 + i)
        wk.positions = wl.fcc_sphere(n, jitter=0.05, seed=31 + i)
        sv = api.Solver(wk, ctx)
        pos = torch.as_tensor(wk.positions, dtype=torch.float64, device="cuda")
        g = api.build_neighbors(ctx, pos, wk.cutoff)
        H = api.assemble_H(ctx, sv.model, pos, g)
        emin, emax = api.spectral_bounds(ctx, H)
        p = min(api.order_for(emax - emin, kT), 400)
        out.append((wk, H, emin, emax, p))
    return out


@pytest.mark.parametrize("graph", [True, False])
def test_batched_moments_equal_single_cluster_moments(api, ctx, graph):
    sizes, kTs = [37, 120, 64, 13, 90], [0.5, 0.1, 0.5, 0.1, 0.025]
    b = _batch(api, ctx, sizes, kTs)
    Hs = [x[1] for x in b]
    mom = api.batched_moments(ctx, Hs, [x[2] for x in b], [x[3] for x in b],
                              [x[0].probe_seed for x in b], 128, [x[4] for x in b], graph=graph)
    for (wk, H, emin, emax, p), m in zip(b, mom):
        ref = api.chebyshev_moments(ctx, H, emin, emax, wk.probe_seed, 128, p)
        n = wk.n_atoms * 9
        assert m.shape == ref.shape
        assert np.abs(m.cpu().numpy() - ref.cpu().numpy()).max() < 1e-9 * n
    # replay of the captured graph gives the same numbers
    mom2 = api.batched_moments(ctx, Hs, [x[2] for x in b], [x[3] for x in b],
                               [x[0].probe_seed for x in b], 128, [x[4] for x in b], graph=graph)
    for m, m2 in zip(mom, mom2):
        assert torch.equal(m, m2)


def test_batched_energies_vs_oracle(api, ctx):
    sizes, kTs = [30, 55, 19], [0.5, 0.1, 0.5]
    b = _batch(api, ctx, sizes, kTs)
    mom = api.batched_moments(ctx, [x[1] for x in b], [x[2] for x in b], [x[3] for x in b],
                              [x[0].probe_seed for x in b], 128, [x[4] for x in b])
    obs = api.batched_fermi_level(ctx, mom, [x[2] for x in b], [x[3] for x in b],
                                  [x[0].n_electrons for x in b], kTs)
    for (wk, H, emin, emax, p), o in zip(b, obs):
        rp, col, Hd = oracle_H(wk)
        est = oracle_estimator(wk, Hd, emin, emax, p)
        n = wk.n_atoms
        assert abs(o[1] - est["Omega"]) / n < 1e-4
        assert abs(o[2] - est["E"]) / n < 1e-4
        assert abs(o[3] - est["N"]) / n < 1e-4
