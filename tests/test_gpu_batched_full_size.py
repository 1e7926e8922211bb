"""Parity of the 64-cluster batch at its full size, in the configuration the benchmark runs it:
64 jittered fcc clusters of 100..5,000 atoms (log-uniform, 92,999 atoms in all), kT in
{0.025, 0.1, 0.5} eV, 128 probes each, every cluster at the order of the error model, all in one
batched energies-and-forces call with windowed outer products, FP32 recurrence, FP64 moments.

Checks:
* every cluster: the bisection meets N^(mu^) = N_e, and the forces sum to zero;
* the three smallest clusters (kept whole by the dense oracle): mu, Omega, E, N within 1e-4 eV per
  atom and the forces within 1e-3 eV/A of the oracle's exact estimator at the batch's own bounds
  and order;
* the largest cluster (5,000-class, no dense oracle): its first 64 moments, all 128 probes,
  against the oracle's host FP64 block-sparse recurrence on the oracle's own H (2e-6 * n, the
  tolerance of the single-cluster full-size test).
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import hamiltonian as oham, neighbors as onb

from gpu_common import oracle_H, oracle_estimator, oracle_estimator_forces

pytestmark = pytest.mark.gpu

S, P_HOST = 128, 64


@pytest.fixture(scope="module")
def api():
    from paper_1812_05264_gb300 import build
    build.build()
    from paper_1812_05264_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def batch(api):
    spec = wl.batched_clusters(64, 100, 5000, (0.025, 0.1, 0.5), seed=6464)
    wks = []
    for i, (n, kT) in enumerate(zip(spec.sizes, spec.kTs)):
        wk = wl.fcc_cu(int(n), kT=float(kT), n_probes=S, seed=5264, probe_seed=64000 + i)
        wk.positions = spec.positions[i]
        wks.append(wk)
    ctx = api.Context()
    model = api.Solver(wks[0], ctx).model
    pos = [torch.as_tensor(np.ascontiguousarray(w.positions), dtype=torch.float64, device="cuda")
           for w in wks]
    graphs = api.batched_build_neighbors(ctx, pos, wks[0].cutoff)
    Hs = [api.assemble_H(ctx, model, p_, g) for p_, g in zip(pos, graphs)]
    e0, e1 = api.batched_spectral_bounds(ctx, Hs)
    ps = [api.order_for(hi - lo, w.kT) for w, lo, hi in zip(wks, e0, e1)]
    mom, obs, _, Fs = api.batched_energies_and_forces(
        ctx, Hs, model, pos, e0, e1, [w.probe_seed for w in wks], S, ps, [w.n_electrons for w in wks],
        [w.kT for w in wks], windowed=True)
    out = dict(wks=wks, e0=e0, e1=e1, ps=ps, mom=[m.cpu().numpy() for m in mom], obs=obs,
               F=[f.cpu().numpy() for f in Fs])
    yield out
    out.clear()
    del Hs, graphs, pos, mom, Fs
    ctx.close()
    torch.cuda.empty_cache()


def test_batch_is_the_benchmarked_configuration(batch):
    wks, ps = batch["wks"], batch["ps"]
    assert len(wks) == 64 and sum(w.n_atoms for w in wks) == 92999
    assert max(ps) > 2000 and min(ps) < 200          # kT = 0.025 and 0.5 eV clusters together


def test_every_cluster_meets_its_electron_count_and_momentum(batch):
    for w, o, F in zip(batch["wks"], batch["obs"], batch["F"]):
        mu, _, _, N = o
        assert abs(N - w.n_electrons) < 1e-6 * w.n_electrons
        assert np.isfinite(F).all()
        assert np.abs(F.sum(axis=0)).max() < 1e-6 * max(1.0, np.abs(F).sum())


def test_smallest_clusters_against_the_oracle(batch):
    wks = batch["wks"]
    for c in np.argsort([w.n_atoms for w in wks])[:3]:
        w, lo, hi, p, o = wks[c], batch["e0"][c], batch["e1"][c], batch["ps"][c], batch["obs"][c]
        rp, col, Hd = oracle_H(w)
        est = oracle_estimator(w, Hd, lo, hi, p)
        n = w.n_atoms
        for j, key in ((1, "Omega"), (2, "E"), (3, "N")):
            assert abs(o[j] - est[key]) / n < 1e-4, (c, key)
        assert abs(o[0] - est["mu"]) < 1e-4
        _, Fo = oracle_estimator_forces(w, rp, col, dict(est, mu=o[0]), lo, hi, p)
        assert np.abs(batch["F"][c] - Fo).max() < 1e-3, c


def test_largest_cluster_moments_against_the_host_recurrence(batch):
    from oracle import o2
    wks = batch["wks"]
    c = int(np.argmax([w.n_atoms for w in wks]))
    w = wks[c]
    rp, col = onb.neighbor_csr(w.positions, w.cutoff)
    Hs = oham.sparse_sk(w.positions, rp, col, w.sk_V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)
    ref, _ = o2.moments(rp, col, Hs.data, batch["e0"][c], batch["e1"][c], w.probe_seed, S, P_HOST,
                        doubled=True)
    n = Hs.shape[0]
    assert np.abs(batch["mom"][c][:P_HOST] - ref).max() < 2e-6 * n
