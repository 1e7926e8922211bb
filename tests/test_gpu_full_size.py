"""Parity at the full size of the benchmarked workload, in the launch configuration the benchmark
times: the 10,000-atom fcc cluster (9 x 9 blocks, kT = 0.025 eV, 512 probes, the order of the
error model), the library's autotuned schedule, FP32 recurrence with FP64 moments.

The dense oracle does not fit at this size (90,000 rows), so the checks are:
* the neighbour pattern, bit for bit, and every stored block of H, against the oracle's sparse
  assembly;
* sampled outputs the oracle computes one by one: the per-probe moments r_i^T C_k(H^) r_i of
  three probes, by the FP64 three-term recurrence on the sparse H (Eq. poly_PQ), against the
  benchmarked mixed path and against the plain FP64 path;
* the moments of all 512 probes against the oracle's host FP64 block-sparse recurrence
  (C/OpenMP, written independently of the CUDA library);
* properties that hold at any size: the bisection meets N^(mu^) = N_e, the forces sum to zero
  (H depends only on the bond vectors), and the one-call path's moments are those of the
  moments call.

Tolerance of the sampled moments: 2e-6 * n.  An FP32 recurrence with FP64 dot products on this
operator, simulated on the host, is off by at most 2.2e-8 * n over the first 64 moments, so
2e-6 * n leaves two orders of magnitude for a different summation order.  A dropped tile or
a sign slip moves a moment by O(1) or more.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import chebyshev as och, hamiltonian as oham, neighbors as onb

pytestmark = pytest.mark.gpu

N_ATOMS, KT, S, SEED, PROBE_SEED = 10000, 0.025, 512, 5264, 52640
SAMPLED = [0, 137, 511]
P_SAMPLED = 64


@pytest.fixture(scope="module")
def api():
    from paper_1812_05264_gb300 import build
    build.build()
    from paper_1812_05264_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def run(api):
    wk = wl.fcc_cu(N_ATOMS, kT=KT, n_probes=S, seed=SEED, probe_seed=PROBE_SEED)
    ctx = api.Context()
    model = api.Model.from_workload(wk, torch.device("cuda"))
    pos = torch.as_tensor(wk.positions, dtype=torch.float64, device="cuda")
    g = api.build_neighbors(ctx, pos, wk.cutoff, None)
    H = api.assemble_H(ctx, model, pos, g, None)
    emin, emax = api.spectral_bounds(ctx, H)
    api.autotune(ctx, H, emin, emax, S)
    p = api.order_for(emax - emin, wk.kT)
    mom, obs, _, F = api.energies_and_forces(ctx, H, model, pos, None, emin, emax, PROBE_SEED, S, p,
                                             wk.n_electrons, wk.kT, False, False, want_G=False,
                                             want_forces=True)
    rp, col = onb.neighbor_csr(wk.positions, wk.cutoff)
    Hs = oham.sparse_sk(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)
    R = och.probes(Hs.shape[0], S, PROBE_SEED)[:, SAMPLED]
    out = dict(wk=wk, ctx=ctx, g=g, H=H, emin=emin, emax=emax, p=p, mom=mom, obs=obs, F=F,
               rp=rp, col=col, Hs=Hs, Hcsr=Hs.tocsr(), R=R)
    yield out
    # the one-call path keeps its panels in device memory: give them back before the next module
    out.clear()
    del g, H, mom, F, pos
    ctx.close()
    torch.cuda.empty_cache()


def test_pattern_and_blocks_at_full_size(run):
    g, rp, col = run["g"], run["rp"], run["col"]
    assert g.nnzb == len(col)
    assert np.array_equal(g.row_ptr.cpu().numpy(), rp.astype(np.int32))
    assert np.array_equal(g.col.cpu().numpy(), col)
    val = run["H"].val.cpu().numpy()
    assert np.abs(val - run["Hs"].data).max() < 1e-13


@pytest.mark.parametrize("fp64,direct", [(False, False), (False, True), (True, False)])
def test_sampled_probe_moments_at_full_size(api, run, fp64, direct):
    """Mixed: the benchmarked precision, within 2e-6 n.  FP64: the plain FP64 path against the
    oracle's FP64 recurrence on the same probes, within 1e-11 n (both sides round in FP64)."""
    n = run["Hs"].shape[0]
    mom, per = api.chebyshev_probe_moments(run["ctx"], run["H"], run["emin"], run["emax"], PROBE_SEED,
                                           S, P_SAMPLED, fp64=fp64, direct=direct)
    ref = och.recurrence_probe_moments(run["Hcsr"], run["R"], run["emin"], run["emax"], P_SAMPLED)
    got = per.cpu().numpy()[:, SAMPLED]
    assert np.abs(got - ref).max() < (1e-11 if fp64 else 2e-6) * n
    # the probe mean is the moments call
    assert np.allclose(per.mean(dim=1).cpu().numpy(), mom.cpu().numpy(), rtol=0,
                       atol=(1e-12 if fp64 else 1e-6) * n)
    if not fp64:
        # and the one-call path's forward sweep gives the same moments
        assert np.allclose(run["mom"][:P_SAMPLED].cpu().numpy(), mom.cpu().numpy(), rtol=0,
                           atol=1e-6 * n)


P_ALL = 24


@pytest.mark.parametrize("fp64", [False, True])
def test_all_probe_moments_at_full_size_against_the_host_recurrence(api, run, fp64):
    """Every probe at once: the moments of all 512 probes (order 24) against the oracle's host
    FP64 block-sparse recurrence (oracle/o2_recurrence.c, C/OpenMP, doubled moments as on the GPU)
    on the oracle's own H: the benchmarked mixed path within 2e-6 n, the plain FP64 path within
    1e-11 n."""
    from oracle import o2
    Hs = run["Hs"]
    n = Hs.shape[0]
    ref, products = o2.moments(run["rp"], run["col"], Hs.data, run["emin"], run["emax"], PROBE_SEED, S, P_ALL,
                               doubled=True)
    assert products == P_ALL // 2
    mom = api.chebyshev_moments(run["ctx"], run["H"], run["emin"], run["emax"], PROBE_SEED, S, P_ALL, fp64=fp64)
    assert np.abs(mom.cpu().numpy() - ref).max() < (1e-11 if fp64 else 2e-6) * n


def test_properties_of_the_full_step(run):
    wk, (mu, Om, E, N) = run["wk"], run["obs"]
    assert run["p"] > 2000                                  # the order the benchmark runs at
    assert run["emin"] < mu < run["emax"]
    assert abs(N - wk.n_electrons) < 1e-6 * wk.n_electrons
    F = run["F"].cpu().numpy()
    assert np.isfinite(F).all()
    assert np.abs(F.sum(axis=0)).max() < 1e-6 * np.abs(F).sum()
