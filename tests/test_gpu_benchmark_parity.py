"""Parity of the benchmarked kernels and configurations against the FP64 oracle, element by
element where the oracle can compute the output.

* The sampled density matrix G = dOmega^/dH on the pattern (Sec. II.D, Eq. polynomial_response)
  from the kernels the benchmark times: the fused adjoint step with its outer products (128, 256
  and 512 probes per task), the windowed schedule (the adjoint step alone plus the window
  kernel) and the tensor-core schedule (the adjoint step alone plus the tcgen05 sampled-product
  kernel), each against the oracle's Daleckii-Krein gradient of the same estimator.
* The 10,000-atom workload's own check on a 500-atom sub-cluster: kT = 0.025 eV, 512 probes, the
  order p of the error model (about 2,400 terms), the benchmark's call (autotuned, one-call
  energies and forces, mixed precision): mu, Omega, E, N, every G entry and the forces against
  the oracle; and central finite differences (dx = 1e-4 A) of the FP64 estimate on 8 atoms
  against the forces that torch.autograd gets from the adjoint kernel.
* A batch with the orders of the error model (no cap), kT = 0.025 eV clusters included.
* The 48^3 periodic 9-orbital lattice (1.0M orbitals, 10 eV band) at the order of the error model
  against the Bloch oracle's exact estimator: three sampled probes of the benchmarked 512-probe
  mixed run, and an 8-probe FP64 run whole.

Tolerances.  Energies: 1e-4 eV/atom mixed, 1e-6 eV/atom FP64; forces 1e-3 eV/A; G: 2e-5 of
max|G|.  An FP32 emulation of the same estimator and adjoint on the host (40 and 60 atoms,
p = 80 and 2,162) is within 6e-7 of max|G| of the oracle, so 2e-5 leaves a factor 30 for the
kernels' summation order; a dropped tile or a wrong sign moves entries by O(max|G|).
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import bloch, chebyshev as och

from gpu_common import blocks_of, oracle_H, oracle_estimator, oracle_estimator_forces

pytestmark = pytest.mark.gpu

G_TOL = 2e-5


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


def _operator(api, ctx, wk):
    model = api.Model.from_workload(wk, torch.device("cuda"))
    pos = _dev(wk.positions)
    g = api.build_neighbors(ctx, pos, wk.cutoff)
    H = api.assemble_H(ctx, model, pos, g)
    emin, emax = api.spectral_bounds(ctx, H)
    return model, pos, H, emin, emax


def _g_err(G, Gd, rp, col):
    ref = blocks_of(Gd, rp, col, 9)
    return np.abs(G.cpu().numpy() - ref).max() / np.abs(ref).max()


# ---- G of the benchmarked adjoint kernels, element by element --------------------------------

@pytest.mark.parametrize("s", [128, 256, 512])
@pytest.mark.parametrize("windowed", [False, True, "tensor"])
def test_adjoint_kernels_G_elementwise_vs_oracle(api, ctx, s, windowed):
    wk = wl.fcc_cu(40, kT=0.5, n_probes=s, seed=5264, probe_seed=11, jitter=0.05)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    p = 80
    est = oracle_estimator(wk, Hd, emin, emax, p)
    Gd, F = oracle_estimator_forces(wk, rp, col, est, emin, emax, p)
    G, Fg = api.density_and_forces(ctx, H, model, pos, None, emin, emax, wk.probe_seed, s, p,
                                   est["mu"], wk.kT, False, False, windowed=windowed)
    err = _g_err(G, Gd, rp, col)
    assert err < G_TOL, err
    assert np.abs(Fg.cpu().numpy() - F).max() < 1e-3


# ---- the 10,000-atom workload's check on a 500-atom sub-cluster -------------------------------

@pytest.fixture(scope="module")
def sub500(api, ctx):
    """The benchmarked model, temperature and probe count on the first 500 atoms of the sphere,
    run as the benchmark runs it, and the oracle's exact estimator on the same inputs."""
    wk = wl.fcc_cu(500, kT=0.025, n_probes=512, seed=5264, probe_seed=52640)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    api.autotune(ctx, H, emin, emax, 512)
    p = api.order_for(emax - emin, wk.kT)
    mom, obs, G, F = api.energies_and_forces(ctx, H, model, pos, None, emin, emax, wk.probe_seed, 512,
                                             p, wk.n_electrons, wk.kT, False, False, want_G=True)
    est = oracle_estimator(wk, Hd, emin, emax, p)
    # G and forces at the GPU's mu (the oracle's mu differs from it by rounding)
    Gd, Fo = oracle_estimator_forces(wk, rp, col, dict(est, mu=obs[0]), emin, emax, p)
    return dict(wk=wk, rp=rp, col=col, model=model, pos=pos, H=H, emin=emin, emax=emax, p=p,
                mom=mom, obs=obs, G=G, F=F, est=est, Gd=Gd, Fo=Fo)


def test_subcluster500_energies_at_the_benchmark_order(sub500):
    r = sub500
    assert r["p"] > 2000                       # "several thousand" terms at kT = 0.025 eV
    n = r["wk"].n_atoms
    mu, Om, E, N = r["obs"]
    est = r["est"]
    assert abs(mu - est["mu"]) < 1e-4
    for got, key in ((Om, "Omega"), (E, "E"), (N, "N")):
        assert abs(got - est[key]) / n < 1e-4, (key, abs(got - est[key]) / n)
    nr = n * 9
    assert np.abs(r["mom"].cpu().numpy() - est["moments"]).max() < 2e-6 * nr


def test_subcluster500_G_and_forces_at_the_benchmark_order(sub500):
    r = sub500
    err = _g_err(r["G"], r["Gd"], r["rp"], r["col"])
    assert err < G_TOL, err
    assert np.abs(r["F"].cpu().numpy() - r["Fo"]).max() < 1e-3
    assert np.abs(r["F"].cpu().numpy().sum(0)).max() < 1e-8


@pytest.mark.parametrize("sched", ["fused", "windowed", "tensor"])
def test_subcluster500_every_schedule_at_the_benchmark_order(api, ctx, sub500, sched):
    """The same one-call run with each outer-product schedule forced: G against the oracle."""
    r = sub500
    wk = r["wk"]
    mom, obs, G, F = api.energies_and_forces(ctx, r["H"], r["model"], r["pos"], None, r["emin"], r["emax"],
                                             wk.probe_seed, 512, r["p"], wk.n_electrons, wk.kT, False, False,
                                             want_G=True, windowed=sched)
    assert torch.equal(mom, r["mom"])
    err = _g_err(G, r["Gd"], r["rp"], r["col"])
    assert err < G_TOL, err
    assert np.abs(F.cpu().numpy() - r["Fo"]).max() < 1e-3


def test_subcluster500_autograd_forces_match_central_differences(api, ctx):
    """Forces of the adjoint kernel through torch.autograd against central differences
    (dx = 1e-4 A) of A^ = Omega^ + mu^ N_e on 8 random atoms of the 500-atom sub-cluster at
    kT = 0.025 eV and the order of the error model, in FP64 (32 probes: the derivative identity
    holds for any probe set; bounds, probes and order fixed)."""
    wk = wl.fcc_cu(500, kT=0.025, n_probes=32, seed=5264, probe_seed=52640, mixed=False)
    s = api.Solver(wk, ctx)
    pos0 = _dev(wk.positions)
    r0 = s.energies(pos0, fp64=True)
    bounds = (r0.emin - 0.5, r0.emax + 0.5)
    p = api.order_for(bounds[1] - bounds[0], wk.kT)
    s.wk.order = p
    assert p > 2000
    pos = pos0.clone().requires_grad_(True)
    A = api.FreeEnergy.apply(pos, s, bounds)
    A.backward()
    grad = pos.grad.cpu().numpy()
    ne = wk.n_electrons

    def a_hat(x):
        r = s.energies(x, fp64=True, bounds=bounds)
        return r.Omega + r.mu * ne

    rng = np.random.default_rng(5264)
    h = 1e-4
    worst = 0.0
    for a in rng.choice(wk.n_atoms, 8, replace=False):
        for c in range(3):
            pp, pm = pos0.clone(), pos0.clone()
            pp[a, c] += h
            pm[a, c] -= h
            fd = (a_hat(pp) - a_hat(pm)) / (2 * h)
            worst = max(worst, abs(grad[a, c] - fd))
    assert worst < 1e-4, worst


# ---- a batch with the orders of the error model ----------------------------------------------

@pytest.mark.parametrize("windowed", [True, False])
def test_batch_at_uncapped_orders_vs_oracle(api, ctx, windowed):
    sizes, kTs = [80, 150, 43, 110], [0.025, 0.1, 0.5, 0.025]
    wks, Hs, pos, e0, e1, ps = [], [], [], [], [], []
    model = None
    for i, (n, kT) in enumerate(zip(sizes, kTs)):
        wk = wl.fcc_cu(n, kT=kT, n_probes=128, seed=5264, probe_seed=900 + i)
        wk.positions = wl.fcc_sphere(n, jitter=0.05, seed=77 + i)
        model, p_, H, lo, hi = _operator(api, ctx, wk)
        wks.append(wk); Hs.append(H); pos.append(p_); e0.append(lo); e1.append(hi)
        ps.append(api.order_for(hi - lo, kT))
    assert max(ps) > 2000
    moms, obs, Gs, Fs = api.batched_energies_and_forces(
        ctx, Hs, model, pos, e0, e1, [w.probe_seed for w in wks], 128, ps,
        [w.n_electrons for w in wks], kTs, want_G=True, windowed=windowed)
    for wk, lo, hi, p, o, G, F in zip(wks, e0, e1, ps, obs, Gs, Fs):
        rp, col, Hd = oracle_H(wk)
        est = oracle_estimator(wk, Hd, lo, hi, p)
        n = wk.n_atoms
        for j, key in ((1, "Omega"), (2, "E"), (3, "N")):
            assert abs(o[j] - est[key]) / n < 1e-4, (n, key)
        assert abs(o[0] - est["mu"]) < 1e-4
        # G and forces at the batch's own mu (the oracle's differs by rounding)
        Gd, Fo = oracle_estimator_forces(wk, rp, col, dict(est, mu=o[0]), lo, hi, p)
        err = _g_err(G, Gd, rp, col)
        assert err < G_TOL, (n, err)
        assert np.abs(F.cpu().numpy() - Fo).max() < 1e-3, n


# ---- the 48^3 periodic lattice against the Bloch oracle --------------------------------------

L48, SAMPLED = 48, [0, 137, 511]


@pytest.fixture(scope="module")
def lattice48(api, ctx):
    wk = wl.sc9_periodic(L=L48, n_probes=512)
    sv = api.Solver(wk, ctx)
    pos = _dev(wk.positions)
    g = api.build_neighbors(ctx, pos, wk.cutoff, sv.box)
    H = api.assemble_H(ctx, sv.model, pos, g, sv.box)
    emin, emax = api.spectral_bounds(ctx, H)
    p = api.order_for(emax - emin, wk.kT)
    eps, U = bloch.bands(L48, wk.disp, wk.blocks)
    x = och.mapped(eps.ravel(), emin, emax)
    return dict(wk=wk, H=H, emin=emin, emax=emax, p=p, eps=eps, U=U, x=x)


def _bloch_moments(lat, seed, cols):
    """Each probe's exact moments r^T C_k(H^) r through the Bloch bands (rows k, columns probes)."""
    wk, U, p, x = lat["wk"], lat["U"], lat["p"], lat["x"]
    n = wk.n_atoms * 9
    Wt = []
    for j in cols:
        r = och.probe_columns(n, [j], seed)
        Wt.append(bloch.estimator_weights(L48, r, U).ravel())
    Wt = np.array(Wt)                         # (probes, k-points x bands)
    out = np.zeros((p, len(cols)))
    t0, t1 = np.ones_like(x), x.copy()
    for k in range(p):
        if k >= 2:
            t0, t1 = t1, 2.0 * x * t1 - t0
        out[k] = Wt @ (t0 if k == 0 else t1)
    return out


def test_lattice48_band_and_order(lattice48):
    lat = lattice48
    w = lat["eps"]
    assert abs((w.max() - w.min()) - 10.0) < 1e-9
    assert lat["emin"] < w.min() and lat["emax"] > w.max()
    assert 480 < lat["p"] < 560                   # (W / kT) ln(1e7) / 6.4 with W ~ 10.2 eV


def test_lattice48_mixed_512_probes_sampled_against_bloch(api, ctx, lattice48):
    """The benchmarked configuration (mixed, 512 probes, autotuned) on the 1.0M-orbital lattice:
    the per-probe moments of three probes against their exact values, and the mean over all
    probes equal to the moments call's."""
    lat = lattice48
    wk, H, emin, emax, p = lat["wk"], lat["H"], lat["emin"], lat["emax"], lat["p"]
    api.autotune(ctx, H, emin, emax, 512)
    mom, per = api.chebyshev_probe_moments(ctx, H, emin, emax, wk.probe_seed, 512, p)
    ref = _bloch_moments(lat, wk.probe_seed, SAMPLED)
    n = wk.n_atoms * 9
    got = per.cpu().numpy()[:, SAMPLED]
    assert np.abs(got - ref).max() < 2e-6 * n, np.abs(got - ref).max() / n
    m2 = api.chebyshev_moments(ctx, H, emin, emax, wk.probe_seed, 512, p)
    assert np.abs(m2.cpu().numpy() - mom.cpu().numpy()).max() < 1e-9 * n
    # the energies of the three sampled probes' estimate
    mu, Om, E, N = api.fermi_level(ctx, _dev(got.mean(1)), emin, emax, wk.n_electrons, wk.kT)
    rm = ref.mean(1)
    mu_o = och.estimator_mu(rm, emin, emax, wk.n_electrons, wk.kT)
    Om_o, E_o, N_o = och.estimator_observables(rm, emin, emax, mu_o, wk.kT)
    for a, b in ((Om, Om_o), (E, E_o), (N, N_o)):
        assert abs(a - b) / wk.n_atoms < 1e-4


@pytest.mark.parametrize("fp64,tol", [(True, 1e-6), (False, 1e-4)])
def test_lattice48_energies_vs_bloch(api, ctx, lattice48, fp64, tol):
    """8 probes, whole: moments and energies per site against the Bloch oracle, FP64 and mixed."""
    lat = lattice48
    wk, H, emin, emax, p = lat["wk"], lat["H"], lat["emin"], lat["emax"], lat["p"]
    seed = 4848
    mom = api.chebyshev_moments(ctx, H, emin, emax, seed, 8, p, fp64=fp64)
    ref = _bloch_moments(lat, seed, range(8)).mean(1)
    n = wk.n_atoms * 9
    assert np.abs(mom.cpu().numpy() - ref).max() < (1e-11 if fp64 else 2e-6) * n
    mu, Om, E, N = api.fermi_level(ctx, mom, emin, emax, wk.n_electrons, wk.kT)
    mu_o = och.estimator_mu(ref, emin, emax, wk.n_electrons, wk.kT)
    Om_o, E_o, N_o = och.estimator_observables(ref, emin, emax, mu_o, wk.kT)
    for a, b in ((Om, Om_o), (E, E_o), (N, N_o)):
        assert abs(a - b) / wk.n_atoms < tol


def test_tensor_schedule_falls_back_on_rows_longer_than_its_groups(api, ctx):
    """A 6 A cutoff gives rows of up to 79 stored blocks, more than the tensor-core kernel's 32:
    the TBK_TC_OUTER schedule then runs the fused kernel, and G equals the fused schedule's."""
    wk = wl.fcc_cu(60, kT=0.5, n_probes=128, seed=5264, probe_seed=21, jitter=0.05)
    wk.cutoff = 6.0
    model, pos, H, emin, emax = _operator(api, ctx, wk)
    assert int((H.graph.row_ptr[1:] - H.graph.row_ptr[:-1]).max()) > 32
    args = (ctx, H, model, pos, None, emin, emax, wk.probe_seed, 128, 40, 3.0, wk.kT, False, False)
    G1, F1 = api.density_and_forces(*args, windowed="tensor")
    G0, F0 = api.density_and_forces(*args, windowed="fused")
    assert torch.equal(G1, G0) and torch.equal(F1, F0)
