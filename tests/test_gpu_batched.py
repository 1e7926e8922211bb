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
    c = api.Context()
    yield c
    c.close()           # give the device memory back before the next module


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


def test_batched_forces_equal_single_cluster_forces(api, ctx):
    sizes, kTs = [37, 70, 13, 52], [0.5, 0.1, 0.5, 0.5]
    b = _batch(api, ctx, sizes, kTs)
    b = [(wk, H, e0, e1, min(p, 90 + 17 * i)) for i, (wk, H, e0, e1, p) in enumerate(b)]
    model = api.Solver(b[0][0], ctx).model
    mus = []
    for wk, H, e0, e1, p in b:
        m = api.chebyshev_moments(ctx, H, e0, e1, wk.probe_seed, 128, p)
        mus.append(api.fermi_level(ctx, m, e0, e1, wk.n_electrons, wk.kT)[0])
    pos = [torch.as_tensor(x[0].positions, dtype=torch.float64, device="cuda") for x in b]
    Gs, Fs = api.batched_density_and_forces(
        ctx, [x[1] for x in b], model, pos, [x[2] for x in b], [x[3] for x in b],
        [x[0].probe_seed for x in b], 128, [x[4] for x in b], mus, kTs, want_G=True)
    for (wk, H, e0, e1, p), mu, G, F, ps in zip(b, mus, Gs, Fs, pos):
        G1, F1 = api.density_and_forces(ctx, H, model, ps, None, e0, e1, wk.probe_seed, 128, p, mu,
                                        wk.kT, False, False, want_G=True)
        gmax = G1.abs().max().item()
        assert torch.allclose(G, G1, rtol=0, atol=2e-5 * gmax)
        assert torch.allclose(F, F1, rtol=0, atol=1e-4)
        assert F.sum(0).abs().max().item() < 1e-9


def test_batched_forces_vs_oracle(api, ctx):
    from gpu_common import oracle_estimator_forces
    sizes, kTs = [19, 28], [0.5, 0.5]
    b = _batch(api, ctx, sizes, kTs)
    b = [(wk, H, e0, e1, 80) for (wk, H, e0, e1, p) in b]
    model = api.Solver(b[0][0], ctx).model
    ests, mus = [], []
    for wk, H, e0, e1, p in b:
        rp, col, Hd = oracle_H(wk)
        est = oracle_estimator(wk, Hd, e0, e1, p)
        ests.append((rp, col, est))
        mus.append(est["mu"])
    pos = [torch.as_tensor(x[0].positions, dtype=torch.float64, device="cuda") for x in b]
    _, Fs = api.batched_density_and_forces(ctx, [x[1] for x in b], model, pos, [x[2] for x in b],
                                           [x[3] for x in b], [x[0].probe_seed for x in b], 128,
                                           [x[4] for x in b], mus, kTs)
    for (wk, H, e0, e1, p), (rp, col, est), F in zip(b, ests, Fs):
        _, Fo = oracle_estimator_forces(wk, rp, col, est, e0, e1, p)
        assert np.abs(F.cpu().numpy() - Fo).max() < 1e-3


def test_batched_adjoint_segments_and_odd_orders(api, ctx):
    """Orders of both parities (so the clusters join the backward sweep at different steps), and
    a panel budget that forces segment replays: the replayed sweep gives the same bits."""
    sizes, kTs = [24, 41, 16], [0.5, 0.5, 0.1]
    b = _batch(api, ctx, sizes, kTs)
    orders = [61, 48, 7]
    model = api.Solver(b[0][0], ctx).model
    mus = []
    for (wk, H, e0, e1, _), p in zip(b, orders):
        m = api.chebyshev_moments(ctx, H, e0, e1, wk.probe_seed, 128, p)
        mus.append(api.fermi_level(ctx, m, e0, e1, wk.n_electrons, wk.kT)[0])
    pos = [torch.as_tensor(x[0].positions, dtype=torch.float64, device="cuda") for x in b]
    args = (ctx, [x[1] for x in b], model, pos, [x[2] for x in b], [x[3] for x in b],
            [x[0].probe_seed for x in b], 128, orders, mus, kTs)
    G1, F1 = api.batched_density_and_forces(*args, want_G=True)
    panel = sum(sizes) * 9 * 128 * 4
    # all stored: K_max + 5 panels; the replay plan for K_max = 30 needs 2 x 4 + 8 + 5 = 21
    G2, F2 = api.batched_density_and_forces(*args, want_G=True, max_panel_bytes=24 * panel)
    for g1, g2, f1, f2 in zip(G1, G2, F1, F2):
        assert torch.equal(g1, g2) and torch.equal(f1, f2)
    for (wk, H, e0, e1, _), p, mu, G, F, ps in zip(b, orders, mus, G1, F1, pos):
        Gs, Fs = api.density_and_forces(ctx, H, model, ps, None, e0, e1, wk.probe_seed, 128, p, mu,
                                        wk.kT, False, False, want_G=True)
        gmax = Gs.abs().max().item()
        assert torch.allclose(G, Gs, rtol=0, atol=2e-5 * gmax)
        assert torch.allclose(F, Fs, rtol=0, atol=1e-4)


def test_batched_energies_and_forces_one_call_equals_separate_calls(api, ctx):
    """The batched one-call path takes every cluster's moments from the adjoint's own forward
    sweep: moments, (mu, Omega, E, N), G and forces equal the three separate batched calls bit
    for bit, also with segment replays."""
    sizes, kTs = [24, 41, 16, 33], [0.5, 0.1, 0.5, 0.5]
    b = _batch(api, ctx, sizes, kTs)
    orders = [61, 48, 7, 90]
    model = api.Solver(b[0][0], ctx).model
    Hs, e0, e1, seeds = [x[1] for x in b], [x[2] for x in b], [x[3] for x in b], [x[0].probe_seed for x in b]
    ne = [x[0].n_electrons for x in b]
    pos = [torch.as_tensor(x[0].positions, dtype=torch.float64, device="cuda") for x in b]
    mom = api.batched_moments(ctx, Hs, e0, e1, seeds, 128, orders)
    obs = api.batched_fermi_level(ctx, mom, e0, e1, ne, kTs)
    G1, F1 = api.batched_density_and_forces(ctx, Hs, model, pos, e0, e1, seeds, 128, orders, obs[:, 0],
                                            kTs, want_G=True)
    panel = sum(sizes) * 9 * 128 * 4
    for mpb in (0, 26 * panel):
        m2, o2, G2, F2 = api.batched_energies_and_forces(ctx, Hs, model, pos, e0, e1, seeds, 128, orders,
                                                         ne, kTs, want_G=True, max_panel_bytes=mpb)
        for a_, b_ in zip(mom, m2):
            assert torch.equal(a_, b_)
        assert np.array_equal(obs, o2)
        for g1, g2, f1, f2 in zip(G1, G2, F1, F2):
            assert torch.equal(g1, g2) and torch.equal(f1, f2)
    for (wk, H, lo, hi, _), p, o in zip(b, orders, obs):
        rp, col, Hd = oracle_H(wk)
        est = oracle_estimator(wk, Hd, lo, hi, p)
        assert abs(o[1] - est["Omega"]) / wk.n_atoms < 1e-4


def test_batched_spectral_bounds_equal_single_cluster_bounds(api, ctx):
    """All clusters' Lanczos steps run together, each on its own vectors and scalars: the bounds
    are those of the single-cluster call, bit for bit, for clusters of different sizes."""
    b = _batch(api, ctx, [37, 70, 13, 52, 5], [0.5, 0.1, 0.5, 0.5, 0.5])
    Hs = [x[1] for x in b]
    lo, hi = api.batched_spectral_bounds(ctx, Hs)
    for H, l_, h_ in zip(Hs, lo, hi):
        assert (l_, h_) == api.spectral_bounds(ctx, H)
    lo2, hi2 = api.batched_spectral_bounds(ctx, Hs, steps=20, margin=0.05, seed=7)
    for H, l_, h_ in zip(Hs, lo2, hi2):
        assert (l_, h_) == api.spectral_bounds(ctx, H, steps=20, margin=0.05, seed=7)


def test_batched_windowed_outer_products_match_fused(api, ctx):
    """Windowed outer products over a batch: each cluster's pairs stop at its own K (the rows of
    steps it never formed are not read); G matches the fused kernel up to FP32 summation order,
    and segment replays change no bit."""
    sizes, kTs = [24, 41, 16], [0.5, 0.5, 0.1]
    b = _batch(api, ctx, sizes, kTs)
    orders = [61, 48, 7]
    model = api.Solver(b[0][0], ctx).model
    Hs, e0, e1, seeds = [x[1] for x in b], [x[2] for x in b], [x[3] for x in b], [x[0].probe_seed for x in b]
    ne = [x[0].n_electrons for x in b]
    pos = [torch.as_tensor(x[0].positions, dtype=torch.float64, device="cuda") for x in b]
    m1, o1, G1, F1 = api.batched_energies_and_forces(ctx, Hs, model, pos, e0, e1, seeds, 128, orders, ne,
                                                     kTs, want_G=True)
    m2, o2, G2, F2 = api.batched_energies_and_forces(ctx, Hs, model, pos, e0, e1, seeds, 128, orders, ne,
                                                     kTs, want_G=True, windowed=True)
    assert np.array_equal(o1, o2)
    for g1, g2, f1, f2 in zip(G1, G2, F1, F2):
        gmax = g1.abs().max().item()
        assert torch.allclose(g1, g2, rtol=0, atol=2e-6 * gmax)
        assert torch.allclose(f1, f2, rtol=0, atol=1e-5)
    panel = sum(sizes) * 9 * 128 * 4
    # all stored: K_max + 2 + 7 panels = 39; the replay plan for K_max = 30 needs 2 x 4 + 8 + 9 = 25
    _, _, G3, F3 = api.batched_energies_and_forces(ctx, Hs, model, pos, e0, e1, seeds, 128, orders, ne,
                                                   kTs, want_G=True, windowed=True, max_panel_bytes=30 * panel)
    for g2, g3, f2, f3 in zip(G2, G3, F2, F3):
        assert torch.equal(g2, g3) and torch.equal(f2, f3)


def test_batched_neighbor_lists_equal_single_cluster_lists(api, ctx):
    """One call for many open clusters of different sizes (one atom, a pair, jittered fcc
    spheres): every cluster's pattern equals its own tbk_build_neighbors call bit for bit, and a
    col capacity that is too small is reported and then met."""
    import workloads as wl
    sizes = [1, 2, 37, 500, 13, 1200]
    pos = []
    for i, n in enumerate(sizes):
        p = wl.fcc_sphere(n, jitter=0.05, seed=40 + i) if n > 2 else np.array([[0.0, 0.0, 0.0], [2.0, 0.5, 0.0]])[:n]
        pos.append(torch.as_tensor(np.ascontiguousarray(p), dtype=torch.float64, device="cuda"))
    cutoff = wl.SK_CUTOFF
    gs = api.batched_build_neighbors(ctx, pos, cutoff)
    for p, g in zip(pos, gs):
        ref = api.build_neighbors(ctx, p, cutoff)
        assert g.n_atoms == ref.n_atoms and g.nnzb == ref.nnzb
        assert torch.equal(g.row_ptr, ref.row_ptr) and torch.equal(g.col, ref.col)
    # exact counts: col arrays one entry short make the call fail without touching them
    from paper_1812_05264_gb300 import _lib as L
    import ctypes as C
    n = len(pos)
    rps = [torch.empty(p.shape[0] + 1, dtype=torch.int32, device="cuda") for p in pos]
    cols = [torch.full((max(1, g.nnzb - 1),), -7, dtype=torch.int32, device="cuda") for g in gs]
    nnz = (C.c_int64 * n)()
    with pytest.raises(L.TbkError) as e:
        L.call("tbk_batched_build_neighbors", ctx.handle, n, (C.c_void_p * n)(*[p.data_ptr() for p in pos]),
               (C.c_int32 * n)(*[p.shape[0] for p in pos]), float(cutoff),
               (C.c_void_p * n)(*[r.data_ptr() for r in rps]), (C.c_void_p * n)(*[c.data_ptr() for c in cols]),
               (C.c_int64 * n)(*[c.numel() for c in cols]), nnz)
    assert e.value.code == L.TBK_ERR_ARG
    assert [nnz[i] for i in range(n)] == [g.nnzb for g in gs]
    assert all(bool((c == -7).all()) for c in cols)


@pytest.mark.parametrize("s", [256, 512])
def test_batch_at_wide_panels(api, ctx, s):
    """A batch at 256 and 512 probes per cluster runs the producer-warp step kernel (probe chunks of
    256 and 512) with per-atom partial sums and the fused adjoint with per-cluster coefficients:
    moments equal the single-cluster calls to the FP64 grouping of the partial sums (1e-9·n),
    G and forces equal them to FP32 summation order, and energies, G and forces match the oracle."""
    from gpu_common import oracle_estimator_forces
    sizes, kTs = [37, 64, 21], [0.5, 0.1, 0.5]
    b = _batch(api, ctx, sizes, kTs, s=s)
    b = [(wk, H, e0, e1, min(p, 70 + 23 * i)) for i, (wk, H, e0, e1, p) in enumerate(b)]
    model = api.Solver(b[0][0], ctx).model
    Hs, e0, e1, seeds = [x[1] for x in b], [x[2] for x in b], [x[3] for x in b], [x[0].probe_seed for x in b]
    orders, ne = [x[4] for x in b], [x[0].n_electrons for x in b]
    pos = [torch.as_tensor(x[0].positions, dtype=torch.float64, device="cuda") for x in b]
    mom, obs, Gs, Fs = api.batched_energies_and_forces(ctx, Hs, model, pos, e0, e1, seeds, s, orders, ne,
                                                       kTs, want_G=True)
    for (wk, H, lo, hi, p), m, o, G, F, ps in zip(b, mom, obs, Gs, Fs, pos):
        n = wk.n_atoms * 9
        ref = api.chebyshev_moments(ctx, H, lo, hi, wk.probe_seed, s, p)
        assert np.abs(m.cpu().numpy() - ref.cpu().numpy()).max() < 1e-9 * n
        G1, F1 = api.density_and_forces(ctx, H, model, ps, None, lo, hi, wk.probe_seed, s, p, o[0],
                                        wk.kT, False, False, want_G=True)
        gmax = G1.abs().max().item()
        assert torch.allclose(G, G1, rtol=0, atol=2e-5 * gmax)
        assert torch.allclose(F, F1, rtol=0, atol=1e-4)
        rp, col, Hd = oracle_H(wk)
        est = oracle_estimator(wk, Hd, lo, hi, p)
        for j, key in ((1, "Omega"), (2, "E"), (3, "N")):
            assert abs(o[j] - est[key]) / wk.n_atoms < 1e-4, key
        _, Fo = oracle_estimator_forces(wk, rp, col, dict(est, mu=o[0]), lo, hi, p)
        assert np.abs(F.cpu().numpy() - Fo).max() < 1e-3


def test_batch_with_one_and_two_atom_clusters(api, ctx):
    """Degenerate members: a one-atom cluster (one 9 x 9 block, a 9-row Krylov space for the
    bounds) and a dimer next to a 37-atom cluster: bounds, moments, energies and forces equal the
    single-cluster calls, the energies and forces match the oracle, and the lone atom feels no force."""
    from gpu_common import oracle_estimator_forces
    sizes, kTs = [1, 2, 37], [0.5, 0.1, 0.5]
    b = _batch(api, ctx, sizes, kTs)
    b = [(wk, H, e0, e1, min(p, 80)) for (wk, H, e0, e1, p) in b]
    Hs = [x[1] for x in b]
    lo, hi = api.batched_spectral_bounds(ctx, Hs)
    for H, l_, h_ in zip(Hs, lo, hi):
        assert (l_, h_) == api.spectral_bounds(ctx, H)
    model = api.Solver(b[0][0], ctx).model
    e0, e1, seeds = [x[2] for x in b], [x[3] for x in b], [x[0].probe_seed for x in b]
    orders, ne = [x[4] for x in b], [x[0].n_electrons for x in b]
    pos = [torch.as_tensor(x[0].positions, dtype=torch.float64, device="cuda") for x in b]
    mom, obs, Gs, Fs = api.batched_energies_and_forces(ctx, Hs, model, pos, e0, e1, seeds, 128, orders, ne,
                                                       kTs, want_G=True)
    for (wk, H, l_, h_, p), m, o, G, F, ps in zip(b, mom, obs, Gs, Fs, pos):
        ref = api.chebyshev_moments(ctx, H, l_, h_, wk.probe_seed, 128, p)
        assert np.abs(m.cpu().numpy() - ref.cpu().numpy()).max() < 1e-9 * wk.n_atoms * 9
        rp, col, Hd = oracle_H(wk)
        est = oracle_estimator(wk, Hd, l_, h_, p)
        for j, key in ((1, "Omega"), (2, "E"), (3, "N")):
            assert abs(o[j] - est[key]) / wk.n_atoms < 1e-4, (wk.n_atoms, key)
        _, Fo = oracle_estimator_forces(wk, rp, col, dict(est, mu=o[0]), l_, h_, p)
        assert np.abs(F.cpu().numpy() - Fo).max() < 1e-3, wk.n_atoms
    assert np.abs(Fs[0].cpu().numpy()).max() < 1e-12
