"""f1: the multi-colour probe ensemble (Sec. II.C.3, colours by Welsh-Powell, Sec. II.E) on the GPU,
through the C ABI, against the oracle's exact value of the same estimator.

Checks: moments (FP64 1e-11 n, mixed 1e-5 n); one-call energies (1e-4 eV/atom), every entry of
the sampled density matrix (2e-5 of max|G|, as for the plain probes) and forces (1e-3 eV/A) with
the fused and the windowed adjoint at panel widths 128, 256 and 512; special cases that fix the
result independently of the oracle: one colour of a 1-orbital model is the plain Rademacher
estimator, and a radius beyond the cluster (every atom its own colour) gives the exact
polynomial trace from a single sample.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import chebyshev as och, coloring as oco, hamiltonian as oham, physics as oph

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


def _setup(api, ctx, wk, r_color):
    model = api.Model.from_workload(wk, torch.device("cuda"))
    pos = _dev(wk.positions)
    g = api.build_neighbors(ctx, pos, wk.cutoff)
    H = api.assemble_H(ctx, model, pos, g)
    emin, emax = api.spectral_bounds(ctx, H)
    ac = oco.atom_colors(wk.positions, r_color)
    return model, pos, H, emin, emax, ac, int(ac.max()) + 1


def _oracle(wk, Hd, ac, n_samples, emin, emax, p):
    w, V = np.linalg.eigh(Hd)
    fc = oco.function_colors(ac, wk.n_orb)
    q = (int(ac.max()) + 1) * wk.n_orb
    R = och.probes(Hd.shape[0], n_samples, wk.probe_seed)
    Rc = oco.colored_probes(fc, q, R)
    mom = oco.exact_colored_moments(w, V, Rc, n_samples, emin, emax, p)
    return w, V, Rc, mom


@pytest.mark.parametrize("r_color,n_samples", [(4.5, 1), (6.0, 1), (6.0, 3)])
@pytest.mark.parametrize("fp64", [True, False])
def test_colored_moments_vs_oracle(api, ctx, r_color, n_samples, fp64):
    wk = wl.fcc_cu(60, kT=0.5, n_probes=8, seed=5264, probe_seed=4242, jitter=0.05)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax, ac, qa = _setup(api, ctx, wk, r_color)
    S = api.colored_columns(qa, 9, n_samples)
    p = 120
    mom = api.colored_moments(ctx, H, emin, emax, wk.probe_seed, ac, qa, n_samples, S, p, fp64=fp64)
    _, _, _, ref = _oracle(wk, Hd, ac, n_samples, emin, emax, p)
    n = Hd.shape[0]
    assert np.abs(mom.cpu().numpy() - ref).max() < (1e-11 if fp64 else 1e-5) * n


@pytest.mark.parametrize("r_color,n_samples,windowed", [(4.5, 1, False), (4.5, 1, True), (4.5, 1, "tensor"),
                                                        (6.0, 1, False), (6.0, 1, True), (6.0, 1, "tensor"),
                                                        (6.0, 3, False), (6.0, 3, True), (6.0, 3, "tensor")])
def test_colored_energies_G_and_forces_vs_oracle(api, ctx, r_color, n_samples, windowed):
    wk = wl.fcc_cu(60, kT=0.5, n_probes=8, seed=5264, probe_seed=4242, jitter=0.05)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax, ac, qa = _setup(api, ctx, wk, r_color)
    S = api.colored_columns(qa, 9, n_samples)
    assert S in (128, 256, 512)
    p = 90
    mom, obs, G, F = api.colored_energies_and_forces(
        ctx, H, model, pos, None, emin, emax, wk.probe_seed, ac, qa, n_samples, S, p,
        wk.n_electrons, wk.kT, want_G=True, windowed=windowed)
    w, V, Rc, ref = _oracle(wk, Hd, ac, n_samples, emin, emax, p)
    n = wk.n_atoms
    assert np.abs(mom.cpu().numpy() - ref).max() < 1e-5 * n * 9
    mu = och.estimator_mu(ref, emin, emax, wk.n_electrons, wk.kT)
    Om, E, N = och.estimator_observables(ref, emin, emax, mu, wk.kT)
    assert abs(obs[0] - mu) < 1e-4
    for got, want in zip(obs[1:], (Om, E, N)):
        assert abs(got - want) / n < 1e-4
    Gd = oco.colored_estimator_gradient(w, V, Rc, n_samples, emin, emax, obs[0], wk.kT, p)
    ref_b = blocks_of(Gd, rp, col, 9)
    err = np.abs(G.cpu().numpy() - ref_b).max() / np.abs(ref_b).max()
    assert err < 2e-5, err
    a, b, dH = oham.sk_bond_grads(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY)
    Fo = oph.forces_from_blocks(Gd, a, b, dH, n, 9)
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-3


def test_colored_panel_padding_does_not_change_the_result(api, ctx):
    """The same ensemble on a 256- and a 512-column panel: the extra columns are zero."""
    wk = wl.fcc_cu(60, kT=0.5, n_probes=8, seed=5264, probe_seed=4242, jitter=0.05)
    model, pos, H, emin, emax, ac, qa = _setup(api, ctx, wk, 6.0)
    p = 90
    outs = [api.colored_energies_and_forces(ctx, H, model, pos, None, emin, emax, wk.probe_seed, ac, qa, 1,
                                            S, p, wk.n_electrons, wk.kT, want_G=True) for S in (256, 512)]
    n = wk.n_atoms * 9
    assert np.abs(outs[0][0].cpu().numpy() - outs[1][0].cpu().numpy()).max() < 1e-9 * n
    g0 = outs[0][2].cpu().numpy()
    assert np.abs(g0 - outs[1][2].cpu().numpy()).max() < 1e-6 * np.abs(g0).max()


def test_one_colour_of_a_one_orbital_model_is_the_plain_estimator(api, ctx):
    """n_orb = 1 and a single colour: sample i is probe column i of the plain Rademacher block."""
    wk = wl.sc_disorder(L=6, n_probes=8)
    s = api.Solver(wk, ctx)
    pos = _dev(wk.positions)
    g = api.build_neighbors(ctx, pos, wk.cutoff)
    H = api.assemble_H(ctx, s.model, pos, g)
    emin, emax = api.spectral_bounds(ctx, H)
    ac = np.zeros(wk.n_atoms, dtype=np.int32)
    for fp64 in (True, False):
        ref = api.chebyshev_moments(ctx, H, emin, emax, wk.probe_seed, 8, 100, fp64=fp64).cpu().numpy()
        got = api.colored_moments(ctx, H, emin, emax, wk.probe_seed, ac, 1, 8, 8, 100, fp64=fp64).cpu().numpy()
        assert np.abs(got - ref).max() < (1e-12 if fp64 else 1e-6) * wk.n_atoms


def test_radius_beyond_the_cluster_gives_the_exact_trace(api, ctx):
    """Every atom its own colour: each column of the one sample is a signed unit vector, so
    (1/1) sum_columns r^T C_k(H^) r = tr C_k(H^) exactly."""
    wk = wl.fcc_cu(13, kT=0.5, n_probes=8, seed=5264, probe_seed=77, jitter=0.05)
    rp, col, Hd = oracle_H(wk)
    model, pos, H, emin, emax, ac, qa = _setup(api, ctx, wk, 100.0)
    assert qa == wk.n_atoms
    p = 150
    mom = api.colored_moments(ctx, H, emin, emax, wk.probe_seed, ac, qa, 1, 128, p, fp64=True)
    w = np.linalg.eigvalsh(Hd)
    exact = och.cheb_T(och.mapped(w, emin, emax), p).sum(axis=1)
    assert np.abs(mom.cpu().numpy() - exact).max() < 1e-11 * len(w)


def test_colored_argument_errors(api, ctx):
    from paper_1812_05264_gb300._lib import TBK_ERR_ARG, TbkError
    wk = wl.fcc_cu(30, kT=0.5, n_probes=8, seed=5264, probe_seed=1)
    model, pos, H, emin, emax, ac, qa = _setup(api, ctx, wk, 4.5)
    bad = ac.copy()
    bad[3] = qa                                   # a colour outside [0, n_colors)
    with pytest.raises(TbkError) as e:
        api.colored_moments(ctx, H, emin, emax, 1, bad, qa, 1, 128, 20)
    assert e.value.code == TBK_ERR_ARG
    with pytest.raises(TbkError) as e:            # fewer columns than one sample needs
        api.colored_moments(ctx, H, emin, emax, 1, ac, qa, 2, 8, 20)
    assert e.value.code == TBK_ERR_ARG
    with pytest.raises(TbkError) as e:            # the coloured adjoint wants 128/256/512 columns
        api.colored_energies_and_forces(ctx, H, model, pos, None, emin, emax, 1, ac, qa, 1, 4 * ((qa * 9 + 3) // 4),
                                        50, wk.n_electrons, wk.kT)
    assert e.value.code == TBK_ERR_ARG
    # the context stays usable
    ok = api.colored_moments(ctx, H, emin, emax, 1, ac, qa, 1, 128, 20)
    assert torch.isfinite(ok).all()
