"""Shared helpers of the GPU parity tests: run the oracle on the same seeded inputs."""
import numpy as np

import workloads as wl
from oracle import chebyshev as och
from oracle import hamiltonian as oham
from oracle import neighbors as onb
from oracle import physics as oph


def small_fcc(n_atoms=40, kT=0.5, n_probes=16, jitter=0.05, seed=11, order=None, mixed=False):
    wk = wl.fcc_cu(n_atoms, kT, n_probes, seed=5264, probe_seed=seed, jitter=jitter, order=order,
                   mixed=mixed)
    return wk


def oracle_H(wk):
    rp, col = onb.neighbor_csr(wk.positions, wk.cutoff, wk.box)
    if wk.sk_V is not None:
        H = oham.dense_sk(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE, wk.box)
    else:
        H = oham.dense_table(wk.positions, rp, col, wk.n_orb, wk.disp, wk.blocks, wk.onsite_site,
                             wk.box)
    return rp, col, H


def oracle_estimator(wk, H, emin, emax, p):
    """Exact estimator quantities for the GPU's probes, order p and bounds."""
    w, V = np.linalg.eigh(H)
    R = och.probes(H.shape[0], wk.n_probes, wk.probe_seed)
    mom = och.exact_moments(w, V, R, emin, emax, p)
    mu = och.estimator_mu(mom, emin, emax, wk.n_electrons, wk.kT, wk.jackson)
    Om, E, N = och.estimator_observables(mom, emin, emax, mu, wk.kT, wk.jackson)
    return dict(w=w, V=V, R=R, moments=mom, mu=mu, Omega=Om, E=E, N=N)


def oracle_estimator_forces(wk, rp, col, est, emin, emax, p):
    G = och.estimator_gradient(est["w"], est["V"], est["R"], emin, emax, est["mu"], wk.kT,
                               wk.jackson, p=p)
    a, b, dH = oham.sk_bond_grads(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY, wk.box)
    F = oph.forces_from_blocks(G, a, b, dH, wk.n_atoms, 9)
    return G, F


def blocks_of(Gdense, rp, col, b):
    n = len(rp) - 1
    out = np.zeros((len(col), b, b))
    for a in range(n):
        for k in range(rp[a], rp[a + 1]):
            c = col[k]
            out[k] = Gdense[b * a:b * a + b, b * c:b * c + b]
    return out
