"""Pins for the host FP64 block-sparse recurrence (oracle/o2.py; CPU only): its moments equal the
oracle's exact estimator (eigen route) and its dense-matrix recurrence, directly and through the
doubling identities, for 9 x 9 and 1 x 1 blocks; they do not depend on the thread count."""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as wl
from oracle import chebyshev as ch, hamiltonian, neighbors, o2


def _bsr(wk):
    rp, col = neighbors.neighbor_csr(wk.positions, wk.cutoff, wk.box)
    if wk.sk_V is not None:
        Hd = hamiltonian.dense_sk(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)
    else:
        Hd = hamiltonian.dense_table(wk.positions, rp, col, wk.n_orb, wk.disp, wk.blocks, wk.onsite_site,
                                     wk.box)
    B = wk.n_orb
    blocks = np.array([Hd[B * a:B * a + B, B * c:B * c + B] for a in range(len(rp) - 1)
                       for c in col[rp[a]:rp[a + 1]]])
    return rp, col, blocks, Hd


@pytest.mark.parametrize("which", ["fcc", "sc"])
@pytest.mark.parametrize("doubled", [False, True])
def test_o2_moments_equal_the_exact_estimator(which, doubled):
    wk = (wl.fcc_cu(40, kT=0.5, n_probes=12, seed=5264, probe_seed=9, jitter=0.05) if which == "fcc"
          else wl.sc_disorder(L=5, n_probes=12))
    rp, col, blocks, Hd = _bsr(wk)
    w, V = np.linalg.eigh(Hd)
    emin, emax = w.min() - 0.3, w.max() + 0.3
    p = 71
    mom, n = o2.moments(rp, col, blocks, emin, emax, wk.probe_seed, 12, p, doubled)
    R = ch.probes(Hd.shape[0], 12, wk.probe_seed)
    ref = ch.exact_moments(w, V, R, emin, emax, p)
    assert n == (p // 2 if doubled else p - 1)
    assert np.abs(mom - ref).max() < 1e-11 * Hd.shape[0]
    rec = ch.recurrence_probe_moments(Hd, R, emin, emax, p).mean(axis=1)
    assert np.abs(mom - rec).max() < 1e-11 * Hd.shape[0]


def test_o2_moments_do_not_depend_on_the_thread_count():
    code = ("import sys; sys.path.insert(0, %r); import numpy as np, workloads as wl; "
            "from oracle import neighbors, hamiltonian, o2; "
            "wk = wl.fcc_cu(60, kT=0.5, n_probes=8, seed=5264, probe_seed=3, jitter=0.05); "
            "rp, col = neighbors.neighbor_csr(wk.positions, wk.cutoff); "
            "Hd = hamiltonian.dense_sk(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE); "
            "b = np.array([Hd[9*a:9*a+9, 9*c:9*c+9] for a in range(len(rp)-1) for c in col[rp[a]:rp[a+1]]]); "
            "m, _ = o2.moments(rp, col, b, -30.0, 40.0, 3, 8, 50, True); print(repr(m.tolist()))"
            % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    outs = []
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                   check=True).stdout)
    assert outs[0] == outs[1]
