"""Operand precision for tensor-core versions of the hot path, emulated on the CPU against the
oracle (no GPU).

The FP32 block products of the recurrence (Eq. poly_PQ) and the outer products of the adjoint
(Eq. polynomial_response, in the doubled-moment form) could move to the tensor cores. Their
operands would be TF32 (10 mantissa bits) or BF16 (7), used directly or split as a = hi + lo,
with products hi*hi' + hi*lo' + lo*hi' accumulated in FP32. This test emulates those formats
on a 100-atom cluster (operands rounded to nearest even, FP32 matrix products, panels stored in
FP32). It checks each format's energy and force errors against the oracle's exact estimator:
* the adjoint's outer products: three-term BF16 and TF32 splits stay within the force
  tolerance, and a single BF16 pass does not;
* the recurrence: the three-term TF32 split keeps FP32's accuracy, and a single TF32 pass
  misses the energy tolerance.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import chebyshev as ch, hamiltonian, neighbors, physics


def _round(a, bits):
    """float32 values rounded to `bits` explicit mantissa bits, to nearest even."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    drop = np.uint64(23 - bits)
    lsb = (u >> drop) & np.uint64(1)
    u = (u + (np.uint64(1) << (drop - np.uint64(1))) - np.uint64(1) + lsb) & ~((np.uint64(1) << drop) - np.uint64(1))
    return u.astype(np.uint32).view(np.float32)


def _trunc(a, bits):
    """float32 values with all but `bits` explicit mantissa bits cleared (rounded toward zero):
    what a TF32 tensor-core operation reads from an FP32 register or shared-memory word."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32)
    return (u & np.uint32((0xFFFFFFFF << (23 - bits)) & 0xFFFFFFFF)).view(np.float32)


def _mm(A, B, fmt):
    """A @ B with float32 operands in the emulated format; float32 result.  "tf32x3t" is the
    split as the tensor cores take it from FP32 words: head = truncation of the value, remainder
    = value - head (exact in FP32), and each operand read truncated to TF32 again."""
    A, B = A.astype(np.float32), B.astype(np.float32)
    if fmt == "fp32":
        return A @ B
    bits = {"tf32": 10, "bf16": 7}[fmt[:4]]
    q = _trunc if fmt.endswith("t") else _round
    Ah, Bh = q(A, bits), q(B, bits)
    out = Ah @ Bh
    if "x3" in fmt:
        out = out + Ah @ q(B - Bh, bits) + q(A - Ah, bits) @ Bh
    return out.astype(np.float32)


@pytest.fixture(scope="module")
def case():
    n_at, kT, s = 100, 0.5, 64
    wk = wl.fcc_cu(n_at, kT=kT, n_probes=s, seed=5264, probe_seed=777, jitter=0.05)
    rp, col = neighbors.neighbor_csr(wk.positions, wk.cutoff)
    H = hamiltonian.dense_sk(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE)
    w, V = np.linalg.eigh(H)
    W0 = w.max() - w.min()
    emin, emax = w.min() - 0.01 * W0, w.max() + 0.01 * W0
    p = max(64, int(np.ceil(((emax - emin) / kT) * np.log(1e7) / 6.4)))
    R = ch.probes(H.shape[0], s, wk.probe_seed)
    mom = ch.exact_moments(w, V, R, emin, emax, p)
    mu = ch.estimator_mu(mom, emin, emax, wk.n_electrons, kT)
    a, b, dH = hamiltonian.sk_bond_grads(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY)
    F = physics.forces_from_blocks(ch.estimator_gradient(w, V, R, emin, emax, mu, kT, p=p), a, b, dH, n_at, 9)
    Om = ch.estimator_observables(mom, emin, emax, mu, kT)[0]
    return dict(n_at=n_at, kT=kT, s=s, H=H, emin=emin, emax=emax, p=p, R=R, mu=mu, a=a, b=b, dH=dH,
                F=F, Om=Om)


def _run(c, rec_fmt, outer_fmt):
    """(Omega^, forces) of the doubled-moment estimator and its adjoint with the recurrence's
    products in rec_fmt and the outer products in outer_fmt."""
    H, emin, emax, p, R, s = c["H"], c["emin"], c["emax"], c["p"], c["R"], c["s"]
    n, W, K = H.shape[0], emax - emin, p // 2
    Hh = (2 * H - (emax + emin) * np.eye(n)) / W
    y = [R.astype(np.float32), _mm(Hh, R, rec_fmt)]
    for _ in range(1, K):
        y.append((np.float32(2) * _mm(Hh, y[-1], rec_fmt) - y[-2]).astype(np.float32))
    Y = [v.astype(np.float64) for v in y]
    mom = np.zeros(p)
    mom[0], mom[1] = n, np.sum(Y[1] * Y[0]) / s
    for k in range(1, K + 1):
        if 2 * k < p:
            mom[2 * k] = 2 * np.sum(Y[k] * Y[k]) / s - mom[0]
        if k >= 2 and 2 * k - 1 < p:
            mom[2 * k - 1] = 2 * np.sum(Y[k] * Y[k - 1]) / s - mom[1]
    Om = ch.estimator_observables(mom, emin, emax, c["mu"], c["kT"])[0]
    _, _, cg = ch.fd_coefficients(p, emin, emax, c["mu"], c["kT"])
    wgt, v = np.zeros(K + 2), np.zeros(K + 2)
    for k in range(1, K + 1):
        if 2 * k < p:
            wgt[k] = 2 * cg[2 * k]
        if k >= 2 and 2 * k - 1 < p:
            v[k] = 2 * cg[2 * k - 1]
    v[1] = cg[1] - sum(cg[2 * k - 1] for k in range(2, K + 1) if 2 * k - 1 < p)

    def g(k):
        out = 2 * wgt[k] * Y[k] + v[k] * Y[k - 1] + (v[k + 1] * Y[k + 1] if k < K else 0.0)
        return (out / s).astype(np.float32)
    yb = [None] * (K + 2)
    yb[K + 1], yb[K] = np.zeros_like(y[0]), g(K)
    for k in range(K - 1, 0, -1):
        yb[k] = (g(k) + np.float32(2) * _mm(Hh, yb[k + 1], rec_fmt) - yb[k + 2]).astype(np.float32)
    Gh = _mm(yb[1], y[0].T, outer_fmt).astype(np.float64)
    for k in range(1, K):
        Gh += 2 * _mm(yb[k + 1], y[k].T, outer_fmt).astype(np.float64)
    G = (1.0 / W) * (Gh + Gh.T)
    return Om, physics.forces_from_blocks(G, c["a"], c["b"], c["dH"], c["n_at"], 9)


def _errors(c, rec_fmt, outer_fmt):
    Om, F = _run(c, rec_fmt, outer_fmt)
    return abs(Om - c["Om"]) / c["n_at"], np.abs(F - c["F"]).max()


def test_fp32_emulation_reproduces_the_mixed_path_accuracy(case):
    e, f = _errors(case, "fp32", "fp32")
    assert e < 1e-5 and f < 1e-5               # the FP32 path's level (tolerances 1e-4, 1e-3)


@pytest.mark.parametrize("fmt,ok", [("bf16x3", True), ("tf32x3", True), ("tf32x3t", True),
                                    ("bf16", False)])
def test_outer_product_formats(case, fmt, ok):
    _, f = _errors(case, "fp32", fmt)
    assert (f < 1e-3) == ok, f
    if fmt in ("bf16x3", "tf32x3t"):
        assert f < 1e-4                          # an order of magnitude inside the tolerance


@pytest.mark.parametrize("fmt,ok", [("tf32x3", True), ("tf32x3t", True), ("tf32", False),
                                    ("tf32t", False)])
def test_recurrence_formats(case, fmt, ok):
    e, f = _errors(case, fmt, "fp32")
    assert (e < 1e-4 and f < 1e-3) == ok, (e, f)
    if fmt in ("tf32x3", "tf32x3t"):
        assert e < 1e-5 and f < 1e-5             # as accurate as FP32


def test_rounding_helper():
    one = np.float32(1.0)
    u = 2.0 ** -10                                   # TF32 spacing at 1
    vals = np.array([1 + u / 2, 1 + 3 * u / 2, 1 + u / 2 + 2.0 ** -20, -(1 + 3 * u / 2), 2 - u / 4],
                    dtype=np.float32)
    got = _round(vals, 10)
    assert got.tolist() == [1.0, 1 + 2 * u, 1 + u, -(1 + 2 * u), 2.0]   # ties to even; carry
    assert _round(np.float32(3.0), 7) == np.float32(3.0) and _round(one, 10) == one
    b = _round(np.float32(1 + 2.0 ** -8 + 2.0 ** -12), 7)            # BF16 spacing 2^-7
    assert b == np.float32(1.0 + 2.0 ** -7)
    t = _trunc(np.array([1 + 3 * u / 2, -(1 + 3 * u / 2), 2 - u / 4, 1 + u], dtype=np.float32), 10)
    assert t.tolist() == [1 + u, -(1 + u), 2 - u, 1 + u]             # toward zero, exact kept
