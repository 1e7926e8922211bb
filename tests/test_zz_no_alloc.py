"""The allocation-free moments entry point (tbk_chebyshev_moments_noalloc), called through the C
ABI, against the regular entry point on the same inputs.

Some callers cannot allocate device memory while they run (latency-bounded loops, frameworks
that own every device allocation); this variant takes its scratch from a fixed static device
array instead.  The file is named so that pytest collects it last: if it fails, a run that stops
at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_1812_05264_gb300 import build
    build.build()
    from paper_1812_05264_gb300 import _lib, api
    ctx = api.Context()
    return _lib, api, ctx


def _problem(api, ctx, n_atoms, n_probes, seed=5):
    wk = wl.fcc_cu(n_atoms, kT=0.5, n_probes=n_probes, jitter=0.05, seed=5264, probe_seed=seed)
    sv = api.Solver(wk, ctx)
    pos = torch.as_tensor(wk.positions, dtype=torch.float64, device="cuda")
    g = api.build_neighbors(ctx, pos, wk.cutoff)
    H = api.assemble_H(ctx, sv.model, pos, g)
    emin, emax = api.spectral_bounds(ctx, H)
    return wk, H, emin, emax


def _noalloc(L, ctx, H, emin, emax, seed, s, order, flags):
    out = torch.empty(order, dtype=torch.float64, device="cuda")
    L.call("tbk_chebyshev_moments_noalloc", ctx.handle, C.byref(H.struct()), emin, emax,
           C.c_uint64(seed), s, order, flags, out.data_ptr())
    return out


@pytest.mark.parametrize("s,fp64", [(128, False), (512, False), (16, True)])
def test_noalloc_matches_regular_entry_point_twice(setup, s, fp64):
    L, api, ctx = setup
    wk, H, emin, emax = _problem(api, ctx, 90, s)
    order = 121
    flags = L.TBK_FP64 if fp64 else L.TBK_MIXED
    ref = api.chebyshev_moments(ctx, H, emin, emax, wk.probe_seed, s, order, fp64=fp64).cpu().numpy()
    n = H.graph.n_atoms * 9
    tol = 1e-11 * n if fp64 else 1e-9 * n
    for _ in range(2):   # the static array keeps the previous call's contents
        got = _noalloc(L, ctx, H, emin, emax, wk.probe_seed, s, order, flags).cpu().numpy()
        assert np.abs(got - ref).max() <= tol


def test_noalloc_rejects_problems_above_the_static_size(setup):
    L, api, ctx = setup
    wk, H, emin, emax = _problem(api, ctx, 400, 4096)   # two FP32 panels of 59 MB: over the limit
    with pytest.raises(L.TbkError) as e:
        _noalloc(L, ctx, H, emin, emax, wk.probe_seed, 4096, 20, L.TBK_MIXED)
    assert e.value.code == L.TBK_ERR_ARG
    assert "static limit" in str(e.value)
    # the context still works afterwards
    ok = _noalloc(L, ctx, H, emin, emax, wk.probe_seed, 128, 20, L.TBK_MIXED)
    assert torch.isfinite(ok).all()


def test_noalloc_on_a_fresh_context_allocates_nothing(setup):
    """On a context that no regular call has touched (so none of its scratch slots exist), after
    one warm call the allocation-free entry point leaves the device's free memory unchanged, with
    the kernel timer switched on (timing would create CUDA events)."""
    L, api, ctx0 = setup
    wk, H, emin, emax = _problem(api, ctx0, 90, 512)
    ref = api.chebyshev_moments(ctx0, H, emin, emax, wk.probe_seed, 512, 61).cpu().numpy()
    ctx = api.Context()
    try:
        ctx.time_kernels("step", "backward", "window")
        out = torch.empty(61, dtype=torch.float64, device="cuda")

        def call():
            L.call("tbk_chebyshev_moments_noalloc", ctx.handle, C.byref(H.struct()), emin, emax,
                   C.c_uint64(wk.probe_seed), 512, 61, L.TBK_MIXED, out.data_ptr())
            torch.cuda.synchronize()

        call()
        free0, _ = torch.cuda.mem_get_info()
        call()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert ctx.kernel_time("step") == (0.0, 0)
        n = H.graph.n_atoms * 9
        assert np.abs(out.cpu().numpy() - ref).max() <= 1e-9 * n
    finally:
        ctx.close()
