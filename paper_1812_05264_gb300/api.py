"""PyTorch-facing wrappers of libtbk: device memory and streams come from torch, every step of
the computation runs in the library's CUDA kernels.

Pipeline (arXiv 1812.05264, Sec. II): neighbour list -> H assembly -> spectral bounds ->
Chebyshev moments with random probes -> chemical potential and Omega, E, N -> analytic adjoint
giving the sampled density matrix dOmega/dH on the pattern and the forces.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


class Context:
    """A libtbk context bound to one CUDA device and the torch stream current at creation."""

    def __init__(self, device: int | None = None, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libtbk needs a CUDA device")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._h = C.c_void_p()
        L.call("tbk_create", C.byref(self._h), self.device, C.c_void_p(self.stream.cuda_stream))

    @property
    def handle(self):
        return self._h

    @property
    def launches(self) -> int:
        return int(L.load().tbk_launch_count(self._h))

    _FAMILIES = {"step": L.TBK_KERNEL_STEP, "backward": L.TBK_KERNEL_BACKWARD,
                 "window": L.TBK_KERNEL_WINDOW}

    def time_kernels(self, *families: str):
        """Bracket every launch of the named kernel families ("step": one recurrence step,
        "backward": one adjoint step, "window": the outer products of a window of steps) with CUDA
        events on this context's stream; no names switches timing off.  Read with kernel_time()."""
        mask = 0
        for f in families:
            mask |= 1 << self._FAMILIES[f]
        L.call("tbk_kernel_timer", self._h, mask)

    def kernel_time(self, family: str) -> tuple[float, int]:
        """(total milliseconds, launches) of one family since time_kernels()."""
        ms, n = C.c_double(), C.c_int64()
        L.call("tbk_kernel_timer_read", self._h, self._FAMILIES[family], C.byref(ms), C.byref(n))
        return ms.value, n.value

    def close(self):
        if self._h:
            L.load().tbk_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Graph:
    n_atoms: int
    nnzb: int
    row_ptr: torch.Tensor   # int32 (n_atoms + 1,)
    col: torch.Tensor       # int32 (nnzb,)


@dataclass
class BSR:
    graph: Graph
    n_orb: int
    val: torch.Tensor       # float64 (nnzb, n_orb, n_orb)

    def struct(self) -> L.tbk_bsr:
        return L.tbk_bsr(self.graph.n_atoms, self.n_orb, self.graph.nnzb,
                         _ptr(self.graph.row_ptr), _ptr(self.graph.col), _ptr(self.val))


class Model:
    """A tbk_model plus the arrays it points to (kept alive with it)."""

    def __init__(self, kind: int, n_orb: int, sk_V=None, r0=2.55, decay=2.0, onsite_spd=(0, 0, 0),
                 disp=None, blocks=None, tol=1e-6, onsite_site: torch.Tensor | None = None):
        self.s = L.tbk_model()
        self.s.kind = kind
        self.s.n_orb = n_orb
        if sk_V is not None:
            for i in range(10):
                self.s.sk_V[i] = float(sk_V[i])
        self.s.sk_r0 = r0
        self.s.sk_decay = decay
        for i in range(3):
            self.s.onsite_spd[i] = float(onsite_spd[i])
        self._disp = None if disp is None else np.ascontiguousarray(disp, dtype=np.float64)
        self._blocks = None if blocks is None else np.ascontiguousarray(blocks, dtype=np.float64)
        self.s.n_disp = 0 if disp is None else int(self._disp.shape[0])
        self.s.disp = None if disp is None else self._disp.ctypes.data
        self.s.disp_blocks = None if blocks is None else self._blocks.ctypes.data
        self.s.disp_tol = tol
        self._onsite = onsite_site
        self.s.onsite_site = _ptr(onsite_site)

    @property
    def is_sk(self) -> bool:
        return self.s.kind == L.TBK_MODEL_SK

    @staticmethod
    def from_workload(wk, device) -> "Model":
        import workloads as wl
        if wk.sk_V is not None:
            return Model(L.TBK_MODEL_SK, 9, sk_V=wk.sk_V, r0=wl.SK_R0, decay=wl.SK_DECAY,
                         onsite_spd=wl.SK_ONSITE)
        ons = None
        if wk.onsite_site is not None:
            a = np.asarray(wk.onsite_site, np.float64).reshape(wk.n_atoms, -1)
            ons = torch.as_tensor(np.broadcast_to(a, (wk.n_atoms, wk.n_orb)).copy(), device=device)
        return Model(L.TBK_MODEL_TABLE, wk.n_orb, disp=wk.disp, blocks=wk.blocks, onsite_site=ons)


def _box_arg(box):
    if box is None:
        return None, None
    arr = (C.c_double * 3)(*[float(x) for x in box])
    return arr, C.cast(arr, C.c_void_p)


SCHEDULES = ("fused", "windowed", "tensor")


def _schedule_flag(windowed) -> int:
    """The adjoint's outer-product schedule: None = the tuned one (else fused); True / False =
    windowed / fused; or a name from SCHEDULES ("tensor": on the tensor cores after each step)."""
    if windowed is None:
        return 0
    if isinstance(windowed, str):
        return {"fused": L.TBK_FUSED_ADJOINT, "windowed": L.TBK_WINDOWED,
                "tensor": L.TBK_TC_OUTER}[windowed]
    return L.TBK_WINDOWED if windowed else L.TBK_FUSED_ADJOINT


def build_neighbors(ctx: Context, pos: torch.Tensor, cutoff: float, box=None) -> Graph:
    """a1: CSR of all pairs with |r_j - r_i| <= cutoff (self included), ascending columns."""
    assert pos.is_cuda and pos.dtype == torch.float64 and pos.is_contiguous()
    n = pos.shape[0]
    row_ptr = torch.empty(n + 1, dtype=torch.int32, device=pos.device)
    nnz = C.c_int64()
    _keep, bx = _box_arg(box)
    # a first capacity that holds every short-cutoff pattern in practice; the call reports the
    # exact count, and a pattern that does not fit is built again with it
    col = torch.empty(max(1, 32 * n), dtype=torch.int32, device=pos.device)
    try:
        L.call("tbk_build_neighbors", ctx.handle, _ptr(pos), n, bx, float(cutoff), _ptr(row_ptr),
               _ptr(col), col.numel(), C.byref(nnz))
    except L.TbkError as e:
        if e.code != L.TBK_ERR_ARG or nnz.value <= col.numel():
            raise
        col = torch.empty(nnz.value, dtype=torch.int32, device=pos.device)
        L.call("tbk_build_neighbors", ctx.handle, _ptr(pos), n, bx, float(cutoff), _ptr(row_ptr),
               _ptr(col), col.numel(), C.byref(nnz))
    return Graph(n, nnz.value, row_ptr, col[:nnz.value])


def welsh_powell(row_ptr: np.ndarray, col: np.ndarray) -> tuple[np.ndarray, int]:
    """Welsh-Powell colours of a symmetric CSR graph (host int32 arrays, ascending columns, self
    entries ignored) and their number; the library's host colouring (Sec. II.E)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    n = rp.size - 1
    color = np.empty(max(n, 1), dtype=np.int32)
    q = C.c_int32()
    L.call("tbk_welsh_powell", n, rp.ctypes.data, cl.ctypes.data if cl.size else None,
           color.ctypes.data, C.byref(q))
    return color[:n], q.value


def atom_colors(ctx: Context, pos: torch.Tensor, r_color: float, box=None) -> tuple[np.ndarray, int]:
    """Colours of the atoms for the multi-colour probe ensemble (Sec. II.C.3): the neighbour
    pattern at the colouring radius built on the device, coloured by Welsh-Powell on the host,
    so that two atoms of one colour are farther apart than r_color."""
    g = build_neighbors(ctx, pos, r_color, box)
    return welsh_powell(g.row_ptr.cpu().numpy(), g.col.cpu().numpy())


def colored_columns(n_colors: int, n_orb: int, n_samples: int = 1) -> int:
    """Panel width for the multi-colour ensemble: n_samples * n_colors * n_orb columns, rounded up
    to a multiple of 128 (the width the TMA-fed and fused kernels take) up to 512, else to 4."""
    need = n_samples * n_colors * n_orb
    for w in (128, 256, 512):
        if need <= w:
            return w
    return (need + 3) // 4 * 4


def colored_moments(ctx: Context, H: BSR, emin: float, emax: float, seed: int, atom_color,
                    n_colors: int, n_samples: int, n_columns: int, order: int,
                    fp64: bool = False, plain: bool = False) -> torch.Tensor:
    """f1: moments of the multi-colour probe ensemble (Sec. II.C.3), divided by n_samples."""
    col = torch.as_tensor(np.ascontiguousarray(atom_color), dtype=torch.int32, device=H.val.device)
    out = torch.empty(order, dtype=torch.float64, device=H.val.device)
    flags = (L.TBK_FP64 if fp64 else L.TBK_MIXED) | (L.TBK_PLAIN_KERNEL if plain else 0)
    L.call("tbk_colored_moments", ctx.handle, C.byref(H.struct()), emin, emax, C.c_uint64(seed),
           _ptr(col), int(n_colors), int(n_samples), int(n_columns), int(order), flags, _ptr(out))
    return out


def colored_energies_and_forces(ctx: Context, H: BSR, model: Model, pos: torch.Tensor, box,
                                emin: float, emax: float, seed: int, atom_color, n_colors: int,
                                n_samples: int, n_columns: int, order: int, n_electrons: float,
                                kT: float, jackson: bool = False, want_G: bool = False,
                                want_forces: bool = True, max_panel_bytes: int = 0,
                                windowed: bool | None = None):
    """f1, a5-a10 in one call for the multi-colour ensemble: (moments, (mu, Omega, E, N), G or
    None, forces or None)."""
    dev = H.val.device
    col = torch.as_tensor(np.ascontiguousarray(atom_color), dtype=torch.int32, device=dev)
    mom = torch.empty(order, dtype=torch.float64, device=dev)
    G = torch.empty_like(H.val) if want_G else None
    F = torch.empty((H.graph.n_atoms, 3), dtype=torch.float64, device=dev) if want_forces else None
    obs = (C.c_double * 4)()
    _keep, bx = _box_arg(box)
    L.call("tbk_colored_energies_and_forces", ctx.handle, C.byref(H.struct()),
           C.byref(model.s) if model is not None else None, _ptr(pos), bx, emin, emax,
           C.c_uint64(seed), _ptr(col), int(n_colors), int(n_samples), int(n_columns), int(order),
           float(n_electrons), float(kT), L.TBK_DAMP_JACKSON if jackson else L.TBK_DAMP_NONE,
           _schedule_flag(windowed), int(max_panel_bytes), _ptr(mom), obs, _ptr(G), _ptr(F))
    return mom, tuple(obs[:]), G, F


def batched_build_neighbors(ctx: Context, positions: list, cutoff: float) -> list:
    """a1 for many open clusters in one call: the patterns of build_neighbors, cluster by
    cluster, with every pass run once over all the clusters' atoms."""
    n = len(positions)
    for p in positions:
        assert p.is_cuda and p.dtype == torch.float64 and p.is_contiguous() and p.shape[0] >= 1
    dev = positions[0].device
    rps = [torch.empty(p.shape[0] + 1, dtype=torch.int32, device=dev) for p in positions]
    pos_p = (C.c_void_p * n)(*[p.data_ptr() for p in positions])
    n_at = (C.c_int32 * n)(*[p.shape[0] for p in positions])
    rp_p = (C.c_void_p * n)(*[r.data_ptr() for r in rps])
    nnz = (C.c_int64 * n)()
    # a first capacity that holds every short-cutoff pattern in practice; the call reports the
    # exact counts, and a cluster that does not fit is built again with them
    cols = [torch.empty(32 * p.shape[0], dtype=torch.int32, device=dev) for p in positions]
    for attempt in range(2):
        col_p = (C.c_void_p * n)(*[c.data_ptr() for c in cols])
        cap = (C.c_int64 * n)(*[c.numel() for c in cols])
        try:
            L.call("tbk_batched_build_neighbors", ctx.handle, n, pos_p, n_at, float(cutoff), rp_p, col_p,
                   cap, nnz)
            break
        except L.TbkError as e:
            if attempt or e.code != L.TBK_ERR_ARG or all(nnz[i] <= cols[i].numel() for i in range(n)):
                raise
            cols = [torch.empty(max(1, nnz[i]), dtype=torch.int32, device=dev) for i in range(n)]
    return [Graph(positions[i].shape[0], nnz[i], rps[i], cols[i][:nnz[i]]) for i in range(n)]


def assemble_H(ctx: Context, model: Model, pos: torch.Tensor, graph: Graph, box=None) -> BSR:
    """a2: BSR values of H on the neighbour pattern."""
    b = model.s.n_orb
    val = torch.empty((max(1, graph.nnzb), b, b), dtype=torch.float64, device=pos.device)
    _keep, bx = _box_arg(box)
    L.call("tbk_assemble_H", ctx.handle, C.byref(model.s), _ptr(pos), graph.n_atoms, bx,
           _ptr(graph.row_ptr), _ptr(graph.col), graph.nnzb, _ptr(val))
    return BSR(graph, b, val[:graph.nnzb])


def spectral_bounds(ctx: Context, H: BSR, steps: int = 64, margin: float = 0.01,
                    seed: int = 0x5EED) -> tuple[float, float]:
    """a3: [emin, emax] enclosing the spectrum (Lanczos + residual + relative margin)."""
    lo, hi = C.c_double(), C.c_double()
    L.call("tbk_spectral_bounds", ctx.handle, C.byref(H.struct()), int(steps), float(margin),
           C.c_uint64(seed), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def batched_spectral_bounds(ctx: Context, Hs: list, steps: int = 64, margin: float = 0.01,
                            seed: int = 0x5EED) -> tuple[list, list]:
    """a3 for a batch: per-cluster [emin, emax], the Lanczos steps of all clusters together."""
    n = len(Hs)
    structs = (L.tbk_bsr * n)(*[h.struct() for h in Hs])
    lo, hi = (C.c_double * n)(), (C.c_double * n)()
    L.call("tbk_batched_spectral_bounds", ctx.handle, n, structs, int(steps), float(margin),
           C.c_uint64(seed), lo, hi)
    return list(lo), list(hi)


def autotune(ctx: Context, H: BSR, emin: float, emax: float, n_probes: int) -> tuple[int, str]:
    """Time the recurrence step's probe chunk and the adjoint's outer-product schedule on this
    operator and keep the fastest in the context for its shape: (probes per task, schedule name
    from SCHEDULES)."""
    out = (C.c_int32 * 2)()
    L.call("tbk_autotune", ctx.handle, C.byref(H.struct()), float(emin), float(emax), int(n_probes), out)
    return int(out[0]), SCHEDULES[int(out[1])]


def chebyshev_coefficients(ctx: Context, fn: int, order: int, emin: float, emax: float, mu: float,
                           kT: float, jackson: bool = False, device=None) -> torch.Tensor:
    """a4: damped Chebyshev coefficients of f, e f or g on [emin, emax]."""
    out = torch.empty(order, dtype=torch.float64, device=device or f"cuda:{ctx.device}")
    L.call("tbk_chebyshev_coefficients", ctx.handle, fn, order, emin, emax, mu, kT,
           L.TBK_DAMP_JACKSON if jackson else L.TBK_DAMP_NONE, _ptr(out))
    return out


def chebyshev_moments(ctx: Context, H: BSR, emin: float, emax: float, seed: int, n_probes: int,
                      order: int, fp64: bool = False, direct: bool = False,
                      out: torch.Tensor | None = None, plain: bool = False,
                      tensor_cores: bool = False) -> torch.Tensor:
    """a5-a7: mu_k = (1/s) sum_i r_i^T C_k(H^) r_i for k < order."""
    if out is None:
        out = torch.empty(order, dtype=torch.float64, device=H.val.device)
    flags = ((L.TBK_FP64 if fp64 else L.TBK_MIXED) | (L.TBK_MOMENTS_DIRECT if direct else 0)
             | (L.TBK_PLAIN_KERNEL if plain else 0) | (L.TBK_TENSOR_CORES if tensor_cores else 0))
    L.call("tbk_chebyshev_moments", ctx.handle, C.byref(H.struct()), emin, emax, C.c_uint64(seed),
           int(n_probes), int(order), flags, _ptr(out))
    return out


def chebyshev_probe_moments(ctx: Context, H: BSR, emin: float, emax: float, seed: int, n_probes: int,
                            order: int, fp64: bool = False, direct: bool = False,
                            plain: bool = False) -> tuple[torch.Tensor, torch.Tensor]:
    """a7 per probe: (moments (order,), per_probe (order, n_probes)) with per_probe[k, i] =
    r_i^T C_k(H^) r_i; the mean over i is moments[k]."""
    dev = H.val.device
    mom = torch.empty(order, dtype=torch.float64, device=dev)
    per = torch.empty((order, n_probes), dtype=torch.float64, device=dev)
    flags = ((L.TBK_FP64 if fp64 else L.TBK_MIXED) | (L.TBK_MOMENTS_DIRECT if direct else 0)
             | (L.TBK_PLAIN_KERNEL if plain else 0))
    L.call("tbk_chebyshev_probe_moments", ctx.handle, C.byref(H.struct()), emin, emax, C.c_uint64(seed),
           int(n_probes), int(order), flags, _ptr(mom), _ptr(per))
    return mom, per


def fermi_level(ctx: Context, moments: torch.Tensor, emin: float, emax: float,
                n_electrons: float | None, kT: float, jackson: bool = False,
                mu: float | None = None) -> tuple[float, float, float, float]:
    """a8: (mu, Omega, E, N); mu from N(mu) = n_electrons unless `mu` is given."""
    out = (C.c_double * 4)()
    ne = -1.0 if n_electrons is None else float(n_electrons)
    L.call("tbk_fermi_level", ctx.handle, _ptr(moments), moments.numel(), emin, emax, ne,
           0.0 if mu is None else float(mu), kT, L.TBK_DAMP_JACKSON if jackson else L.TBK_DAMP_NONE,
           out)
    return out[0], out[1], out[2], out[3]


def density_and_forces(ctx: Context, H: BSR, model: Model | None, pos: torch.Tensor | None, box,
                       emin: float, emax: float, seed: int, n_probes: int, order: int, mu: float,
                       kT: float, jackson: bool = False, fp64: bool = False, want_G: bool = True,
                       want_forces: bool = True, max_panel_bytes: int = 0, plain: bool = False,
                       windowed: bool | None = None):
    """a9-a10: (G, F) with G = dOmega^/dH (nnzb, b, b) and F = -dOmega^/dR (N, 3)."""
    dev = H.val.device
    G = torch.empty_like(H.val) if want_G else None
    F = torch.empty((H.graph.n_atoms, 3), dtype=torch.float64, device=dev) if want_forces else None
    _keep, bx = _box_arg(box)
    L.call("tbk_density_and_forces", ctx.handle, C.byref(H.struct()),
           C.byref(model.s) if model is not None else None, _ptr(pos), bx, emin, emax,
           C.c_uint64(seed), int(n_probes), int(order), float(mu), float(kT),
           L.TBK_DAMP_JACKSON if jackson else L.TBK_DAMP_NONE,
           (L.TBK_FP64 if fp64 else L.TBK_MIXED) | (L.TBK_PLAIN_KERNEL if plain else 0)
           | _schedule_flag(windowed),
           int(max_panel_bytes), _ptr(G), _ptr(F))
    return G, F


def direct_density(ctx: Context, H: BSR, model: Model | None, pos: torch.Tensor | None, box,
                   emin: float, emax: float, seed: int, n_probes: int, order: int, mu: float,
                   kT: float, jackson: bool = False, fp64: bool = False, want_P: bool = True,
                   want_Q: bool = True, want_forces: bool = False, plain: bool = False):
    """f2: (M o P~, M o Q~, forces) of the direct random estimate (Eq. poly_PQ, Eq. random_density)
    at a given mu; P~ and Q~ as (nnzb, b, b) blocks on H's pattern (not symmetric), forces from the
    symmetric part of M o P~ (or None)."""
    dev = H.val.device
    P = torch.empty_like(H.val) if want_P else None
    Q = torch.empty_like(H.val) if want_Q else None
    F = torch.empty((H.graph.n_atoms, 3), dtype=torch.float64, device=dev) if want_forces else None
    _keep, bx = _box_arg(box)
    L.call("tbk_direct_density", ctx.handle, C.byref(H.struct()),
           C.byref(model.s) if model is not None else None, _ptr(pos), bx, emin, emax,
           C.c_uint64(seed), int(n_probes), int(order), float(mu), float(kT),
           L.TBK_DAMP_JACKSON if jackson else L.TBK_DAMP_NONE,
           (L.TBK_FP64 if fp64 else L.TBK_MIXED) | (L.TBK_PLAIN_KERNEL if plain else 0),
           _ptr(P), _ptr(Q), _ptr(F))
    return P, Q, F


def rational_density(ctx: Context, H: BSR, model: Model | None, pos: torch.Tensor | None, box,
                     seed: int, n_probes: int, mu: float, kT: float, n_pairs: int, tol: float = 1e-10,
                     max_iter: int = 20000, want_P: bool = True, want_Q: bool = True,
                     want_forces: bool = False):
    """f4: (M o P~, M o Q~, forces, (CGLS iterations, worst relative residual)) of the rational
    approximation with n_pairs continued-fraction pole pairs and CGLS solves (FP64)."""
    dev = H.val.device
    P = torch.empty_like(H.val) if want_P else None
    Q = torch.empty_like(H.val) if want_Q else None
    F = torch.empty((H.graph.n_atoms, 3), dtype=torch.float64, device=dev) if want_forces else None
    info = (C.c_double * 2)()
    _keep, bx = _box_arg(box)
    L.call("tbk_rational_density", ctx.handle, C.byref(H.struct()),
           C.byref(model.s) if model is not None else None, _ptr(pos), bx, C.c_uint64(seed),
           int(n_probes), float(mu), float(kT), int(n_pairs), float(tol), int(max_iter), L.TBK_FP64,
           _ptr(P), _ptr(Q), _ptr(F), info)
    return P, Q, F, (int(info[0]), float(info[1]))


def local_density(ctx: Context, H: BSR, pos: torch.Tensor, box, r_max: float, emin: float,
                  emax: float, order: int, mu: float, kT: float, jackson: bool = False,
                  fp64: bool = False, want_P: bool = True, want_Q: bool = True):
    """f3: (M o P~_L, M o Q~_L) of the local approximation (Sec. II.C.1, Eq. local_density) with
    regions of radius r_max; block (b, a) holds rows b of column block a (not symmetric)."""
    P = torch.empty_like(H.val) if want_P else None
    Q = torch.empty_like(H.val) if want_Q else None
    _keep, bx = _box_arg(box)
    L.call("tbk_local_density", ctx.handle, C.byref(H.struct()), _ptr(pos), bx, float(r_max), emin, emax,
           int(order), float(mu), float(kT), L.TBK_DAMP_JACKSON if jackson else L.TBK_DAMP_NONE,
           L.TBK_FP64 if fp64 else L.TBK_MIXED, _ptr(P), _ptr(Q))
    return P, Q


def batched_moments(ctx: Context, Hs: list, emins, emaxs, seeds, n_probes: int, orders,
                    direct: bool = False, graph: bool = True) -> list:
    """a11: moments of many clusters in one launch per recurrence step (list of tensors)."""
    n = len(Hs)
    structs = (L.tbk_bsr * n)(*[h.struct() for h in Hs])
    e0 = (C.c_double * n)(*map(float, emins))
    e1 = (C.c_double * n)(*map(float, emaxs))
    sd = (C.c_uint64 * n)(*map(int, seeds))
    od = (C.c_int32 * n)(*map(int, orders))
    out = torch.empty(int(sum(orders)), dtype=torch.float64, device=Hs[0].val.device)
    flags = (L.TBK_MOMENTS_DIRECT if direct else 0) | (0 if graph else L.TBK_NO_GRAPH)
    L.call("tbk_batched_moments", ctx.handle, n, structs, e0, e1, sd, int(n_probes), od, flags,
           _ptr(out))
    return list(torch.split(out, [int(p) for p in orders]))


def batched_fermi_level(ctx: Context, moments: list, emins, emaxs, n_electrons, kTs,
                        jackson: bool = False) -> np.ndarray:
    """a8 for every cluster of a batch: rows (mu, Omega, E, N)."""
    n = len(moments)
    cat = torch.cat(moments).contiguous()
    od = (C.c_int32 * n)(*[m.numel() for m in moments])
    arr = lambda v: (C.c_double * n)(*map(float, v))
    out = (C.c_double * (4 * n))()
    L.call("tbk_batched_fermi_level", ctx.handle, n, _ptr(cat), od, arr(emins), arr(emaxs),
           arr(n_electrons), arr(kTs), L.TBK_DAMP_JACKSON if jackson else L.TBK_DAMP_NONE, out)
    return np.array(out[:], dtype=np.float64).reshape(n, 4)


def batched_density_and_forces(ctx: Context, Hs: list, model: Model, positions: list, emins,
                               emaxs, seeds, n_probes: int, orders, mus, kTs,
                               jackson: bool = False, want_G: bool = False,
                               max_panel_bytes: int = 0, windowed: bool = False):
    """a9-a11: (G list or None, forces list) of a batch, backward sweeps in one launch per step."""
    n = len(Hs)
    structs = (L.tbk_bsr * n)(*[h.struct() for h in Hs])
    arr = lambda v: (C.c_double * n)(*map(float, v))
    Fs = [torch.empty((h.graph.n_atoms, 3), dtype=torch.float64, device=h.val.device) for h in Hs]
    Gs = [torch.empty_like(h.val) for h in Hs] if want_G else None
    pp = (C.c_void_p * n)(*[p.data_ptr() for p in positions])
    fp = (C.c_void_p * n)(*[f.data_ptr() for f in Fs])
    gp = (C.c_void_p * n)(*[g.data_ptr() for g in Gs]) if want_G else None
    L.call("tbk_batched_density_and_forces", ctx.handle, n, structs, C.byref(model.s), pp,
           arr(emins), arr(emaxs), (C.c_uint64 * n)(*map(int, seeds)), int(n_probes),
           (C.c_int32 * n)(*map(int, orders)), arr(mus), arr(kTs),
           L.TBK_DAMP_JACKSON if jackson else L.TBK_DAMP_NONE, L.TBK_WINDOWED if windowed else 0,
           int(max_panel_bytes), gp, fp)
    return Gs, Fs


def batched_energies_and_forces(ctx: Context, Hs: list, model: Model, positions: list, emins,
                                emaxs, seeds, n_probes: int, orders, n_electrons, kTs,
                                jackson: bool = False, want_G: bool = False,
                                max_panel_bytes: int = 0, windowed: bool = False):
    """a5-a11 for a batch in one call: (moments list, observables (n, 4) array of
    (mu, Omega, E, N), G list or None, forces list)."""
    n = len(Hs)
    structs = (L.tbk_bsr * n)(*[h.struct() for h in Hs])
    arr = lambda v: (C.c_double * n)(*map(float, v))
    dev = Hs[0].val.device
    mom = torch.empty(int(sum(orders)), dtype=torch.float64, device=dev)
    obs = (C.c_double * (4 * n))()
    Fs = [torch.empty((h.graph.n_atoms, 3), dtype=torch.float64, device=h.val.device) for h in Hs]
    Gs = [torch.empty_like(h.val) for h in Hs] if want_G else None
    pp = (C.c_void_p * n)(*[p.data_ptr() for p in positions])
    fp = (C.c_void_p * n)(*[f.data_ptr() for f in Fs])
    gp = (C.c_void_p * n)(*[g.data_ptr() for g in Gs]) if want_G else None
    L.call("tbk_batched_energies_and_forces", ctx.handle, n, structs, C.byref(model.s), pp,
           arr(emins), arr(emaxs), (C.c_uint64 * n)(*map(int, seeds)), int(n_probes),
           (C.c_int32 * n)(*map(int, orders)), arr(n_electrons), arr(kTs),
           L.TBK_DAMP_JACKSON if jackson else L.TBK_DAMP_NONE, L.TBK_WINDOWED if windowed else 0,
           int(max_panel_bytes), _ptr(mom), obs, gp, fp)
    moms = list(torch.split(mom, [int(p) for p in orders]))
    return moms, np.array(obs[:], dtype=np.float64).reshape(n, 4), Gs, Fs


def energies_and_forces(ctx: Context, H: BSR, model: Model | None, pos: torch.Tensor | None, box,
                        emin: float, emax: float, seed: int, n_probes: int, order: int,
                        n_electrons: float, kT: float, jackson: bool = False, fp64: bool = False,
                        want_G: bool = False, want_forces: bool = True, max_panel_bytes: int = 0,
                        windowed: bool | None = None):
    """a5-a10 in one call: (moments, (mu, Omega, E, N), G or None, forces or None)."""
    dev = H.val.device
    mom = torch.empty(order, dtype=torch.float64, device=dev)
    G = torch.empty_like(H.val) if want_G else None
    F = torch.empty((H.graph.n_atoms, 3), dtype=torch.float64, device=dev) if want_forces else None
    obs = (C.c_double * 4)()
    _keep, bx = _box_arg(box)
    L.call("tbk_energies_and_forces", ctx.handle, C.byref(H.struct()),
           C.byref(model.s) if model is not None else None, _ptr(pos), bx, emin, emax,
           C.c_uint64(seed), int(n_probes), int(order), float(n_electrons), float(kT),
           L.TBK_DAMP_JACKSON if jackson else L.TBK_DAMP_NONE,
           (L.TBK_FP64 if fp64 else L.TBK_MIXED) | _schedule_flag(windowed),
           int(max_panel_bytes), _ptr(mom), obs, _ptr(G), _ptr(F))
    return mom, tuple(obs[:]), G, F


def order_for(W: float, kT: float, eps: float = 1e-7, p_min: int = 64) -> int:
    """Chebyshev terms from the paper's error model eps_poly ~ exp(-6.4 p kT / W) (Sec. II.B.1)."""
    return max(p_min, int(math.ceil((W / kT) * math.log(1.0 / eps) / 6.4)))


# ----------------------------------------------------------------------------------------------
# End-to-end solver and the autograd entry point
# ----------------------------------------------------------------------------------------------

@dataclass
class Result:
    emin: float
    emax: float
    order: int
    mu: float
    Omega: float
    E: float
    N: float
    moments: torch.Tensor
    H: BSR
    G: torch.Tensor | None = None
    forces: torch.Tensor | None = None

    @property
    def A(self) -> float:
        return self.Omega + self.mu * self.N


class Solver:
    """Runs the whole path for one workload (see ``workloads``) on one device."""

    def __init__(self, wk, ctx: Context | None = None, lanczos_steps: int = 64,
                 margin: float = 0.01, bounds_seed: int = 0x5EED):
        self.wk = wk
        self.ctx = ctx or Context()
        self.device = torch.device(f"cuda:{self.ctx.device}")
        self.model = Model.from_workload(wk, self.device)
        self.box = None if wk.box is None else [float(x) for x in wk.box]
        self.lanczos_steps = lanczos_steps
        self.margin = margin
        self.bounds_seed = bounds_seed
        self.graph = None

    def energies(self, pos: torch.Tensor, order: int | None = None, fp64: bool | None = None,
                 bounds=None, direct: bool = False) -> Result:
        wk = self.wk
        fp64 = (not wk.mixed) if fp64 is None else fp64
        self.graph = build_neighbors(self.ctx, pos, wk.cutoff, self.box)
        H = assemble_H(self.ctx, self.model, pos, self.graph, self.box)
        emin, emax = bounds if bounds is not None else spectral_bounds(
            self.ctx, H, self.lanczos_steps, self.margin, self.bounds_seed)
        p = order or wk.order or order_for(emax - emin, wk.kT)
        mom = chebyshev_moments(self.ctx, H, emin, emax, wk.probe_seed, wk.n_probes, p, fp64, direct)
        mu, Om, E, N = fermi_level(self.ctx, mom, emin, emax, wk.n_electrons, wk.kT, wk.jackson)
        return Result(emin, emax, p, mu, Om, E, N, mom, H)

    def forces(self, pos: torch.Tensor, res: Result, fp64: bool | None = None, want_G=False,
               max_panel_bytes: int = 0) -> Result:
        wk = self.wk
        fp64 = (not wk.mixed) if fp64 is None else fp64
        G, F = density_and_forces(self.ctx, res.H, self.model, pos, self.box, res.emin, res.emax,
                                  wk.probe_seed, wk.n_probes, res.order, res.mu, wk.kT, wk.jackson,
                                  fp64, want_G=want_G or not self.model.is_sk,
                                  want_forces=self.model.is_sk, max_panel_bytes=max_panel_bytes)
        res.G, res.forces = G, F
        return res

    def energies_and_forces(self, pos: torch.Tensor, order: int | None = None,
                            fp64: bool | None = None, bounds=None, want_G: bool = False,
                            max_panel_bytes: int = 0) -> Result:
        """energies() then forces() in one library call (one forward sweep instead of two)."""
        wk = self.wk
        fp64 = (not wk.mixed) if fp64 is None else fp64
        self.graph = build_neighbors(self.ctx, pos, wk.cutoff, self.box)
        H = assemble_H(self.ctx, self.model, pos, self.graph, self.box)
        emin, emax = bounds if bounds is not None else spectral_bounds(
            self.ctx, H, self.lanczos_steps, self.margin, self.bounds_seed)
        p = order or wk.order or order_for(emax - emin, wk.kT)
        is_sk = self.model.is_sk
        mom, (mu, Om, E, N), G, F = energies_and_forces(
            self.ctx, H, self.model if is_sk else None, pos if is_sk else None, self.box, emin,
            emax, wk.probe_seed, wk.n_probes, p, wk.n_electrons, wk.kT, wk.jackson, fp64,
            want_G=want_G or not is_sk, want_forces=is_sk, max_panel_bytes=max_panel_bytes)
        return Result(emin, emax, p, mu, Om, E, N, mom, H, G, F)


class FreeEnergy(torch.autograd.Function):
    """A^(R) = Omega^ + mu^ N_e of the probe estimate; backward returns -F (bounds held fixed).

    At fixed electron count dA^/dR = dOmega^/dR at fixed mu (the polynomial coefficients satisfy
    d beta[g]/d mu = -alpha[f] exactly), which the adjoint kernel evaluates.  ``bounds`` (emin,
    emax) fixes the spectral interval instead of taking it from Lanczos at ``pos``: with it, A^ is
    the smooth function of the positions whose gradient the backward pass returns.
    """

    @staticmethod
    def forward(fctx, pos: torch.Tensor, solver: Solver, bounds=None):
        res = solver.energies(pos.detach().contiguous(), bounds=bounds)
        fctx.solver = solver
        fctx.res = res
        fctx.save_for_backward(pos)
        return torch.tensor(res.Omega + res.mu * solver.wk.n_electrons, dtype=torch.float64,
                            device=pos.device)

    @staticmethod
    def backward(fctx, grad):
        (pos,) = fctx.saved_tensors
        res = fctx.solver.forces(pos.detach().contiguous(), fctx.res)
        return -res.forces * grad, None, None
