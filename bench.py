#!/usr/bin/env python
"""Benchmark of the Chebyshev random-probe tight-binding path on GB300.

One step = the whole path on one synthetic workload: neighbour list, H assembly, Lanczos
spectral bounds, Chebyshev moments with random probes, chemical potential and Omega / E / N,
then the adjoint (sampled density matrix dOmega/dH on the pattern) and the atomic forces.

Default workload: a 10,000-atom copper-like fcc sphere (9-orbital Slater-Koster model, 4.0 A
cutoff, 90,000 orbitals), kT = 0.025 eV, 11 electrons/atom, 512 Rademacher probes, FP32
recurrence with FP64 moments; the number of Chebyshev terms p follows the error model
exp(-6.4 p kT / W) of Sec. II.B.1 with eps = 1e-7.

Metric: atom*vector*Chebyshev-steps/s = N_atoms * probes * p / (time of one full step, energies
and forces).  Every launch of the three kernel families of the path (recurrence step, adjoint
step, windowed outer products) is bracketed by CUDA events inside the timed steps; `kernels`
gives each family's roofline (HBM bytes or FP32 FMA flops, whichever bounds it) and `roofline`
repeats the one with the largest share of the step.  `cpu_baseline` times the FP64 oracle on a
bounded sub-cluster.  More measured records ride along in the same line (single GPU, after the
main workload's memory is given back): `colored_sigma`, the sampling error of Omega^ for plain
probes and for the multi-colour ensemble at a 6 A colouring radius at equal columns; `fp64_compare`, the 48^3 periodic 9-orbital
lattice (1.0M orbitals, 10 eV band, kT = 0.05 eV, 512 probes) run whole by the mixed path and by
the plain FP64 GPU path, with both times, both results and the speed-up at equal accuracy; and
`batched64`, the 64-cluster batch (energies and forces of every cluster per step) with its own
value, e2e and roofline.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (replicas only: the path has no
exchange step), value = units of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

METRIC = "atom*vector*Chebyshev-steps/s"
UNIT = "atom*vector*steps/s"


def replica_times(*times_ms: float, device: str = "cpu") -> list:
    """Max over the ranks of each time: N replicas of the step make one job that lasts as long as
    its slowest rank.  One process: the local values."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return list(times_ms)
    t = torch.tensor(list(times_ms), dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return t.tolist()


def job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units of every rank over the slowest rank's time per step."""
    return units_per_rank * world / (ms / 1e3)


def make_workload(name: str, rank: int = 0, atom_order: str = "radial", probes: int | None = None):
    if name == "fcc10k":
        return wl.fcc_cu(10000, kT=0.025, n_probes=probes or 512, seed=5264, probe_seed=52640 + rank,
                         atom_order=atom_order)
    if name == "fcc1k":
        return wl.fcc_cu(1000, kT=0.5, n_probes=256, seed=5264, probe_seed=52640 + rank)
    if name == "sc1k":
        return wl.sc_disorder(L=10, probe_seed=18120 + rank)
    if name == "sc9-48":
        return wl.sc9_periodic(L=48, probe_seed=48480 + rank)
    if name == "batched64":
        # a representative member of the batch (mean size, middle temperature): the oracle sample
        return wl.fcc_cu(1253, kT=0.1, n_probes=128, seed=5264, probe_seed=64000 + rank)
    raise SystemExit(f"unknown workload {name}")


def order_rule(W: float, kT: float) -> int:
    return max(64, int(math.ceil((W / kT) * math.log(1e7) / 6.4)))


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, enabled: bool = True):
        self.device = device
        self.enabled = enabled
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        if not self.enabled:
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            why = "not sampled (--no-clocks)" if not self.enabled else "nvidia-smi unavailable"
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [why]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------------------------

SAMPLE_ATOMS = 600


def oracle_sample(wk_full, n_atoms: int = SAMPLE_ATOMS):
    """The same model, kT, probes and electron density on the first n_atoms of the cluster."""
    wk = wl.fcc_cu(n_atoms, kT=wk_full.kT, n_probes=wk_full.n_probes, seed=5264,
                   probe_seed=wk_full.probe_seed) if wk_full.sk_V is not None else None
    return wk


def oracle_step(wk, want=False):
    """Exact estimator energies + forces for wk by the oracle (dense FP64); returns (units, s, p)
    and, with want, the bounds, mu, Omega, E and forces."""
    from oracle import chebyshev as och, hamiltonian as oham, neighbors as onb, physics as oph
    t0 = time.perf_counter()
    rp, col = onb.neighbor_csr(wk.positions, wk.cutoff, wk.box)
    H = oham.dense_sk(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE, wk.box)
    w, V = np.linalg.eigh(H)
    W = w.max() - w.min()
    emin, emax = w.min() - 0.01 * W, w.max() + 0.01 * W
    p = order_rule(emax - emin, wk.kT)
    R = och.probes(H.shape[0], wk.n_probes, wk.probe_seed)
    mom = och.exact_moments(w, V, R, emin, emax, p)
    mu = och.estimator_mu(mom, emin, emax, wk.n_electrons, wk.kT)
    Om, E, _ = och.estimator_observables(mom, emin, emax, mu, wk.kT)
    G = och.estimator_gradient(w, V, R, emin, emax, mu, wk.kT, p=p)
    a, b, dH = oham.sk_bond_grads(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY, wk.box)
    F = oph.forces_from_blocks(G, a, b, dH, wk.n_atoms, 9)
    dt = time.perf_counter() - t0
    if want:
        return wk.n_atoms * wk.n_probes * p, dt, p, dict(emin=emin, emax=emax, mu=mu, Omega=Om, E=E, F=F)
    return wk.n_atoms * wk.n_probes * p, dt, p


def host_recurrence_rate(wk, steps: int = 24):
    """The oracle's host FP64 block-sparse recurrence (C/OpenMP, doubled moments, the GPU path's
    work per moment) on the full workload, a bounded number of block products: the CPU rate in the
    benchmark's own unit (the analogue of the paper's block-sparse solver throughput)."""
    from oracle import hamiltonian as oham, neighbors as onb, o2
    rp, col = onb.neighbor_csr(wk.positions, wk.cutoff, wk.box)
    Hs = oham.sparse_sk(wk.positions, rp, col, wk.sk_V, wl.SK_R0, wl.SK_DECAY, wl.SK_ONSITE, wk.box)
    # bounds that enclose the spectrum (Gershgorin): the rate does not depend on them
    absrow = np.asarray(abs(Hs).sum(axis=1)).ravel()
    diag = Hs.diagonal()
    lo, hi = float((diag - (absrow - np.abs(diag))).min()), float((diag + (absrow - np.abs(diag))).max())
    o2.moments(rp, col, Hs.data, lo, hi, wk.probe_seed, wk.n_probes, 3, doubled=True)   # warm-up
    t0 = time.perf_counter()
    _, products = o2.moments(rp, col, Hs.data, lo, hi, wk.probe_seed, wk.n_probes, 2 * steps + 1, doubled=True)
    dt = time.perf_counter() - t0
    return {"value": wk.n_atoms * wk.n_probes * products / dt, "unit": UNIT, "cores": cpu_cores(),
            "kind": "oracle (host FP64 block-sparse recurrence, C/OpenMP)",
            "sample": f"{wk.name}: all {wk.n_atoms} atoms and {wk.n_probes} probes, {products} block "
                      f"products (doubled moments), {dt:.1f} s"}


def cpu_cores() -> int:
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(k, "").isdigit():
            return int(os.environ[k])
    return os.cpu_count() or 1


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    wk = oracle_sample(make_workload(args.workload, 0, args.atom_order, args.probes))
    if wk is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle sample defined for the fcc workloads only"}))
        return 0
    for _ in range(args.warmup):
        oracle_step(wk)
    units, tot, p = 0, 0.0, 0
    for _ in range(args.steps):
        u, dt, p = oracle_step(wk)
        units += u
        tot += dt
    v = units / tot
    sample = (f"FP64 oracle (dense eigh + exact estimator + Daleckii-Krein forces) on the first "
              f"{wk.n_atoms} atoms of the same cluster, {wk.n_probes} probes, p={p}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wk.name, "sample_of": args.workload},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------

def traffic_from_profile(kernel_file: str, src_name: str, workload: str):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary, if that summary was taken
    on this workload and on the current source of the file that holds the kernel (matching
    sha256 prefix); else None."""
    import hashlib
    src = os.path.join(ROOT, "paper_1812_05264_gb300", "csrc", src_name)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", kernel_file)
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
        if ": " in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].split(": ", 1)
            vals[k.strip()] = v.strip()
    if vals.get(f"{src_name} sha256[:16]") != sha or vals.get("workload") != workload:
        return None
    try:
        return float(vals["dram bytes per launch (full size)"])
    except (KeyError, ValueError):
        return None


# FP32 FMA issue of one GB300: 152 SMs x 128 lanes x 2 flops per cycle at the maximum SM clock
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
L2_BYTES = 126 * 2 ** 20


def run_ours(args, rank, world):
    import torch
    from paper_1812_05264_gb300 import build as _build
    _build.build()
    from paper_1812_05264_gb300 import api

    dist = world > 1
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))

    def barrier():
        if dist:
            torch.distributed.barrier()

    wk = make_workload(args.workload, rank, args.atom_order, args.probes)
    ctx = api.Context()
    solver = api.Solver(wk, ctx)
    stream = ctx.stream
    pos_host = torch.from_numpy(np.ascontiguousarray(wk.positions)).pin_memory()
    pos = pos_host.to(f"cuda:{local}")
    box = solver.box
    fp64 = not wk.mixed
    esz = 8 if fp64 else 4
    def step(p_dev):
        g = api.build_neighbors(ctx, p_dev, wk.cutoff, box)
        H = api.assemble_H(ctx, solver.model, p_dev, g, box)
        emin, emax = api.spectral_bounds(ctx, H)
        p = args.order or wk.order or order_rule(emax - emin, wk.kT)
        _, obs, _, F = api.energies_and_forces(
            ctx, H, solver.model if solver.model.is_sk else None, p_dev, box, emin, emax,
            wk.probe_seed, wk.n_probes, p, wk.n_electrons, wk.kT, wk.jackson, fp64,
            want_G=not solver.model.is_sk, want_forces=solver.model.is_sk,
            windowed=None if args.adjoint == "auto" else args.adjoint)
        return p, obs, F, H.graph.nnzb

    if args.only_moments:
        return moments_only(args, ctx, solver, wk, pos)
    if args.only_adjoint:
        return adjoint_only(args, ctx, solver, wk, pos)
    if args.compare_fp64:
        return precision_compare(args, ctx, solver, wk, pos)
    # the library's timing-based choices for this operator (outside the timed region)
    tuned = None
    if wk.mixed and wk.n_orb == 9 and wk.n_probes % 128 == 0:
        g = api.build_neighbors(ctx, pos, wk.cutoff, box)
        Ht = api.assemble_H(ctx, solver.model, pos, g, box)
        lo, hi = api.spectral_bounds(ctx, Ht)
        tuned = api.autotune(ctx, Ht, lo, hi, wk.n_probes)
    for _ in range(max(args.warmup, 0)):
        step(pos)
    torch.cuda.synchronize()
    barrier()
    # every launch of the three kernel families of the path is bracketed by events
    ctx.time_kernels("step", "backward", "window")
    clocks = ClockSampler(local, enabled=not args.no_clocks)
    clocks.start()
    launches0 = ctx.launches
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        p, obs, F, nnzb = step(pos)
    t1.record(stream)
    torch.cuda.synchronize()
    launches = ctx.launches - launches0
    fam = {f: ctx.kernel_time(f) for f in ("step", "backward", "window")}
    ctx.time_kernels()
    barrier()
    ms = t0.elapsed_time(t1) / args.steps
    # end to end: positions from pinned host memory in, energies and forces back to the host
    e_ms = []
    h2d = pos_host.numel() * 8
    d2h = 0
    for _ in range(max(1, min(args.steps, 3))):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        pos_e = pos_host.to(f"cuda:{local}", non_blocking=True)
        p_e, obs_e, F_e, _ = step(pos_e)
        out = F_e.cpu() if F_e is not None else None
        s1.record(stream)
        torch.cuda.synchronize()
        d2h = (out.numel() * 8 if out is not None else 0) + 4 * 8
        e_ms.append(s0.elapsed_time(s1))
    clk = clocks.stop()
    ms, e_med = replica_times(ms, statistics.median(e_ms), device=f"cuda:{local}")
    units = wk.n_atoms * wk.n_probes * p
    value = job_rate(units, world, ms)
    # roofline of the dominant kernel from its own launches inside the timed steps
    n_rows = wk.n_atoms * wk.n_orb
    panel = n_rows * wk.n_probes * esz
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    B2 = wk.n_orb ** 2
    alu = 1.25 if fp64 else SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    K = p // 2
    nwin = (K - 1 + 3) // 4 + 1 if K >= 1 else 0
    # algorithmic bytes and flops (2 per FMA) of each family over the timed steps
    hb, blk = nnzb * B2 * esz, 2 * nnzb * B2 * wk.n_probes
    sched = args.adjoint if args.adjoint != "auto" else (tuned[1] if tuned else "fused")
    windowed = sched == "windowed"
    tensor = sched == "tensor"
    # the kernels that ran: 128-probe tasks take the self-fed kernels; the profiles under
    # profiles/ are of the TMA-fed step and the fused adjoint step
    chunk = tuned[0] if tuned else wk.n_probes
    step_k = "cheb_step_self" if chunk == 128 or wk.n_probes == 128 else "cheb_step_bulk"
    bwd_k = "clenshaw_self" if sched != "fused" and wk.n_probes == 128 else "clenshaw_sddmm_bulk"
    alone = sched != "fused"     # the backward step without its outer products
    alg = {
        # y_{k+1} = 2 H^ y_k - y_{k-1}: reads y_k, y_{k-1}, the H^ blocks, writes y_{k+1}
        "step": (lambda n: n * (3 * panel + hb), lambda n: n * blk, step_k,
                 "cheb_step_bulk_fcc10000.md" if step_k == "cheb_step_bulk" else None, "recurrence.cu"),
        # ybar_k = g_k + 2 H^ ybar_{k+1} - ybar_{k+2}: reads ybar_{k+1}, ybar_{k+2}, y_k, y_{k-1},
        # y_{k+1}, the H^ blocks, writes ybar_k; fused: and G += 2 y_k ybar_{k+1}^T (the same
        # tiles, as many FMAs again, the FP64 accumulator read and written once)
        "backward": (lambda n: n * (6 * panel + hb + (0 if alone else nnzb * B2 * 16)),
                     lambda n: n * blk * (1 if alone else 2), bwd_k,
                     None if alone else "clenshaw_sddmm_bulk_fcc10000.md", "adjoint.cu"),
        # windowed: G += sum_j y_j ybar_{j+1}^T (j = 0 .. K-1, K pairs a step): reads both panels
        # of every pair, reads and writes the FP64 accumulator once per window; tensor: one pair
        # per launch (K - 1 a step), the accumulator read and written every launch
        "window": ((lambda n: n * (2 * panel + nnzb * B2 * 16)) if tensor else
                   (lambda n: args.steps * (K * 2 * panel + nwin * nnzb * B2 * 16)),
                   (lambda n: n * blk) if tensor else (lambda n: args.steps * K * blk),
                   "sddmm_tc" if tensor else "sddmm_window_g", None,
                   "tc_sddmm.cu" if tensor else "adjoint.cu"),
    }
    kernels = {}
    for f, (tms, nl) in fam.items():
        if nl == 0:
            continue
        byf, flf, kname, prof, src = alg[f]
        by, fl = byf(nl) / args.steps, flf(nl) / args.steps
        sec = tms / 1e3 / args.steps
        t_mem, t_alu = by / (hbm * 1e9), fl / (alu * 1e12)
        if f == "window" and tensor:
            # a contraction on the TF32 tensor cores: HBM-bound at its algorithmic bytes unless
            # its useful flops take longer at the TF32 peak (measured BF16 peak x 1/2, nominal ratio)
            tf32 = float(peaks.get("bf16_tflops", 1895.3)) / 2
            if fl / (tf32 * 1e12) >= t_mem:
                r = {"bound": "tensor", "achieved": fl / sec / 1e12, "peak": tf32, "unit": "TFLOP/s",
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops x 1/2 (TF32, nominal ratio; of measured)"}
            else:
                r = {"bound": "hbm", "achieved": by / sec / 1e9, "peak": hbm, "unit": "GB/s",
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
        elif t_alu >= t_mem:
            r = {"bound": "alu", "achieved": fl / sec / 1e12, "peak": alu, "unit": "TFLOP/s",
                 "peak_source": ("152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (derived, FP32 FMA)"
                                 if not fp64 else "152 SMs x 64 FP64 ops x 2070 MHz / 64 (derived)")}
        else:
            r = {"bound": "hbm", "achieved": by / sec / 1e9, "peak": hbm, "unit": "GB/s",
                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
        r["frac"] = r["achieved"] / r["peak"]
        r.update(kernel=kname, traffic=traffic_from_profile(prof, src, wk.name) if prof else None,
                 algorithmic_bytes_per_launch=by * args.steps / nl,
                 algorithmic_flops_per_launch=fl * args.steps / nl,
                 avg_launch_ms=tms / nl, launches_timed=nl, share_of_step=tms / (ms * args.steps))
        kernels[f] = r
    dom = max(kernels, key=lambda f: kernels[f]["share_of_step"])
    roof = dict(kernels[dom])
    # (the fused schedule's y_0 launch is an outer product only)
    n_products = (fam["step"][1] + fam["backward"][1]) / args.steps - (0 if windowed else 1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if fp64 else "f32", "data": "synthetic",
        "config": {"workload": wk.name, "n_atoms": wk.n_atoms, "orbitals": n_rows,
                   "probes": wk.n_probes, "order_p": p, "kT": wk.kT, "nnzb": nnzb,
                   "moments": "FP64", "recurrence": "FP64" if fp64 else "FP32",
                   "l2": ("panels (%.0f MB each) larger than L2" if panel > L2_BYTES else
                          "panels (%.0f MB each) fit in L2: an L2-resident workload, not flushed")
                         % (panel / 1e6),
                   "parallelism": f"replicas x{world}", "seeds": [5264, wk.probe_seed],
                   "adjoint": sched + (" (tuned)" if args.adjoint == "auto" else ""),
                   "autotune": None if tuned is None else {"probes_per_task": tuned[0], "outer_products": tuned[1]},
                   "order_rule": "fixed by --order (profiling run)" if args.order else "exp(-6.4 p kT/W) = 1e-7"},
        "e2e": {"value": job_rate(units, world, e_med), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "kernels": {f: {k: v for k, v in r.items() if k != "peak_source"} for f, r in kernels.items()},
        # the same rate counting the block products actually run (the doubling identities need
        # K = p/2 forward and K - 1 backward products for p moments and their gradient)
        "spmm_rate": {"value": wk.n_atoms * wk.n_probes * n_products * world / (ms / 1e3),
                      "unit": "atom*vector*block-products/s", "block_products_per_step": n_products},
        "clocks": clk,
        "observables_per_atom": {"mu": obs[0], "Omega": obs[1] / wk.n_atoms,
                                 "E": obs[2] / wk.n_atoms, "N": obs[3] / wk.n_atoms},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        swk = oracle_sample(wk)
        if swk is not None:
            u, dt, ps, ref = oracle_step(swk, want=True)
            # the same estimator on the GPU (same probes, order and bounds): errors of the
            # benchmarked precision against the FP64 oracle
            ssv = api.Solver(swk, ctx)
            spos = torch.as_tensor(swk.positions, dtype=torch.float64, device=f"cuda:{local}")
            sres = ssv.energies_and_forces(spos, order=ps, bounds=(ref["emin"], ref["emax"]))
            line["accuracy_vs_oracle"] = {
                "sample": f"first {swk.n_atoms} atoms, {swk.n_probes} probes, p={ps}, "
                          f"{'FP64' if fp64 else 'FP32 recurrence, FP64 moments'}",
                "omega_per_atom_abs_eV": abs(sres.Omega - ref["Omega"]) / swk.n_atoms,
                "energy_per_atom_abs_eV": abs(sres.E - ref["E"]) / swk.n_atoms,
                "mu_abs_eV": abs(sres.mu - ref["mu"]),
                "force_max_abs_eV_per_A": float(np.abs(sres.forces.cpu().numpy() - ref["F"]).max()),
                "tolerances": {"energy_per_atom_eV": 1e-6 if fp64 else 1e-4, "force_eV_per_A": 1e-3}}
            line["cpu_recurrence_baseline"] = host_recurrence_rate(wk)
            line["cpu_baseline"] = {
                "value": u / dt, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                "sample": (f"FP64 oracle (dense eigh, exact estimator, Daleckii-Krein forces) on "
                           f"the first {swk.n_atoms} atoms of the cluster, {swk.n_probes} probes, "
                           f"p={ps}, {dt:.1f} s")}
    if world == 1 and not args.no_extras and args.workload == "fcc10k" and not args.order:
        # the other two measured configurations, each in a context of its own after this
        # workload's panels (229 GB) are given back:
        # - the 48^3 periodic lattice, mixed against the plain FP64 GPU path at equal accuracy;
        # - the 64-cluster batch (energies and forces of every cluster per step).
        ctx.close()
        torch.cuda.empty_cache()
        line["colored_sigma"] = colored_sigma(wk, obs[0], local, rank)
        c5 = api.Context()
        wk5 = make_workload("sc9-48", rank)
        s5 = api.Solver(wk5, c5)
        line["fp64_compare"] = fp64_compare(c5, s5, wk5, torch.as_tensor(
            wk5.positions, dtype=torch.float64, device=f"cuda:{local}"))
        c5.close()
        torch.cuda.empty_cache()
        b = batched_line(args.batch_steps, max(3, args.batch_warmup), "windowed", rank, world,
                         not args.no_clocks)
        line["batched64"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup",
                                                 "config", "e2e", "gpu_launches", "roofline",
                                                 "kernels", "phases_ms_per_step", "clocks")}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        torch.distributed.destroy_process_group()
    return 0


def moments_only(args, ctx, solver, wk, pos):
    """Profiling aid: just the fused recurrence (moments) with a fixed small order."""
    import torch
    from paper_1812_05264_gb300 import api
    g = api.build_neighbors(ctx, pos, wk.cutoff, solver.box)
    H = api.assemble_H(ctx, solver.model, pos, g, solver.box)
    emin, emax = api.spectral_bounds(ctx, H)
    p = args.order or 64
    for _ in range(args.warmup):
        api.chebyshev_moments(ctx, H, emin, emax, wk.probe_seed, wk.n_probes, p, not wk.mixed)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(args.steps):
        api.chebyshev_moments(ctx, H, emin, emax, wk.probe_seed, wk.n_probes, p, not wk.mixed)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"only": "moments", "workload": wk.name, "order": p, "ms": ms,
                      "ms_per_launch": ms / (p // 2)}))
    return 0


def precision_compare(args, ctx, solver, wk, pos):
    """Mixed (FP32 recurrence, FP64 moments) against the plain FP64 GPU path on the same
    workload, probes and order: time per recurrence step and the energy difference per site."""
    print(json.dumps({"compare": "mixed_vs_fp64", **fp64_compare(ctx, solver, wk, pos)}))
    return 0


def colored_sigma(wk, mu, local, rank, r_color=6.0, n_runs=12):
    """Sampling error of Omega^ (at the given mu) per atom for plain Rademacher probes and for the
    multi-colour ensemble at the colouring radius r_color, at equal columns: the plain error from
    the spread of the 512 single-probe estimates (sigma_1 / sqrt(columns)); the coloured error as
    the spread over n_runs single-sample runs with independent seeds."""
    import torch
    from paper_1812_05264_gb300 import api
    ctx = api.Context()
    pos = torch.as_tensor(wk.positions, dtype=torch.float64, device=f"cuda:{local}")
    model = api.Model.from_workload(wk, pos.device)
    g = api.build_neighbors(ctx, pos, wk.cutoff)
    H = api.assemble_H(ctx, model, pos, g)
    emin, emax = api.spectral_bounds(ctx, H)
    p = order_rule(emax - emin, wk.kT)
    cg = api.chebyshev_coefficients(ctx, 2, p, emin, emax, mu, wk.kT).cpu().numpy()
    t0 = time.perf_counter()
    _, per = api.chebyshev_probe_moments(ctx, H, emin, emax, wk.probe_seed, wk.n_probes, p)
    om1 = cg @ per.cpu().numpy()                    # single-probe estimates of Omega
    t_plain = time.perf_counter() - t0
    colors, q = api.atom_colors(ctx, pos, r_color)
    cols = q * wk.n_orb
    S = api.colored_columns(q, wk.n_orb, 1)
    t0 = time.perf_counter()
    omc = []
    for j in range(n_runs):
        m = api.colored_moments(ctx, H, emin, emax, 777000 + 101 * rank + j, colors, q, 1, S, p)
        omc.append(float(cg @ m.cpu().numpy()))
    t_col = (time.perf_counter() - t0) / n_runs
    ctx.close()
    sig_plain = float(np.std(om1, ddof=1)) / math.sqrt(cols)
    sig_col = float(np.std(omc, ddof=1))
    n = wk.n_atoms
    return {"workload": wk.name, "order_p": p, "mu": mu, "colouring_radius_A": r_color,
            "atom_colours": int(q), "columns_per_sample": int(cols), "panel_width": int(S),
            "sigma_omega_per_atom_plain_eV": sig_plain / n,
            "sigma_omega_per_atom_coloured_eV": sig_col / n,
            "ratio_coloured_over_plain": sig_col / sig_plain,
            "coloured_runs": n_runs,
            "note": (f"plain: spread of {wk.n_probes} single-probe estimates scaled to {cols} columns; "
                     f"coloured: spread over {n_runs} independent single-sample runs (its own "
                     f"relative uncertainty ~{1 / math.sqrt(2 * (n_runs - 1)):.0%})"),
            "s_per_coloured_sample": t_col, "s_plain_512_probe_sweep": t_plain}


def fp64_compare(ctx, solver, wk, pos):
    """One full moments run of each path (after a short warm-up of each kernel) on the same
    operator, bounds, probes and order, then mu, Omega, E, N of each.  The FP64 path equals the
    exact estimator to rounding (its moments agree with the Bloch oracle's to 1e-11 n in the
    tests), so the mixed path's difference from it is the mixed path's error."""
    import torch
    from paper_1812_05264_gb300 import api
    g = api.build_neighbors(ctx, pos, wk.cutoff, solver.box)
    H = api.assemble_H(ctx, solver.model, pos, g, solver.box)
    emin, emax = api.spectral_bounds(ctx, H)
    p = wk.order or order_rule(emax - emin, wk.kT)
    out = {"workload": wk.name, "sites": wk.n_atoms, "orbitals": wk.n_atoms * wk.n_orb,
           "probes": wk.n_probes, "order_p": p, "recurrence_steps": p // 2,
           "bounds_eV": [emin, emax]}
    for name, fp64 in (("mixed", False), ("fp64", True)):
        api.chebyshev_moments(ctx, H, emin, emax, wk.probe_seed, wk.n_probes, 8, fp64)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        mom = api.chebyshev_moments(ctx, H, emin, emax, wk.probe_seed, wk.n_probes, p, fp64)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        mu, Om, E, N = api.fermi_level(ctx, mom, emin, emax, wk.n_electrons, wk.kT, wk.jackson)
        out[name] = {"ms": e0.elapsed_time(e1), "ms_per_step": e0.elapsed_time(e1) / (p // 2),
                     "mu": mu, "Omega_per_site": Om / wk.n_atoms, "E_per_site": E / wk.n_atoms,
                     "N_per_site": N / wk.n_atoms}
    out["speedup_mixed_over_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    out["energy_diff_per_site_eV"] = abs(out["mixed"]["E_per_site"] - out["fp64"]["E_per_site"])
    out["omega_diff_per_site_eV"] = abs(out["mixed"]["Omega_per_site"] - out["fp64"]["Omega_per_site"])
    out["tolerance_per_site_eV"] = 1e-4
    out["equal_accuracy"] = bool(max(out["energy_diff_per_site_eV"], out["omega_diff_per_site_eV"]) < 1e-4)
    return out


def adjoint_only(args, ctx, solver, wk, pos):
    """Profiling aid: just the adjoint (density matrix and forces) with a fixed small order."""
    import torch
    from paper_1812_05264_gb300 import api
    g = api.build_neighbors(ctx, pos, wk.cutoff, solver.box)
    H = api.assemble_H(ctx, solver.model, pos, g, solver.box)
    emin, emax = api.spectral_bounds(ctx, H)
    p = args.order or 64
    mom = api.chebyshev_moments(ctx, H, emin, emax, wk.probe_seed, wk.n_probes, p, not wk.mixed)
    mu = api.fermi_level(ctx, mom, emin, emax, wk.n_electrons, wk.kT)[0]
    args_ = (ctx, H, solver.model, pos, solver.box, emin, emax, wk.probe_seed, wk.n_probes, p, mu,
             wk.kT, wk.jackson, not wk.mixed)
    sched = None if args.adjoint == "auto" else args.adjoint
    for _ in range(args.warmup):
        api.density_and_forces(*args_, windowed=sched)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(args.steps):
        api.density_and_forces(*args_, windowed=sched)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    print(json.dumps({"only": "adjoint", "workload": wk.name, "order": p,
                      "ms": e0.elapsed_time(e1) / args.steps}))
    return 0


def run_batched(args, rank, world):
    """Many fcc clusters (sizes log-uniform in [100, 5000], kT in {0.025, 0.1, 0.5} eV, N(0, 0.05 A)
    jitter, 128 probes each): energies and forces of the whole batch per step, the recurrence of
    all clusters in one launch per step (CUDA-graph replay) and the backward sweeps likewise."""
    import torch
    from paper_1812_05264_gb300 import build as _build
    _build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    line = batched_line(args.steps, args.warmup, args.adjoint, rank, world, not args.no_clocks)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        torch.distributed.destroy_process_group()
    return 0


def batched_line(steps, warmup, adjoint, rank, world, clocks_on=True):
    """The 64-cluster batch timed over `steps` steps after `warmup`; returns its JSON record."""
    import torch
    from paper_1812_05264_gb300 import api
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1

    def barrier():
        if dist:
            torch.distributed.barrier()

    spec = wl.batched_clusters(64, 100, 5000, (0.025, 0.1, 0.5), seed=6464 + rank)
    s = 128
    wks = []
    for i, (n, kT) in enumerate(zip(spec.sizes, spec.kTs)):
        wk = wl.fcc_cu(int(n), kT=float(kT), n_probes=s, seed=5264, probe_seed=64000 + 97 * rank + i)
        wk.positions = spec.positions[i]
        wks.append(wk)
    ctx = api.Context()
    model = api.Solver(wks[0], ctx).model
    hosts = [torch.from_numpy(np.ascontiguousarray(w.positions)).pin_memory() for w in wks]
    devs = [h.to(f"cuda:{local}") for h in hosts]
    phase_ev = []

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(ctx.stream)
        return e

    def step(pos, record=False):
        Hs, e0, e1, ps = [], [], [], []
        marks = [ev()] if record else None
        graphs = api.batched_build_neighbors(ctx, pos, wks[0].cutoff)
        for p_, g in zip(pos, graphs):
            Hs.append(api.assemble_H(ctx, model, p_, g))
        e0, e1 = api.batched_spectral_bounds(ctx, Hs)
        ps = [order_rule(hi - lo, w.kT) for w, lo, hi in zip(wks, e0, e1)]
        seeds = [w.probe_seed for w in wks]
        if record:
            marks.append(ev())
        _, obs, _, Fs = api.batched_energies_and_forces(ctx, Hs, model, pos, e0, e1, seeds, s, ps,
                                                        [w.n_electrons for w in wks],
                                                        [w.kT for w in wks],
                                                        windowed=adjoint == "windowed")
        if record:
            marks.append(ev())
            phase_ev.append((marks, Hs, ps))
        return ps, obs, Fs

    for _ in range(warmup):
        step(devs)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local, enabled=clocks_on)
    clocks.start()
    l0 = ctx.launches
    ctx.time_kernels("step", "backward", "window")
    t0 = torch.cuda.Event(enable_timing=True); t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(ctx.stream)
    for _ in range(steps):
        ps, obs, Fs = step(devs, record=True)
    t1.record(ctx.stream)
    torch.cuda.synchronize()
    barrier()
    launches = ctx.launches - l0
    fam = {f: ctx.kernel_time(f) for f in ("step", "backward", "window")}
    ctx.time_kernels()
    ms = t0.elapsed_time(t1) / steps
    e_ms = []
    for _ in range(max(1, min(steps, 2))):
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record(ctx.stream)
        pe = [h.to(f"cuda:{local}", non_blocking=True) for h in hosts]
        _, obs_e, Fe = step(pe)
        outs = [f.cpu() for f in Fe]
        b.record(ctx.stream)
        torch.cuda.synchronize()
        e_ms.append(a.elapsed_time(b))
    clk = clocks.stop()
    units = sum(w.n_atoms * s * p for w, p in zip(wks, ps))
    ms, e_med = replica_times(ms, statistics.median(e_ms), device=f"cuda:{local}")
    # rooflines of the two kernel families from their own launches in the timed steps: cluster c
    # takes part in K_c = p_c/2 recurrence steps and K_c adjoint steps
    _, Hs, ps_ = phase_ev[-1]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    alu = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    windowed = adjoint == "windowed"
    fb = ff = bb = bf = wb = wf = 0.0
    for H, p in zip(Hs, ps_):
        K = p // 2
        panel = H.graph.n_atoms * 9 * s * 4
        blocks = H.graph.nnzb * 81
        fb += K * (3 * panel + blocks * 4)
        ff += K * 2 * blocks * s
        bb += K * (6 * panel + blocks * 4 + (0 if windowed else blocks * 16))
        bf += K * (2 if windowed else 4) * blocks * s
        wb += K * 2 * panel + (K / 4 + 1) * blocks * 16
        wf += K * 2 * blocks * s
    kernels = {}
    for f, by, fl, kname in (("step", fb, ff, ("cheb_step_self" if s == 128 else "cheb_step_bulk") + " (batched)"),
                             ("backward", bb, bf, "clenshaw_self (batched)" if windowed
                              else "clenshaw_sddmm_bulk (batched)"),
                             ("window", wb, wf, "sddmm_window_g (batched)")):
        tms, nl = fam[f]
        if nl == 0:
            continue
        sec = tms / 1e3 / steps
        if fl / (alu * 1e12) >= by / (hbm * 1e9):
            r = {"bound": "alu", "achieved": fl / sec / 1e12, "peak": alu, "unit": "TFLOP/s",
                 "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (derived, FP32 FMA)"}
        else:
            r = {"bound": "hbm", "achieved": by / sec / 1e9, "peak": hbm, "unit": "GB/s",
                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
        r.update(frac=r["achieved"] / r["peak"], kernel=kname, traffic=None,
                 algorithmic_bytes_per_step=by, algorithmic_flops_per_step=fl,
                 avg_launch_ms=tms / nl, launches_timed=nl, share_of_step=tms / (ms * steps))
        kernels[f] = r
    dom = max(kernels, key=lambda f: kernels[f]["share_of_step"])
    h2d = sum(h.numel() * 8 for h in hosts)
    d2h = sum(w.n_atoms * 3 * 8 for w in wks)
    line = {"metric": METRIC, "value": job_rate(units, world, ms), "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched64-fcc-sk9", "clusters": len(wks),
                       "atoms": int(sum(w.n_atoms for w in wks)), "probes": s,
                       "orders_p": [int(p) for p in ps], "kT": [float(w.kT) for w in wks],
                       "l2": "merged panels (%.0f MB each) larger than L2" % (sum(w.n_atoms for w in wks) * 9 * s * 4 / 1e6),
                       "parallelism": f"replicas x{world}", "adjoint": adjoint},
            "e2e": {"value": job_rate(units, world, e_med), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": dict(kernels[dom]),
            "kernels": {f: {k: v for k, v in r.items() if k != "peak_source"} for f, r in kernels.items()},
            "phases_ms_per_step": {
                name: sum(m[i].elapsed_time(m[i + 1]) for m, _, _ in phase_ev) / len(phase_ev)
                for i, name in enumerate(("neighbours_H_bounds", "energies_and_forces"))},
            "clocks": clk}
    ctx.close()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fcc10k")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-moments", action="store_true", help="profiling aid: recurrence only")
    ap.add_argument("--only-adjoint", action="store_true", help="profiling aid: adjoint only")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="time the mixed path against the plain FP64 GPU path (same p, probes)")
    ap.add_argument("--no-clocks", action="store_true",
                    help="do not run the nvidia-smi clock sampler (for runs under a profiler)")
    ap.add_argument("--order", type=int, default=None,
                    help="fixed Chebyshev order (default: the error rule; 64 for --only-moments / "
                         "--only-adjoint); a reduced order is for profiler runs, not bench lines")
    ap.add_argument("--probes", type=int, default=None,
                    help="probe count of the fcc10k workload (default 512; a profiling aid)")
    ap.add_argument("--atom-order", default="radial", choices=["radial", "morton"],
                    help="listing order of the fcc10k atoms (same cluster)")
    ap.add_argument("--no-extras", action="store_true",
                    help="fcc10k: skip the 48^3 mixed-vs-FP64 record and the 64-cluster batch record")
    ap.add_argument("--batch-steps", type=int, default=2,
                    help="timed steps of the 64-cluster batch record in the default line")
    ap.add_argument("--batch-warmup", type=int, default=3)
    ap.add_argument("--adjoint", default="auto", choices=["auto", "fused", "windowed", "tensor"],
                    help="outer products inside each backward step, over windows of 4 steps, or on "
                         "the tensor cores after each step (auto: the tuned choice; windowed for "
                         "the 128-probe batch)")
    args = ap.parse_args()
    if args.adjoint == "auto" and args.workload == "batched64":
        # the batch's merged operator is not tuned: with 128 probes per cluster the fused step's
        # per-tile lane reduction dominates and windows of 4 steps measured faster
        args.adjoint = "windowed"
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched64":
        return run_batched(args, rank, world)
    return run_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
