"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no arithmetic of the method itself: it only draws geometry and model
parameters from fixed seeds (NumPy PCG64) in FP64 on the host.  Both the CUDA library and the
oracle receive the arrays it returns.  The probe vectors are *not* drawn here: each side
regenerates them from the counter-based SplitMix64 definition (Steele, Lea & Flood, OOPSLA 2014).

Workloads (shapes follow the copper clusters of the paper, Sec. III, and its proposed
simple-cubic test model, Sec. IV):

* ``sc_cluster``       -- simple-cubic L x L x L open cluster, unit spacing, 1 orbital per site.
* ``fcc_sphere``       -- fcc sphere (lattice constant 3.61 A) centred on an atom; the first N
                          sites in (r^2, x, y, z) lexicographic order, optional N(0, sigma) jitter.
* ``sk_integrals``     -- the 10 Slater-Koster bond integrals ss_sigma .. dd_delta, N(0, 1) eV.
* ``lattice9_blocks``  -- 9x9 hopping blocks for the 3 nearest- and 6 next-nearest-neighbour
                          directions of a 9-orbital simple-cubic lattice, scaled to a given Bloch
                          band width (a stored constant written by make_lattice9_width.py) or to
                          a Gershgorin half-width.
* ``batched_clusters`` -- sizes (log-uniform in [lo, hi]) and temperatures for a batch of fcc
                          clusters.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np

# Orbital order used everywhere: s, px, py, pz, dxy, dyz, dzx, dx2-y2, d3z2-r2.
ORBITALS = ("s", "px", "py", "pz", "dxy", "dyz", "dzx", "dx2-y2", "d3z2-r2")
# Order of the 10 two-centre integrals.
SK_NAMES = ("sss", "sps", "sds", "pps", "ppp", "pds", "pdp", "dds", "ddp", "ddd")

FCC_A = 3.61          # lattice constant, Angstrom
SK_R0 = 2.55          # reference bond length of the radial factor exp(-decay (r/r0 - 1)), A
SK_DECAY = 2.0
SK_CUTOFF = 4.0       # hard cutoff, A
SK_ONSITE = (5.0, 10.0, 0.0)   # s, p, d on-site energies, eV

# The 9 positive directions of the 9-orbital simple-cubic lattice model: 3 nearest neighbours
# and the 6 next-nearest neighbours whose first nonzero component is positive.
LATTICE9_DIRS = np.array([
    [1, 0, 0], [0, 1, 0], [0, 0, 1],
    [1, 1, 0], [1, -1, 0], [1, 0, 1], [1, 0, -1], [0, 1, 1], [0, 1, -1],
], dtype=np.float64)


def sc_cluster(L: int) -> np.ndarray:
    """Sites of an L^3 simple-cubic cluster with unit spacing, index (i*L + j)*L + k."""
    g = np.arange(L, dtype=np.float64)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def onsite_uniform(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """n on-site energies uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n)


def fcc_sphere(n_atoms: int, a: float = FCC_A, jitter: float = 0.0, seed: int = 0) -> np.ndarray:
    """The n_atoms fcc sites closest to an atom at the origin.

    Sites are enumerated in integer units of a/2 (x + y + z even), so r^2 is an exact integer and
    ties are broken by (x, y, z) lexicographically.  ``jitter`` adds N(0, jitter) A per coordinate.
    """
    if n_atoms <= 0:
        return np.zeros((0, 3))
    # radius (in units of a/2) with a comfortable margin: 4 atoms per a^3 = 8 (a/2)^3 cells
    r = int(np.ceil((3.0 * n_atoms * 8.0 / (4.0 * 4.0 * np.pi)) ** (1.0 / 3.0))) + 3
    g = np.arange(-r, r + 1)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    keep = ((x + y + z) % 2) == 0
    x, y, z = x[keep], y[keep], z[keep]
    r2 = x * x + y * y + z * z
    order = np.lexsort((z, y, x, r2))[:n_atoms]
    pos = np.stack([x[order], y[order], z[order]], axis=1).astype(np.float64) * (a / 2.0)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        pos = pos + rng.normal(0.0, jitter, size=pos.shape)
    return pos


def morton_order(pos: np.ndarray, cell: float) -> np.ndarray:
    """Permutation that lists atoms by the Morton (Z-order) code of their cell on a grid of
    spacing ``cell`` (ties by input index): atoms close in space get close indices."""
    if len(pos) == 0:
        return np.zeros(0, dtype=np.int64)
    q = np.floor((pos - pos.min(axis=0)) / cell).astype(np.int64)
    code = np.zeros(len(pos), dtype=np.int64)
    for bit in range(20):
        for d in range(3):
            code |= ((q[:, d] >> bit) & 1) << (3 * bit + d)
    return np.lexsort((np.arange(len(pos)), code))


def sk_integrals(seed: int) -> np.ndarray:
    """The 10 bond integrals (order ``SK_NAMES``) drawn N(0, 1) eV."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(10)


def lattice9_width(seed: int) -> float:
    """The Bloch band width (eV) of the unscaled blocks of ``seed`` on the 48^3 k-grid, as stored
    by make_lattice9_width.py (which computes it with the oracle's Bloch eigenvalues)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lattice9_width.txt")
    with open(path) as f:
        for ln in f:
            parts = ln.split()
            if parts and not ln.startswith("#") and int(parts[0]) == seed:
                return float(parts[2])
    raise KeyError(f"no stored Bloch band width for seed {seed}; run workloads/make_lattice9_width.py")


def lattice9_blocks(seed: int, half_width: float | None = None, band_width: float | None = None,
                    scale: float | None = None):
    """Hopping blocks h_d for the 9 directions ``LATTICE9_DIRS`` (h_{-d} = h_d^T), on-site block 0.

    The blocks are N(0, 1) times one scale c:
    * ``band_width``: c = band_width / (stored Bloch band width of the unscaled blocks on the 48^3
      k-grid), so the scaled model's band is band_width wide;
    * ``half_width``: the largest Gershgorin row sum over all 18 bonds,
      max_i sum_d sum_l |c h_d[i, l]|, equals half_width (the band lies in [-half_width,
      half_width]);
    * ``scale``: c itself.
    Exactly one may be given; none means half_width = 5.
    Returns (dirs (9, 3), blocks (9, 9, 9)).
    """
    if sum(x is not None for x in (half_width, band_width, scale)) > 1:
        raise ValueError("give one of half_width, band_width, scale")
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((9, 9, 9))
    if band_width is not None:
        h *= band_width / lattice9_width(seed)
    elif scale is not None:
        h *= scale
    else:
        rows = np.zeros(9)
        for d in range(9):
            rows += np.abs(h[d]).sum(axis=1) + np.abs(h[d].T).sum(axis=1)
        h *= (5.0 if half_width is None else half_width) / rows.max()
    return LATTICE9_DIRS.copy(), h


def sc_lattice(L: int) -> tuple[np.ndarray, np.ndarray]:
    """Periodic L^3 simple-cubic lattice: sites and the box (L, L, L)."""
    return sc_cluster(L), np.array([float(L)] * 3)


@dataclass
class BatchSpec:
    sizes: np.ndarray            # atoms per cluster
    kTs: np.ndarray              # temperature per cluster, eV
    seeds: np.ndarray            # jitter seed per cluster
    positions: list = field(default_factory=list)


def batched_clusters(n_clusters: int, lo: int, hi: int, temps, seed: int,
                     jitter: float = 0.05) -> BatchSpec:
    """Cluster sizes log-uniform in [lo, hi], one temperature from ``temps`` each, jittered fcc."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_clusters))).astype(np.int64)
    kTs = np.asarray(temps, dtype=np.float64)[rng.integers(0, len(temps), size=n_clusters)]
    seeds = rng.integers(1, 2**31 - 1, size=n_clusters)
    spec = BatchSpec(sizes=sizes, kTs=kTs, seeds=seeds)
    spec.positions = [fcc_sphere(int(n), jitter=jitter, seed=int(sd)) for n, sd in zip(sizes, seeds)]
    return spec


# ---------------------------------------------------------------------------------------------
# Named workloads (sizes and seeds fixed; the recipe is restated in the design notes).
# ---------------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    positions: np.ndarray
    n_orb: int
    kT: float
    n_electrons: float
    n_probes: int
    probe_seed: int
    box: np.ndarray | None = None
    # SK model
    sk_V: np.ndarray | None = None
    # table model: displacement vectors and blocks, per-site on-site diagonal
    disp: np.ndarray | None = None
    blocks: np.ndarray | None = None
    onsite_site: np.ndarray | None = None
    cutoff: float = SK_CUTOFF
    order: int | None = None      # Chebyshev terms; None -> chosen from the spectral width
    jackson: bool = False
    mixed: bool = True

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])


def sc_disorder(L: int = 10, t: float = -1.0, w: float = 0.5, seed: int = 1812,
                n_probes: int = 32, order: int = 200, probe_seed: int = 18120) -> Workload:
    """Simple-cubic open cluster, nearest-neighbour hopping t, on-site U[-w, w], half filling."""
    pos = sc_cluster(L)
    n = pos.shape[0]
    disp = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    blocks = np.full((6, 1, 1), t)
    return Workload(name=f"sc{L}^3-open-1orb", positions=pos, n_orb=1, kT=0.1 * abs(t),
                    n_electrons=float(n), n_probes=n_probes, probe_seed=probe_seed,
                    disp=disp, blocks=blocks, onsite_site=onsite_uniform(n, -w, w, seed),
                    cutoff=1.0, order=order, jackson=True, mixed=False)


def fcc_cu(n_atoms: int, kT: float, n_probes: int, seed: int = 5264, probe_seed: int = 52640,
           jitter: float = 0.0, order: int | None = None, mixed: bool = True,
           atom_order: str = "radial") -> Workload:
    """Copper-like fcc sphere with a seed-drawn s/p/d Slater-Koster model, 11 electrons/atom.

    atom_order: "radial" lists the atoms by (r^2, x, y, z); "morton" lists the same atoms by the
    Z-order of their FCC_A-sized cells (the same cluster, spatially local indices)."""
    pos = fcc_sphere(n_atoms, jitter=jitter, seed=seed + 1)
    tag = ""
    if atom_order == "morton":
        pos = pos[morton_order(pos, FCC_A)]
        tag = "-morton"
    elif atom_order != "radial":
        raise ValueError(f"unknown atom order {atom_order}")
    return Workload(name=f"fcc{n_atoms}-sk9-kT{kT:g}{tag}", positions=pos, n_orb=9, kT=kT,
                    n_electrons=11.0 * n_atoms, n_probes=n_probes, probe_seed=probe_seed,
                    sk_V=sk_integrals(seed), order=order, mixed=mixed)


def sc9_periodic(L: int = 48, kT: float = 0.05, n_probes: int = 512, seed: int = 4848,
                 probe_seed: int = 48480, order: int | None = None, mixed: bool = True) -> Workload:
    """Periodic 9-orbital simple-cubic lattice with NN and NNN 9x9 hopping blocks scaled to a
    10 eV Bloch band (on the 48^3 k-grid), half filling."""
    pos, box = sc_lattice(L)
    dirs, h = lattice9_blocks(seed, band_width=10.0)
    disp = np.concatenate([dirs, -dirs])
    blocks = np.concatenate([h, np.transpose(h, (0, 2, 1))])
    return Workload(name=f"sc9-{L}^3-periodic-kT{kT:g}", positions=pos, n_orb=9, kT=kT,
                    n_electrons=9.0 * pos.shape[0], n_probes=n_probes, probe_seed=probe_seed,
                    box=box, disp=disp, blocks=blocks, onsite_site=None, cutoff=1.5,
                    order=order, mixed=mixed)
