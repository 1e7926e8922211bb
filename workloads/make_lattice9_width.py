"""Writes lattice9_width.txt: the Bloch band width of the unscaled 9-orbital lattice model.

The periodic 9-orbital simple-cubic workload asks for hopping blocks "scaled to bandwidth ~10 eV".
The width of a Bloch band is max_k lambda_max(H(k)) - min_k lambda_min(H(k)); it needs the
eigenvalues of every H(k), which is the oracle's arithmetic, not the input module's.  So this
script, which calls only the oracle, computes it once for the N(0, 1) blocks of each seed on the
48^3 k-grid and stores it; ``workloads.lattice9_blocks`` multiplies the blocks by
band_width / stored width.  The width is linear in the blocks, so the scaled model's Bloch band
on the 48^3 grid is band_width wide.

Run:  python workloads/make_lattice9_width.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import workloads as wl  # noqa: E402
from oracle import bloch  # noqa: E402

SEEDS = (4848,)
GRID = 48


def main():
    lines = ["# seed  k-grid  Bloch band width (eV) of the unscaled N(0,1) blocks, h_{-d} = h_d^T"]
    for seed in SEEDS:
        dirs, h = wl.lattice9_blocks(seed, scale=1.0)
        disp = np.concatenate([dirs, -dirs])
        blocks = np.concatenate([h, np.transpose(h, (0, 2, 1))])
        w, _ = bloch.bands(GRID, disp, blocks)
        lines.append(f"{seed} {GRID} {w.max() - w.min():.17g}")
    with open(os.path.join(HERE, "lattice9_width.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
