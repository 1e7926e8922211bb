"""Plain, slow FP64 CPU oracle for the Chebyshev-probe tight-binding path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports, links or executes this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference arm
of ``bench.py`` use it.  It shares no code with the CUDA library; both sides receive the same
seeded inputs from ``workloads`` and each regenerates the probe vectors from the published
SplitMix64 definition on its own.

Modules (each function cites the part of arXiv 1812.05264 it follows):

* ``neighbors``  -- brute-force O(N^2) pair search (mask M, Sec. II.A).
* ``slater_koster`` -- two-centre s/p/d blocks (Sec. II.A, the Slater-Koster form of the
  NRL model), derivatives by the complex-step method.
* ``hamiltonian`` -- dense H from the SK or lattice-table model; dense dH/dR.
* ``physics``    -- f, g, exact chemical potential, Omega, E, N, P and Hellmann-Feynman forces
  from dense diagonalisation (Eqs. 1-5).
* ``chebyshev``  -- Chebyshev coefficients by Chebyshev-Gauss quadrature (Sec. II.B.1),
  Jackson damping, Rademacher probes, the exact value of the random-probe estimator
  (Sec. II.C.2) evaluated through the eigen-decomposition, its exact gradient (Sec. II.D,
  Daleckii-Krein form), estimator forces and the Hutchinson variance (Eq. sampling_error).
* ``bloch``      -- Bloch-theorem oracle for translation-invariant periodic lattices
  (Sec. II.E, periodic reference algorithm).
* ``coloring``   -- Welsh-Powell colouring of the atom graph (Sec. II.E) and the multi-colour
  probe ensemble (Sec. II.C.3): coloured probes, the estimator's exact moments and gradient,
  its sampling error.
* ``direct``     -- direct random estimates M o P~ and M o Q~ of the density and
  energy-density matrices (Eq. poly_PQ, Eq. random_density) and their element-wise
  sampling error.
* ``local``      -- local approximation of M o P and M o Q (Sec. II.C.1, Eq. local_density):
  one dense local problem per atom within the localization radius.

Parity status: every public function is pinned by a ``-m "not gpu"`` test against closed
forms, invariants or brute force (see ``tests/test_oracle_*.py``).
"""
