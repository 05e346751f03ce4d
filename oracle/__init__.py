"""Plain, slow, FP64 CPU oracle of the sparse-lattice D3Q19 TRT stream-collide step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code,
constants or helpers with the CUDA library; the one module both sides use is
``geometry`` (seeded input generators, no method arithmetic).

What it computes (Wittmann et al., "Modeling and analyzing performance for
highly optimized propagation steps of the lattice Boltzmann method on sparse
lattices"):

* ``tables``  - fluid-node enumeration (lexicographic with blocking factor B,
  Hilbert curve; Sect. 5.6), the adjacency list of the sparse lattice
  (Sect. 4, "Loop Balance") and the RIA run-length table (Sect. 4.1).
* ``lbm``     - the lattice Boltzmann equation (Eq. 1, Sect. 2) with the TRT
  collision, pull streaming with halfway bounce-back and pressure
  anti-bounce-back, and the two storage forms OS-NT (two grids) and the AA
  pattern (one grid, even/odd steps) of Sect. 4; macroscopic moments and the
  mean-flux objective.
* ``esotwist`` - the Esoteric Twist single-grid form that Sect. 1 and Sect. 4
  name without evaluating (its slot rules are a reading, stated there).
* ``dense``   - the same LBM on the full voxel array with push streaming; it
  never builds an adjacency list, so it checks tables and streaming.
* ``adjoint`` - the reverse sweep of T steps taped by torch autograd over
  ``lbm`` (the discrete adjoint the CUDA kernels hand-derive).

Parity status: every function is pinned by a test in ``tests/`` against a
closed form, an invariant, brute force or a number printed in the paper,
except the pressure (anti-bounce-back) boundary, whose form the paper never
states: its parity is unpinned beyond the rest-state fixed point and the
dense/sparse agreement.
"""
