"""CPU oracle for the d-level block Toeplitz matrix-vector product y = T x.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls, links
or executes anything in this package: only ``tests/``, the smoke check in
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may use it.  It shares no code with the CUDA library.

Everything is plain NumPy / SciPy in complex128 (FP64), written to be checked
against the paper by eye:

* ``toeplitz``  -- the definition (Sec. I, the 2x2 -> 4x4 embedding example
  fixes "block (i, j) holds t[i - j]"): explicit dense matrix, direct sum over
  offsets, direct sums at sampled output points, pure-Python brute force.
* ``embed``     -- the standard multilevel circulant embedding (Sec. I):
  embedded generator with free entry s0, its multidimensional DFT (the
  symbol), and the embedded FFT matvec followed by projection.
* ``split``     -- Algorithm 1 (Sec. II.B) restated: the recursive
  lazy-embedding / eager-projection tree with the splitting property and the
  merge of Sec. II.A, plus the flat sum over leaf parities it is equal to.

Pins (tests/test_oracle.py, all CPU): dense brute force on tiny grids,
np.convolve for d=1, identity and single-offset generators, linearity, shift
equivariance, the adjoint identity, symmetric and skew bilinear identities,
s0-invariance, level-order invariance, the splitting identity against an
explicit DFT sum, the paper's 2x2 -> 4x4 embedding and two-level symmetric
layout examples (tests/golden/), and the mirror (skew-)symmetry of the symbol.

Parity unpinned: the paper's measured wall-clock ratios (Fig. 3) have no data
in the text, so no oracle function reproduces them.
"""
