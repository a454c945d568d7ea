"""FP64 CPU oracle for the swift left inverse of a localized ensemble square root.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code with
the CUDA library (``paper_2609_13327_b300``) and imports nothing from it.

The oracle is deliberately plain: NumPy in float64, batched over grid columns
only where the paper's own statement is "for each column m", and otherwise
written as the definitions of Sardelli & Bishop (arxiv 2609.13327) read:

* ``basis``  -- the localization's horizontal eigenbasis on a periodic grid
  (economical eigendecomposition of C_b, Sec. 3.9) and the periodized-Gaussian
  spectrum with its closed form (Poisson summation).
* ``swift``  -- the vector-form swift algorithm V1-V4 (Sec. 3.10) for the left
  inverse, with the n_w != K generalisation A^{-1} -> A^+, and the square root
  A V Delta^{1/2} (Sec. 3.9) and both adjoints.
* ``dense``  -- brute force at tiny sizes: the modulated square root
  Zh = C^{1/2} (triangle) Z (Sec. 3.7), the matrix A (Sec. 3.7), its
  pseudo-inverse by dense SVD, the dense left inverse Delta^{-1/2} V^T A^+
  (Sec. 3.9, "InverseSquareRootSwift") and the accuracy indicators Xi and delta
  (Sec. 4.8, 4.9).

Parity pins: every function is checked by ``tests/test_oracle_pins.py``
against closed forms, brute force and the paper's identities.  The only
"parity unpinned" quantities are the paper's reported accuracy numbers
(RMSE_Xi, MAX_Xi, RMSE_delta of Sec. 4.8-4.9), whose inputs (spherical grid,
spherical-harmonics covariance and localization) the paper does not specify
fully enough to rebuild.
"""

from . import basis, swift, dense  # noqa: F401
