"""FP64 CPU oracle for the two-colour D2Q9 chromodynamic MRT scheme.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, whole-field NumPy
restatement of the method of Spendlove, Xu, Halliday, Schenkel & Halliday,
"Chromodynamic multi-relaxation time lattice Boltzmann scheme for fluids with
density difference" (arXiv 2005.04642).  Only the tests, the smoke check of the
package entry module and the CPU-baseline leg of the benchmark may import it.
The CUDA library never calls it, links it or reads anything it writes.

Modules
-------
``cmrt_oracle``  the per-time-step update (Sec. 2, Sec. 3, App. A, App. B)
``analytic``     reference solutions used as physics pins (App. C, App. D and
                 textbook single-phase flows)
``cmrt_adjoint`` the discrete adjoint (reverse mode) of the step, the L2
                 colour-field objective and its gradient with checkpointing;
                 pinned by central finite differences of ``cmrt_oracle``

Every function cites the passage of the paper it follows.  Where the paper is
silent, garbled or self-contradictory, the reading taken is stated in the
docstring of the function that takes it.  All readings are pinned by the
``-m "not gpu"`` tests; no function here is "parity unpinned".
"""
