"""CPU FP64 oracle for the usFFT sampling-and-detection increment.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it and shares no code with it; the only
module both sides import is ``workloads`` (seeded input definitions).

Modules, each following the paper (Kaemmerer, Potts, Taubert, "The uniform
sparse FFT with application to PDEs with random coefficients"):

- ``rng``      counter-based SplitMix64 draws for the random tails y' and the
               lattice search (the paper draws them "uniformly at random",
               Algorithm 1, steps 1/2a and 2b).
- ``model``    the coefficient models (Eq. (1.2), Sec. 4.2, Sec. 4.3 with the
               mode ordering of Table 4.2).
- ``fe``       the black-box sampler: P1 finite elements for Eq. (1.1) in its
               weak form (Sec. 2.1), assembled element by element and solved by
               banded Cholesky.
- ``lattice``  candidate sets J_t (Algorithm 1, step 2), rank-1 lattices
               (Appendix A, Eq. (3.4)) and the reconstructing-lattice search.
- ``dft``      the projected Fourier coefficients by a naive DFT (Algorithm 1,
               steps 1/2a and 2d).
- ``detect``   thresholding to the s~ largest coefficients >= theta and the
               union over mesh nodes (Algorithm 1, steps 2d/2e).
- ``usfft``    the increment driver (Algorithm 1, steps 1, 2a, 2).

Pins: every function is checked by ``tests/test_oracle_*.py`` against closed
forms, brute force or values printed in the paper (see each module header).
"""
