"""FP64 CPU oracle for the GPUTB hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously correct NumPy/SciPy restatement of
what the GPU path computes.  It exists to check the CUDA library, never to
stand in for it: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import it.  It shares no code with the CUDA path (no
kernels, headers, helpers, tables or constant generators); both sides only
consume the same seeded inputs.

Modules and the passages they follow (arXiv 2509.06525):

* neighbors    -- N(i) of Eq. 1: all periodic images within r_cut.
* teacher      -- the analytic environment-dependent pz teacher model that
                  replaces the DFT labels (Sec. 2.3) here.
* descriptors  -- Chebyshev radial functions f_k, the species-mixed C_n and
                  the node feature v_i of Eq. 2.
* mlp          -- the SiLU MLP of Sec. 3 (forward, backward), the loss of
                  the form of Eq. 3 (band-energy loss, here on H elements)
                  and the AdamW update of Sec. 2.1.
* hamiltonian  -- sparse H of Eq. 1, symmetric hopping (Sec. 3 symmetry).
* bounds       -- spectral bounds (Gershgorin, Lanczos + Sturm bisection)
                  that map the spectrum into [-1, 1] for the Chebyshev
                  expansion of Sec. 2.4.
* kpm          -- random-phase vectors and the Chebyshev moment recursion of
                  the LSQT/KPM method (Sec. 2.4).
* dos          -- Jackson-damped KPM density of states, Eq. 4.
* lsqt         -- velocity operator, time evolution and the velocity
                  autocorrelation conductivity of Eq. 3 (sigma), Sec. 2.4.
* slater_koster -- the s, p, d Slater-Koster Hamiltonian (angular factors
                  of Sec. 3) by rotation of the bond-frame block.
* env_bands    -- the environment network of Eq. 2, the SK-form pz hopping
                  and onsite networks of Sec. 3, the Bloch sum H(k), bands
                  by dense diagonalisation, the band loss of Eq. 3 and its
                  Hellmann-Feynman gradient.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(closed forms, dense diagonalisation, invariants, brute force, independent
library routines).  None is marked "parity unpinned".
"""
