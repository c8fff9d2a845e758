"""CPU FP64 oracle for the multigrid waveform-relaxation solver of the time-fractional
heat equation (Hu, Rodrigo & Gaspar, arXiv 1706.07632).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The product path
(the CUDA library and its Python binding) never calls it and shares no code with it.

Everything here is plain, slow and written to be checked against the paper by eye:

* ``l1``      -- graded time mesh (Section 2) and the Petrov-Galerkin L1 matrix R of Eq.
                 (elements_matrix_R), evaluated from its integral definition; the initial-data
                 coefficient; the Mittag-Leffler function used by the 1D experiment (Section 5.1).
* ``hmatrix`` -- the H-matrix approximation of R from Section 3: index bisection, the
                 admissibility condition (Definition 3.1), Taylor degenerate kernel and the
                 Rk factors A, B (Eqs. A_elements, B_elements), plus the bound of Theorem 3.1.
* ``direct``  -- the fully discrete problem (Eqs. discrete_model_IVP_1-3) solved directly:
                 O1 implicit time stepping with the dense history sum, O2 per-sine-mode
                 triangular solves, O3 brute-force dense solve of the whole space-time system.
* ``wrmg``    -- Algorithm 2 (multigrid waveform relaxation) in its plain recursive form:
                 red-black zebra-in-time smoothing, defect, full weighting, linear/bilinear
                 interpolation, coarsest direct solve.

Pins (in ``tests/test_oracle_*.py``) tie every function to something other than itself:
50-digit mpmath evaluations, the textbook uniform-mesh L1 weights, exactness of the scheme
on piecewise-linear functions, the Theorem 3.1 bound, brute force on tiny inputs, and the
printed values of Table 1 and the cycle counts of Tables 3 and 5.
"""
