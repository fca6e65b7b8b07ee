"""Plain FP64 CPU oracle for the IMEX forward step and its exact discrete adjoint.

TEST INFRASTRUCTURE ONLY.  Nothing under ``oracle/`` is part of the product:
only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import it.  It shares no code with the CUDA path (different transforms,
different operator assembly, dense complex LU instead of the structured
pencil sweep) and it never reads a value produced by the CUDA path.

Every routine follows the paper's own statement of the method
(arXiv 2506.14792, "Fast automated adjoints for spectral PDE solvers"):

* ``imex``        -- multistep IMEX (Supplementary A.4, eq. imex) and its
                     adjoint (eq. IMEX_adjoint); Runge-Kutta IMEX stage
                     equation and its adjoint (Supplementary A.4).
* ``fourier``     -- collocation transforms T, T^-1 and their adjoints
                     (Methods, "Spectral transforms").
* ``chebyshev``   -- Chebyshev/ultraspherical sparse operators (Sparse
                     spectral methods section) and the Chebyshev matrix
                     transform.
* ``burgers``     -- 1D viscous Burgers on a periodic Fourier basis.
* ``rayleigh_benard`` -- 2D Boussinesq convection, Fourier x Chebyshev-tau.
* ``kolmogorov``  -- 2D periodic vorticity equation with sin(4y) forcing and a
                     4D-Var misfit objective.
* ``cnn``         -- FP64 reference of the 3x3 periodic CNN closure.
* ``couette``     -- 3D plane Couette flow, Fourier(x, y) x Chebyshev-tau, with the
                     energy-gain (optimal perturbation) objective.
* ``shear_evp``   -- linear stability eigenproblems of plane Couette and plane
                     Poiseuille flow, adjoint eigenvectors and eigenvalue
                     sensitivities (Problem types, "Eigenvalue problems").

Pins (what fixes each function independently of itself) live in
``tests/test_oracle_*.py`` and are listed in the design notes.
"""
