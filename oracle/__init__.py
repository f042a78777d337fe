"""FP64 CPU oracle of the GCG eigensolver -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct reference that the CUDA
path is checked against.  Only the test-suite, the package's smoke check and
the benchmark's CPU-baseline leg may import it; the library never calls it
and shares no code with it (the two sides meet only through the seeded
inputs of the ``workloads`` module).

Modules
-------
``linalg``  CSR products, B-inner products, the dense symmetric eigensolve
            (LAPACK through numpy, the same role as the paper's ``dsyevx``).
``cg``      STEP 6: column-wise CG on the shifted system, Eq. (compW).
``orth``    STEP 2: deflation against a B-orthonormal block and Algorithm 3
            (RecursiveOrthSVD); Algorithm 2 (modified block orthogonalisation).
``gcg``     Algorithm 1 with locking (Section 3.2), the P construction of
            Eq. (CP_tilde)/(Equality_Cpx), the dynamic shift, the moving
            mechanism (Section 3.3), and an explicit full V^T A V Rayleigh-Ritz.
``grad``    Reference eigenvalue / eigenvector-functional gradients (standard
            first-order perturbation theory; not in the paper).

Every function is FP64.  Numerical thresholds that the paper leaves as
"small enough" are collected in ``gcg.Params`` with the reading taken.
"""
