"""CPU oracle for topology-based transient analysis of power grids.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, FP64 reference
that the CUDA path is checked against.  Only the test suite, the package
smoke check and the CPU-baseline leg of the benchmark may import it; the
product path never routes through it and shares no code with it (the seeded
input generator ``pgsynth`` is the only module both sides read).

Modules
-------
``matrices``   incidence matrices and the nodal system matrices (Eq. 4-6, 9, 11)
``pwl``        piecewise-linear current-source evaluation (the I_s of Eq. 8)
``transient``  backward-Euler transient, RC (Eq. 2) and RLC with explicit
               inductor currents (Eq. 10) or the eliminated three-level form
               (Eq. 11); DC operating point for the initial conditions
``relax``      the paper's node-by-node Gauss-Seidel / SOR update (Eq. 14-17),
               natural ordering, pure Python, for small grids
``bounds``     ||M^-1||_inf and the step-to-step error gain q used by the
               stopping rule, computed by direct solves
``adjoint``    discrete adjoint of the RC transient (not in the paper)
``rbsor``      the multicore CPU baseline: red-black SOR (Eq. 16-17) in C with
               OpenMP under the certified stopping rule, timed by the benchmark
               (not used for parity)

Sign conventions are those of Eq. 4-7 with the source-term signs fixed so
that they agree with KVL (Eq. 7): the RHS of a BE step is
``(C/h) v - A_l^T i_l - A_i^T I - G_s v_d - h L_s v_d`` (see ``transient``).
"""
