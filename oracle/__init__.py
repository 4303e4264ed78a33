"""Plain FP64 CPU oracle for the Parareal exponential-integrator Q1 FEM.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute this package: only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference arm use it.  It shares no code
with the CUDA library; the only common module is the seeded descriptor
generator ``paper_2412_01138_gb300.inputs``, which holds no arithmetic of
the method.

The oracle follows Huang & Xu, "A Parareal exponential integrator finite
element method for linear parabolic equations" (arXiv 2412.01138):

* ``fem``        Q1 space, Kronecker-assembled mass/stiffness, both
                 diagonalisation routes (dense generalized eigensolve and
                 the closed-form DST-I eigenpairs), Sec. 2.1 and Sec. 2.3.
* ``quadrature`` Gauss-Legendre consistent loads, the L2 projection P_h
                 and the element-quadrature L2 error, Sec. 2.1 and Sec. 5.
* ``phi``        phi_j functions and the weights b_i of Eq. (3-12).
* ``solver``     the EIFE-linear step Eq. (1-7), sequential EIFE, the
                 coarse/fine propagators and Algorithm 1 literally.

Every function computes in float64 and is written for clarity, not speed.
Parity status of each function is stated in its docstring; all are pinned
by tests in ``tests/test_oracle_*.py`` against values the paper prints,
closed forms, invariants or an independent library route.
"""
