"""Oracle: a plain, slow, FP64 CPU statement of what the hot path computes.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package;
only the tests, the smoke check and the bench's CPU-baseline leg do.  It
shares no code with the CUDA library (which has its own mesh builder, its own
element matrix and its own solver) and takes its inputs from ``workloads``.

Modules
-------
``mesh``    leaves -> canonical node numbering, connectivity, hanging-node
            constraints (paper Sec. 6, Eq. 6), Dirichlet mask.
``fem``     the B8 reference stiffness K0, sparse assembly of K(rho) (Eq. 1-2),
            the constraint operator C = [I; P] and the reduced system
            A = C^T K C, f = C^T f_full (Eq. 7-9).
``solve``   sparse direct solve of the reduced system, Jacobi-PCG.
``topopt``  compliance, element sensitivities, the filters (Eq. 3-5) and the
            optimality-criteria update.
``amr``     adaptation marks, the sibling and incompatibility sweeps, the new
            leaf set with density transfer (Sec. 4, 6) and Eq. 10.
``learn``   the learned initial guess (no paper counterpart): grid transfers,
            a 3D U-Net and its energy loss.
``coarse``  the two-level preconditioner (no paper counterpart): Galerkin coarse
            space on the base-grid lattice and its l1-Jacobi V-cycle.
``cpcg``    loader of ``pcg_omp.c``, Jacobi-PCG in C with OpenMP: the timed CPU
            baseline of the benchmark.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, exact rational
arithmetic, brute force on tiny inputs, finite differences, beam theory).
"""
