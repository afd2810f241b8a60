"""FP64 CPU oracle for the spacetime-multigrid smoke-control method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code with
the CUDA library (``paper_1608_01102_gb300/csrc``) and imports nothing from
the product package.

Every function is a plain, slow, fp64 restatement of the paper
(Pan & Manocha, "Efficient Optimal Control of Smoke using Spacetime
Multigrid"), citing the section / equation / algorithm it follows, on the
2D grid (``mac.Grid``) and the 3D grid (``mac.Grid3``; ``kkt.Problem(nz=..)``):

* ``mac``        -- staggered (MAC) grid operators: div, grad, vorticity form
                    self-advection Adv (Sec. 3.1, Eq. NSA), QUICK upwind
                    passive advection matrix A(v) (Sec. 3.1, Eq. Conv).
* ``advection``  -- truncated Taylor exponential A[rho, v] (Eq. Adv) and its
                    two adjoints (Eq. KKTPO).
* ``projection`` -- exact solenoidal projection Q (Eq. KKTPO).
* ``metric``     -- keyframe metric C_i = c_i sum G^T G (Sec. 4.1).
* ``kkt``        -- reduced objective / gradient, relative KKT residual,
                    NSO residual f (Eq. KKTAO, Appendix A).
* ``scgs``       -- temporally augmented SCGS smoother (Eq. HESS, Sec. 4.3).
* ``stfas``      -- restriction / prolongation and the FAS V-cycle (Alg. 2).
* ``admm``       -- AO fixed point (Alg. 1) and the ADMM outer loop (Alg. 3).
* ``brute``      -- full-resimulation gradient-descent reference solver
                    (the gradient-based comparison of Sec. 5) for tiny grids.

Parity status: every function listed above is pinned by ``tests/`` against
closed forms, library routines, finite differences or invariants (the 3D
operators also against the pinned 2D ones on each coordinate plane), except the
full ADMM solve, whose agreement with the paper's own runs is unpinned (the
paper's workloads are not available); only its self-consistency is pinned.
"""
