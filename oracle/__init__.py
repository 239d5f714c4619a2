"""FP64 CPU oracle for the constrained forward-dynamics step (TEST INFRASTRUCTURE ONLY).

This package is the slow, plain reference that the CUDA path is checked against.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it; the
product path (the C-ABI library and its Python binding) never calls it and has no CPU fallback.
It shares no code with the CUDA path: both consume the world descriptions of ``worldgen`` and
nothing else.

What it computes, in the paper's order (Kamino, arXiv 2603.16536):

* ``rigid``       -- Sec. 3: maximal-coordinate body state, the block-diagonal mass matrix (Eq. 1),
                     Newton-Euler forces h, semi-implicit Euler with the SO(3) exponential map.
* ``constraints`` -- Sec. 3: joint constraints f(q) = 0 (loop closures are ordinary joints),
                     Signorini-Coulomb contacts in (t1, t2, n) frames, Baumgarte bias v*, the dense
                     constraint Jacobian J; joint coordinates with implicit PD / armature / damping
                     rows (Eq. 2's R and v*) and unilateral joint limits.
* ``padmm``       -- Sec. 4: Delassus matrix and free velocity (Eq. 4), the Jacobi preconditioner,
                     the De Saxce operator, the friction-cone projection and Proximal-ADMM
                     (Alg. 1) with Nesterov acceleration and adaptive restart; Sec. 5.1's sparse
                     formulation: the matrix-free Delassus operator and a Conjugate Residual x-step
                     warm-started at the previous iterate.
* ``timestep``    -- one full time step of a set of worlds (Eq. 2 solved through Alg. 1), with
                     the cached warm start; semi-implicit Euler or the Moreau-Jean midpoint scheme.
* ``audit``       -- independent checks: the direct KKT solve of Eq. 2 for bilateral-only worlds
                     and the natural-map NCP residual of a returned (lambda, u+).
* ``kinematics``  -- Sec. 6.3: Gauss-Newton forward kinematics, consistent poses from joint
                     coordinates for resets of mechanisms with loops.
* ``mlp``         -- the warm-start network (3 GELU layers) forward, loss and backward in FP64,
                     the reference for the GPU kernels' gradients.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants or brute force; none is "parity unpinned".
"""
from .timestep import SolverParams, WorldState, step, simulate, initial_state  # noqa: F401
