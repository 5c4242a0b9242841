"""CPU oracle for the recursive-linearization hot path (TEST INFRASTRUCTURE ONLY).

Plain, slow, FP64 NumPy/SciPy restatement of what the method computes at one
frequency k (paper Sec. 2 and Sec. 3): forward scattering by a contrast q on
Omega = [-1, 1]^2, the scattered field read on the circle of radius R
(eq. farfielddef), its Frechet derivative with respect to the sine-series
coefficients (Theorem 3.1, eqs. vdef and sineseries) and the Gauss-Newton
update from the normal equations (eq. normaleq).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA library and
never imports it; the two meet only through the seeded inputs of ``synth``.

Reading of the discretisation (the paper defers the solver's internals to the
HPS literature, Sec. 2): the forward map is the solution of one global
spectral-collocation system -- 16 x 16 Chebyshev-Lobatto grids on a uniform
n_L x n_L quadtree of leaves, continuity of u and of its normal derivative on
leaf interfaces, and on the boundary of Omega the exterior Green identity
(D - I/2) u_s = S d_n u_s (Sec. 2, Remark) discretised by Nystrom on the
leaf-edge panels.  The GPU solver reaches the solution of that same system
by hierarchical merges; the oracle assembles it whole and hands it to a
sparse direct solver.  Every function cites the passage it follows.

Parity status of each function (see the pins in tests/test_oracle_*.py):
pinned against closed forms, brute force or invariants; none is unpinned.
"""
