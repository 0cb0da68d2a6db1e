"""FP64 CPU oracle for the rational time stepper of Haut, Babb, Martinsson and
Wingate, "A high-order scheme for solving wave propagation problems via the
direct construction of an approximate time-evolution operator".

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the GPU path computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
or run anything here; the product library never does, and it shares no code,
tables or helpers with this package (only the seeded input generators in
``workloads`` serve both).

Modules
-------
rational   -- rational approximants R(z) = sum_m b_m / (z - alpha_m) of e^z on
              the imaginary axis (Section 1.2, eqs. def_RM, RM_prop1, RM_prop2),
              the oracle's own least-squares fit, and an evaluator of the
              Table 1 rational (Section 3.2).
sem        -- multidomain Chebyshev collocation (Section 2.2, eq. Bu=f).
resolvent  -- the elliptic reformulations of Section 2.1 on the global sparse
              system and the rational step (Section 1.1; Section 3.3 for the
              conjugate-pole form).
reference  -- the semi-discrete wave operator as a dense matrix, its exact
              exponential by eigendecomposition, and RK4 (the independent
              references of the self-checks).

Every function computes in FP64.  Each is pinned by a ``-m "not gpu"`` test
against a closed form, a printed value of the paper, an invariant or an
independent dense construction; none is "parity unpinned".
"""
