"""FP64 CPU oracle for the mini-batch quasi-Newton proximal method (BQNPM/MQNPM).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the GPU hot path computes.  Only the test-suite, the
``smoke()`` check of ``__graft_entry__`` and the CPU-baseline / reference leg
of ``bench.py`` may import it.  The CUDA library never calls it, shares no
code with it and has no fallback to it.

Modules
-------
physics  Lippmann-Schwinger / first-Born forward model, detector, data term
         f_l, gradient by the adjoint solve (Section 6; the discretisation is
         our stated reading, the paper defers it to a supplement).
tv       finite differences D^d (Section 3.1), discrete TV (Eqs. 3.1-3.2),
         its dual map d(P) and the projection onto the dual ball (Eqs. 3.3-3.4).
wprox    structured weighted proximal mapping: Woodbury inverse (Section 4.3),
         prox of the box under tau*I + U U^T (Theorem 3.1) by semi-smooth Newton
         (Algorithm 4.3), and the dual fast projected gradient on T(P)
         (Eq. 4.10, Lemma 4.1).
sr1      the memory-efficient SR1 estimate of B_s (Algorithm 4.2).
bqnpm    the outer loop (Algorithm 4.1) with strategies I and II.

Parity status: every function listed above is pinned by a ``-m "not gpu"``
test in tests/test_oracle_*.py against a closed form, a brute-force or
independent solver, or a mathematical invariant.
"""
