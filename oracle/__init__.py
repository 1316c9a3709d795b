"""CPU FP64 oracle for the well-conditioned IPM Newton solve (arXiv 2407.14013).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA library (no kernels, headers, tables or helpers);
the only common module is ``workloads`` (seeded input generators).

Modules
-------
linalg     svec / smat / Psi_n / symmetric Kronecker product (Notations).
operators  the constraint operator A and its adjoint for the three storage
           kinds, written from <A_i, X> (eq. sdp-pd, A3).
newton     NT scaling (eq. newt) and the Newton direction of (Newt-eps) by the
           plain definition: Schur-complement elimination, and a dense full
           KKT solve for tiny n.
reform     the paper's reformulation, step by step: the split (eq. EQSigdef),
           the matrix-free products of Section 5, the augmented system and the
           recovery (eq. augsys / recover), the block preconditioner of
           Section 6 and the indefinite PCG of Cor. pcg / Def. pcg.
lpcone     the nonnegative variables of Section 7's robust problems (eq. rmc-sdp)
           in the Newton system: plain definition, dense KKT, and the
           reformulation with the linear block and its preconditioner.
ipm_lp     the outer loop with those variables (the method of ipm.py plus the
           orthant), its directions from the reformulated solve, and the
           re-centring at a fixed mu used by the derivative pins.
grad       the implicit derivative of the optimum (vector-Jacobian product):
           one Newton solve at the final scaling point, with and without the
           orthant.
ipm        a textbook infeasible primal-dual NT path-following method (the
           outer loop; the paper leaves it to SeDuMi, so its details are the
           oracle's own definitions -- parity unpinned beyond its invariants).
maxcut     brute-force cut enumeration for tiny graphs (a pin).

All arithmetic is numpy/scipy float64.
"""
