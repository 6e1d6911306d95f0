"""Plain FP64 CPU oracle for adaptive hypergraph learning -- TEST INFRASTRUCTURE.

This package is the correctness reference for the CUDA library in
``paper_1908_08281_gb300``.  It is slow and written to be checked against the paper
by eye: numpy / scipy in float64, one step per equation, no blocking, fusion or
reordering beyond what the definitions state.  It shares no code with the CUDA path
and neither imports the other; the only common code is the seeded input generator
module ``synth``, which holds none of the method's arithmetic.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import anything from here.  The product path never routes
through it.

Notation: n vertices, m hyperedges (the paper, Section 2, swaps the two letters),
c right-hand-side columns; H is the n x m 0/1 incidence matrix, w the hyperedge
weights, dv = H w (weighted vertex degrees), de = H^T 1 (hyperedge sizes),
Theta = Dv^-1/2 H W De^-1 H^T Dv^-1/2 (the paper's A, Eq. 1), Delta = I - Theta
(Zhou's normalised Laplacian), and the ranking system of Eqs. 3 and 6 in the
equivalent symmetric form  M F = lam Y,  M = (1 + lam) I - Theta.

Functions and their pins (tests/test_oracle_*.py):
  incidence.build_incidence      pinned: dense brute force, scipy CSR->CSC
  core.theta_dense / theta_apply pinned: triple-loop brute force, invariants,
                                 networkx normalised Laplacian (2-uniform case),
                                 rank-one single-edge case, k-regular closed form
  core.solve_dense / cg_solve    pinned: residual, error certificate, CG identities,
                                 Chebyshev iteration bound
  core.weight_grad               pinned: central differences, torch.autograd of a
                                 dense objective, dv-frozen reading
  core.project_simplex           pinned: KKT conditions, brute force over supports
  rsvd.*                         pinned: exact low-rank blocks vs eigh, HMT bound,
                                 orthonormality, Woodbury identity
  philox.*                       pinned: published Philox4x32-10 known answers
"""
from . import core, incidence, philox, rsvd  # noqa: F401
