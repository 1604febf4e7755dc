"""FP64 CPU oracle of the PSTT2 hot path (Shi, Ruth & Townsend, "Parallel
algorithms for computing the tensor-train decomposition", Sec. 2-3).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import, call or run anything in this package.  The product
path (the CUDA library and its binding) never does, and shares no code with it;
the two meet only in the seeded input generators of `ttinputs`, which hold none
of the method's arithmetic.

Modules:
  philox   the counter-based Gaussian stream (Philox4x32-10 + Box-Muller)
  linalg   Householder CPQR / QR and the right least-squares solve
  tt       unfoldings, TT contraction, TT-SVD (Sec. 2)
  pstt2    PSTT2 / PSTT2-onepass step by step, slab streaming (Sec. 3.2, 4.2)
  grad     reference gradient of the one-pass map (torch CPU float64 autograd)

Pins (tests/test_oracle_*.py): Philox known-answer vectors published with
Random123; Gaussian moments; CPQR/QR/LS against LAPACK through numpy/scipy;
TT contraction against a brute-force loop; exact recovery of random low-rank
TT tensors; the deterministic error bound of Theorem 3.2 (eq. proj_acc) per
run; the d = 2 reduction to the randomized range finder; the Frobenius bound
of TT-SVD; Table 1's TT sizes.  Functions without such a pin say so.
"""
