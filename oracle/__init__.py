"""Plain FP64 CPU oracle for the RFM + IPN/AMIPN hot path (arXiv 2510.04170).

TEST INFRASTRUCTURE ONLY.  This package is a slow, obviously-correct restatement
of the method, written from the paper and from the published definitions of the
algorithms it names (Philox4x32-10, Householder QR, Paige-Saunders LSQR,
golden-section search).  It shares no code with the CUDA library.  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference
leg may import it; the product path never does.

Modules
  philox     counter-based RNG, features, count-sketch hashes, Gaussian sketch
  problem    subdomains, collocation rows, manufactured data          (Sec. 2.2, Sec. 5)
  assemble   residual F, Jacobian J, row scaling                      (Alg. 3, Sec. 5)
  linalg     sketch, Householder QR, triangular solves, LSQR          (Sec. 4.1)
  newton     golden-section line search, IPN, AMIPN, evaluation       (Alg. 1, Alg. 2)
"""
