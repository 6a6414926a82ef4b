"""FP64 CPU oracle for SPCG (Sequential Preconditioned Conjugate Gradient).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the package
``paper_2607_25272_b300`` and its CUDA library) imports, links or runs
anything here.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it.

The oracle is plain, slow and written from the paper's definitions:

* ``philox``  - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the
  Feistel permutation built on it (the random draws of the SRHT, Sec. 2.1).
* ``srht``    - the nested SRHT construction (Sec. 2.2): Z = H D P X', the
  nested row sets I_1 c ... c I_K and the independent preconditioner sample.
* ``linalg``  - Householder QR, the OLS estimator (Eq. ols) and the R factor
  of the sketched Hessian (Sec. 2.2, Sec. 4 experimental setup).
* ``spcg``    - PCG(A, b, H, beta_init, a) (Sec. 2.2), Algorithm 1 (SPCG),
  the default schedule (Sec. 4) and the Theorem 3.3 iteration bound.
* ``metrics`` - the prediction errors used by the paper (Sec. 4) and the
  relative OLS prediction error.

Precision: IEEE FP64 throughout (numpy float64, round to nearest even, no
fast math).  Library primitives (BLAS matrix-vector products, LAPACK's
Householder QR, triangular solves) serve as single steps only.

Parity status of each function is stated in its module header.
"""
