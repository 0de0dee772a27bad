"""CPU oracle for the masked sparse-DFT LASSO interior-point method.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
what the method computes, written from the paper (arXiv 2502.04217) so that a
reader can check it against the paper by eye.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  The product path (the CUDA library and its Python binding) never imports,
calls or links anything here, and nothing here imports the product path.

Modules
-------
mapping   the real parametrisation beta <-> v of a conjugate-symmetric
          spectrum (Sec. 3, Eq. (beta), Eq. (v), Eq. (map)); the 2D/3D
          analogue is our own reading (the paper defers it to package docs).
dft       the orthonormal DFT / IDFT by explicit Vandermonde matrices
          (Sec. 3, the matrix C), one axis at a time (separable definition).
lasso     the masked operators M_perp, M_perp^T (Sec. 3.1, Eq. (xi)),
          the LASSO objective (Eq. (realopt)) and a duality-gap certificate.
ipm       the primal-dual interior-point method: Newton system (Eq. (augkkt)),
          condensed KKT operator K (Eq. (condensedkkt)), the preconditioner P
          and its closed-form inverse (Eq. (invprecond1), Prop. exprbd), PCG,
          back-substitution and step rule (Sec. 3.3-3.5).
brute     independent solvers for tiny instances used as pins: active-set
          enumeration and proximal gradient; soft-thresholding closed form.
warmstart the learned warm start (not in the paper): features, the 3D
          convolution network, its loss and gradients, in plain numpy FP64.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, numpy/scipy library routines, invariants the paper
proves, or brute force on tiny inputs.  No function is "parity unpinned".
"""
