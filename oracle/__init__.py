"""FP64 CPU oracle for the TPCG hot path of "A low-rank isogeometric solver based on Tucker
tensors" (Montardini, Sangalli, Tani).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import anything from this package.  The CUDA path shares no code with
it; the only shared module is ``synth`` (seeded inputs, no arithmetic of the method).

Every routine is plain numpy/scipy in float64 and follows the paper step by step:

  bspline   -- Cox-de Boor B-splines, Gauss quadrature, univariate mass/stiffness (Sec. 2.1, App. A)
  geometry  -- parametric coefficients Q = det(J) J^-1 J^-T and omega = det(J) f (App. A)
  lowrank   -- Chebyshev-sampled low-rank approximation of Q and omega, Tucker operator and rhs
               (App. A, eq. matrix_CP), folded into a Kronecker sum
  tucker    -- Tucker vectors/matrices: full tensor, m-mode product, matvec, dot, sum (Sec. 2.3)
  rounding  -- ST-HOSVD, relative truncation (Alg. 1), dynamic truncation (Alg. 2)
  fd        -- exact FD (Alg. 3), approximate eigenpairs (App. B), exponential sums (Prop. 1),
               low-rank FD application (Alg. 4)
  tpcg      -- TPCG (Alg. 5)
  fullcg    -- assembled Kronecker-sum matrix and full-vector PCG (reference for tiny n)

Functions without an independent pin say "parity unpinned" in their docstring.
"""
