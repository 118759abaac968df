"""Plain float64 CPU oracle for the Nystrom-preconditioned reconstruction path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls, links or
executes this package: only the tests, the smoke check and the CPU-baseline leg
of the benchmark use it.  It shares no code with the CUDA library (no kernels,
headers, helpers, tables or constant generators); the only module both sides
use is `workloads`, which holds seeded input data and none of the method.

Each module restates the paper's definitions and algorithms in plain numpy,
slowly and obviously, one step at a time:
  philox    -- Philox4x32-10 + Box-Muller for the Gaussian test matrix (Alg. 1 step 1)
  operators -- blur, blur + decimation, Joseph ray transform, Haar, first and
               second differences (Sec. IV, Appendix A)
  nystrom   -- Algorithm 1 and the preconditioner of Eq. (RYPreconditioner)
  prox      -- Theorem 1 prox (semi-smooth Newton) and the dual APG prox (Sec. III-B)
  wapg      -- Algorithm 3 (WAPG / APG), power-iteration step size, objectives
  unroll    -- K unrolled Algorithm 3 iterations (TV) and their hand-derived
               reverse-mode gradient with respect to lambda and the blur kernel
  irm       -- Algorithm 2 (IRM for l_p - l_q) with PCG and the on-the-fly
               Nystrom preconditioner
Every function is pinned by a `-m "not gpu"` test against something other than
itself (closed forms, invariants, brute force, published test vectors); see
the tests named test_oracle_*.
"""
from . import operators, philox, nystrom, prox, wapg, unroll, irm  # noqa: F401
