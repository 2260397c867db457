"""FP64 CPU oracle for the LMA hot path — TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The GPU library never calls it, and it
shares no code with the CUDA path: it is written from the paper's
definitions with numpy/scipy library primitives (Cholesky, triangular
solves, matrix products) as steps.

  lma_dense   the dense definition: R-bar by the recursion of Eq. (ares),
              Sigma-bar by Eq. (acov), predictive mean/variance by
              Eqs. (vapmu)/(vapvar), log N(y; mu, Sigma-bar_DD); plus the
              textbook full GP and the PIC prior used as special-case pins.
  lma_oracle  the summary form: local summaries (Definition 1), global
              summary (Definition 2), Theorem 2, the local-route prediction,
              the log-likelihood in summary form and its hand adjoint.
"""
