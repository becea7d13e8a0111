"""FP64 CPU oracle of the embedded-boundary (EB) method of Peng, Appelo & Liu,
"Universal AMG accelerated embedded boundary method without small cell
stiffness" (arXiv 2204.06083).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or calls
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library; both consume the seeded descriptors of
``eb_inputs``.

It is written for readability, not speed: plain numpy / scipy, every step in
the paper's order, each function citing the passage it follows.

Modules
  geometry  level sets, node classification, grid-line / boundary roots
            (Sec. 2, mask m_ij and boundary / computational points; Sec. 2.1)
  eb        line-by-line closure, CSR assembly of A = -L and the right-hand
            side (Sec. 2.1, Algorithm 1 steps 1-3), the segment matrices
            D^(n)(a,b) of Lemma 1 / Theorem 2, ghost-point negative control
  amg       deterministic smoothed-aggregation AMG (the paper delegates AMG to
            a library, Sec. 3 preamble), V-cycle with Chebyshev smoothing
  solvers   CG / PCG (Algorithm 1 step 4), dense Cholesky, Lanczos
            extremes, leapfrog and theta-method time stepping (Sec. 3.4-3.5)
  cnn       the learned correction stage added to the preconditioner (no
            counterpart in the paper): network forward / backward, energy-norm
            loss, solver-generated training pairs, Adam, flexible PCG

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against a closed form, an invariant the paper states,
the paper's Table 1, or brute force on tiny inputs.
"""
