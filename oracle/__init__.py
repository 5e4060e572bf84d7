"""CPU oracle for mixed-precision LOBPCG (Kressner, Ma, Shao, arXiv 2302.12528).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's algorithms in NumPy/SciPy (FP64 unless the paper
fixes the precision: the "lower" precision parts run in float32 / complex64,
Section 5, first paragraph).  It shares no code with the CUDA library and never
imports it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the product path never routes through it.

Modules
  dense     -- norm estimate (Section 5.1), stopping test (Eq. stop),
               lower-precision Cholesky with the breakdown shift policy, the
               preconditioner application T = Pi L^-* L^-1 Pi^* (Section 5.1).
  mqr       -- Algorithm 2 (mixed-precision QR).
  lobpcg    -- Algorithm 3 (two-stage mixed-precision LOBPCG) and the
               DLOBPCG-dchol / DLOBPCG-schol variants (Section 5.1);
               Algorithm 1 (mixed-precision PINVIT).
  symbolic  -- grid nested-dissection ordering, elimination tree, column
               counts, fundamental supernodes, level schedule (the sparse
               Cholesky structure the paper takes from CHOLMOD, Section 5.1).
  sparse    -- CSR helpers and the lower-precision sparse factor by definition.
  bounds    -- the rounding-error quantities of Section 4 (Lemma 1, Lemma 2,
               Theorem 1) used as test pins.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(brute-force eigh, closed-form Laplacian spectra, diagonal matrices,
invariants, Section 4 bounds, boolean elimination).  Iteration counts are
"parity unpinned": the paper's iteration counts (Section 5.3) are for
matrices that are not available.
"""
