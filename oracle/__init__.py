"""Oracle: a plain, slow, FP64 CPU restatement of the data-aware distance
estimation path of "Effective and General Distance Computation for
Approximate Nearest Neighbor Search" (arXiv 2404.16322).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import,
call, link or run anything in it.  The product path (the CUDA library and
its Python binding) never touches it, and it shares no code with that path:
no kernels, headers, helpers, tables or pre/post-processing.

Modules and the passages they follow:

* ``pca``      -- PCA rotation (Section IV-B, Theorem 1, Eq. 2; the Remark
                  on decorrelation; data centred per the footnote of IV-B);
                  the Haar-random rotation of ADS (Section III).
* ``ivf``      -- IVF candidate generation: Lloyd k-means, assignment and
                  top-nprobe probing (Section II-A).
* ``storage``  -- the stored precision of the rotated slabs (FP32, BF16
                  round-to-nearest-even, FP8-E4M3 with per-dimension scale).
* ``search``   -- the refinement loop: partial distances over Delta_d steps
                  (Algorithm 2 loop structure), the learned test
                  ``m1_s * dis' + beta_s > tau`` (Section V-A/B,
                  "Incremental Correction"), exact distance at d = D, and
                  the result queue with threshold tau (Section I); the RES
                  (Section IV-C), ADS (Section III) and OPQ-L (Section V-B)
                  tests.  The loops are plain C (``search.c``), wrapped by
                  ctypes.
* ``pq``       -- OPQ-L's product quantiser: OPQ's dimension allocation,
                  codebooks, codes, tables, quantisation errors.
* ``fit``      -- the data-driven correction: labelled samples, logistic
                  regression, the beta' adjustment to a target label-0
                  recall, one classifier per step (Section V-A/B); OPQ-L's
                  three-feature classifier.
* ``knn``      -- exact brute-force KNN (Section II-A definition).

Parity status: every function is pinned by a ``-m "not gpu"`` test against
closed forms, invariants, library special cases or brute force, except the
*values* of the fitted classifiers (m1_s, beta'_s; OPQ-L's m1, m3, beta'),
which have no closed form:
parity unpinned for those values (only their defining constraints --
label-0 recall >= r_s, the beta' quantile, the IRLS optimum -- are pinned).
"""
