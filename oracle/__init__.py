"""FP64 CPU oracle of the FastMap first-order solve (test infrastructure).

This package is a plain, slow, obviously-correct restatement of what the
paper's objectives, gradients and optimiser compute, in float64 numpy.  It is
TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never imports, links or calls anything here, and nothing
here imports the CUDA library: the two share no code; the only shared module
is the seeded input generator ``synthetic.scenes``.

Modules and what pins them (pins live in ``tests/test_oracle_*.py``):
  so3          6D rotation representation (Sec. 3.3, Zhou et al.) and the
               geodesic distance (Eq. 4)      -- pinned by round trip,
               orthonormality, finite differences, closed-form angles.
  epipolar     epipolar adjustment, direct L1 (Eq. 7), L2 / IRLS (Eqs. 8-9),
               the compact 9x9 form (Eq. 8, Appendix "Epipolar Adjustment",
               Eqs. 15-17)
                                               -- pinned by zero loss at
               noise-free ground truth, similarity invariance, the
               direct == compact identity, brute-force per-pair loops and
               central finite differences.
  rotation     global rotation loss (Eq. 3) and the modified Martinec-Pajdla
               initialisation (Appendix "Global Rotation", Eqs. 10-14)
                                               -- pinned by zero loss at
               ground truth, right-multiplication gauge invariance, exact
               recovery on noise-free rotations, finite differences.
  translation  global translation loss (Eqs. 5-6) and the multi-init merge
               (Appendix "Multiple Initializations")
                                               -- pinned by zero loss at
               ground truth, shift / positive-scale invariance, finite
               differences.
  adam         Adam (Kingma & Ba), the paper's cited first-order optimiser
                                               -- pinned by a hand-computed
               two-step example.
  mlp          learned per-pair inlier weights (the learned extension; the
               paper has none): features, the 8-64-64-1 GELU network, its
               binary cross-entropy and hand-derived gradient, bfloat16
               emulation            -- pinned by torch's bfloat16 conversion
               and float64 autograd, central finite differences, closed forms
               with zero weights, a per-pair feature loop, invariances and the
               generator's track lengths.
"""
