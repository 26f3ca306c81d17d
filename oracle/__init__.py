"""CPU oracle for the online tensor method (Huang, Niranjan, Hakeem, Anandkumar).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 NumPy
restatement of the method, written from the paper.  It exists to check the
CUDA library.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library itself never does,
and this package never imports the library.  The two share no code: the only
common module is ``synth`` (seeded random inputs, no arithmetic of the method).

Modules and the part of the paper each follows:
  moments  -- Section 2.1 Eqs. (1)-(3) (topic moments), Section 2.2 Eqs. (7)-(11)
              (community moments, transition matrices Z_B, Z_C).
  whiten   -- Section 3.1 (whitening W^T M2 W = I), Section 4.2 (randomised
              low-rank whitening and pseudo-inverse, Algorithms 2 and 3).
  stgd     -- Section 3.2 (whitened tensor, loss Eq. (15), Lemma 3 / Eq. (16)
              stochastic update), Appendix A (gradient, shift operator); the
              same gradient with the whole Eq. (3) for topics (self-token
              terms kept).
  post     -- Section 3.3 Lemma 4 (eigenvalues, unwhitening, alpha estimate),
              plus the reconstruction error used to measure convergence.
  community-- Section 3.3 Lemma 4, community case (membership Pi_hat,
              thresholding) and the validation section (p-value graph,
              recovery ratio, average error).
  warmstart-- tensor sketches T(I, I, theta_j) and the warm-start MLP
              (forward, backward, Gram-Schmidt), not in the paper.

Every function states the passage it follows.  Readings of ambiguous or
garbled passages are listed in the design notes and repeated at the function.

Parity status: every function here is pinned by a CPU test against something
other than itself (brute-force counts, closed forms, library routines, finite
differences, exact recovery).  The paper's real-dataset tables are not
reproduced (their data are absent): parity unpinned for those numbers only.
"""
from . import moments, whiten, stgd, post, community, warmstart  # noqa: F401
