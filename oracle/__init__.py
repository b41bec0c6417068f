"""CPU oracle for temporal 3-path sampling (Pu et al., ICDM 2024).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it; the two meet only on the inputs
that the seeded generators produce.

Contents (each function names the passage it follows):
  * ``compile_motif``     -- anchor choice and 3-path class (Alg. 5, Def. 5)
  * ``build_csr``         -- time-sorted out/in/pair lists (Sec. III, III-B)
  * ``path_weights``      -- w_e = product of windowed degrees (Claim 1, Alg. 1)
  * ``prefix_sum``        -- W and the cumulative weights (Alg. 1)
  * ``philox4x32_10``     -- counter RNG of Salmon et al. (SC'11)
  * ``bounded``           -- Lemire's bounded draw (ACM TOMACS 2019)
  * ``sample_run``        -- Sample + CheckMotif over sample ids (Alg. 2, 3, 5)
  * ``list_count``        -- ListCount (Alg. 4, reading fixed below)
  * ``path_sum``          -- sum over all anchor-class paths of CheckMotif
                             (proof of Claim 2: equals the exact count C)
  * ``exact_count``       -- chronological backtracking count of M-matches (Def. 2)
  * ``brute_force_count`` -- literal Def. 2 over all edge tuples (tiny graphs)
  * ``set_threads``       -- OpenMP threads of the loops above (default 1:
                             serial; integer results identical)
  * ``estimate``          -- C_hat = (sum X / k) * W (Alg. 5) and its standard error
  * ``learned``           -- features, FP64 network, proposal sampler (learned proposal)

Parity of every function here is pinned by the ``-m "not gpu"`` tests against
closed forms, brute force and published known answers; see the test files.
"""
from .core import *  # noqa: F401,F403
from . import learned  # noqa: F401
