"""FP64 CPU oracle for Algorithm 1 of arXiv 2310.17556 (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
and imports nothing from it.
"""

from .alg1 import (  # noqa: F401
    NotPositiveDefinite,
    apply_operator,
    back_substitution_transposed,
    cholesky_lower,
    errors,
    forward_substitution,
    gram,
    residual_n_space,
    solve,
    solve_batched,
    solve_steps,
    sr_scores,
)
from .exact import solve_dense_exact  # noqa: F401
from .complex_sr import real_part_scores, solve_complex  # noqa: F401
