"""FP64 CPU oracle of SPARTan's PARAFAC2-ALS (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference arm may import this package.  The CUDA path never does, and the
two share no code.
"""
from .parafac2 import (  # noqa: F401
    RANK_RTOL, subject_block, all_blocks, procrustes_q, form_y, mttkrp_spartan,
    pinv_sym, normalize_columns, cp_als_sweep, surrogate_loss, exact_loss, norm_x_sq,
    fit_from_loss, als_iteration, parafac2_als, assemble_u, project_subject,
)
