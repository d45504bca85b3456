"""Plain FP64 CPU oracle of the HyRes hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path
(``paper_2204_06979_gb300``) never imports it, links it or falls back to it.

The oracle shares no code with the CUDA path: it has its own wavelet filters,
regression, eigensolver call, SURE evaluation and reconstruction, written as
slow, direct numpy in float64 so each step can be checked against the method
by eye. Every function cites the passage it follows.
"""

from .hyres import (  # noqa: F401
    db2_filters, gram, noise_est_regression, noise_est_schur, noise_est_lstsq,
    whiten_gram, eig_desc, padded_shape, pad_symmetric, dwt2, idwt2,
    soft_threshold, lambda_grid, sure_table, sure_rank_lambda,
    select_rank_lambda, select_rank_lambda_per_component, sure_table_levels,
    select_rank_lambda_per_level, hyres,
    rel_l2, psnr, sam, level_map, hyres_scaled, hyres_scaled_grad, mse_loss,
    sure_loss_scaled,
)
from .hysime import hysime, hysime_noise, hysime_select  # noqa: F401,E402
from .hyminor import (  # noqa: F401,E402
    hyminor, tvl1_split_bregman, tvl1_objective,
)
