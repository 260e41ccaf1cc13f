"""FP64 CPU oracle for the Polar Express hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
product (the C-ABI library and its Python binding) never imports, links or
executes it, and shares no code with it.

Contents
--------
``minimax``   the offline stage: greedy minimax composition (Thm. 1), the
              degree-5 Remez solve (Alg. 3, App. F), the degree-3 closed form
              (Eq. deg3_solution), cushioning and the 1.01 safety factor
              (Sec. 3.4, App. G).
``iteration`` the online stage in FP64: Frobenius normalisation, the odd
              quintic iteration X <- aX + (bA + cA^2)X with A = X X^T on the
              short side (Alg. 1, Sec. 3.5 Horner form), its spectral form
              U p(S) V^T (App. C), polar via SVD (Eq. matrixsign) and the error
              metrics.
``spectrum_init`` the spectrum-aware initialisation of App. H (k = 1): power
              method lower bound z of sigma_1, the cubic of Eq. init_poly, and
              the table that puts it before the Polar Express steps.

Every function is pinned by ``tests/test_oracle_*.py`` against facts fixed by
the paper or by mathematics (printed table, equioscillation, closed forms,
invariants, library routines, brute force). The one claim left unpinned is the
``p(x)/x >= 0.236`` remark of App. G, which the oracle does not implement.
"""
from . import minimax, iteration, spectrum_init  # noqa: F401
from .minimax import (  # noqa: F401
    KAPPA,
    NoConvergence,
    gepp_solve,
    optimal_cubic,
    optimal_quintic,
    optimal_composition,
    newton_schulz5_table,
    jordan_table,
    eval_odd,
)
from .iteration import (  # noqa: F401
    normalise,
    fast_rectangular,
    fast_rectangular_spectral,
    polar_express,
    polar_express_spectral,
    compose_scalar,
    polar_svd,
    polar_2x2,
    err_polar_fro,
    max_sigma_err,
    restricted_errors,
    rel_fro,
)
