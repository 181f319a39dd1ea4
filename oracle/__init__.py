"""FP64 CPU oracle of the C-A / CUR method (arXiv:1611.01391, Section 6.5,
Section 12.2 and Appendix F).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the product package.

Pins (tests marked ``not gpu``): exact recovery of rank-l inputs with a
nonsingular cross (Section 6.5); Eckart-Young lower bound (Lemma 2.3, letrnc);
brute-force maximal volume on tiny strips; GEPP pivot order against LAPACK
getrf; Moore-Penrose identities of the nucleus; Cauchy determinant closed
form for the generator; full residual equals the Appendix F estimate when the
sample is the whole matrix; Table tb_ranrc error levels (Section 12.3).
"""
from .ca import (CAP, GEPP, STOP, SWAP, Cauchy, CrossResult, Dense, Gauss,
                 InvDist, OracleSingular, columns, cross_approximation,
                 cross_approximation_adaptive, draw_columns, splitmix64, cynical, ca_cynical,
                 top_svd_of_cur, sampling_scores, exactly_sample, refine_by_leverage,
                 abridged_hadamard, butterfly, aph_left, aph_right, Preprocessed, recover_lra,
                 full_residual, gepp_rows, maxvol, nucleus, random_cross, rows,
                 sampled_residual)
from .rf_lsr import (RangeFinderFailure, RangeFinderResult, asph_columns, asph_rows, dual_lsr,
                     lsr_solution, numerical_rank, range_finder, relative_residual)

__all__ = [
    "CAP", "GEPP", "STOP", "SWAP", "Cauchy", "CrossResult", "Dense", "Gauss",
    "InvDist", "OracleSingular", "columns", "cross_approximation",
    "cross_approximation_adaptive", "draw_columns", "splitmix64", "cynical", "ca_cynical",
    "top_svd_of_cur", "sampling_scores", "exactly_sample", "refine_by_leverage",
    "abridged_hadamard", "butterfly", "aph_left", "aph_right", "Preprocessed", "recover_lra",
    "full_residual", "gepp_rows", "maxvol", "nucleus", "random_cross", "rows",
    "sampled_residual",
    "RangeFinderFailure", "RangeFinderResult", "asph_columns", "asph_rows", "dual_lsr", "lsr_solution",
    "numerical_rank", "range_finder", "relative_residual",
]
