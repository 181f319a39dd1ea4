"""The pins bite: plant a plausible mistake in a copy of an oracle function
(a dropped term, a flipped sign, a transposed operand, a swapped factor) and
check that at least one pin of ``test_oracle_pins`` then fails.  Mutants live
only in this process, on the CPU."""
import inspect

import pytest

import oracle
import oracle.ca as ca
from tests import test_oracle_pins as pins


def _mutant(func, old, new):
    src = inspect.getsource(func)
    assert old in src, f"mutation anchor not found in {func.__name__}: {old!r}"
    ns = dict(vars(ca))
    exec(src.replace(old, new, 1), ns)
    return ns[func.__name__]


def _run_pins(checks):
    """True when at least one check raises."""
    for check in checks:
        try:
            check()
        except Exception:
            return True
    return False


MUTANTS = [
    # maxvol: drop the -e_j term of the rank-one update
    ("maxvol", "r[j] -= 1.0", "pass",
     [lambda: pins.test_maxvol_volume_grows_by_recorded_factor(),
      lambda: pins.test_maxvol_dominant_and_locally_maximal(3)]),
    # maxvol: transposed operand when forming B
    ("maxvol", "np.linalg.solve(X.T, S.T).T", "np.linalg.solve(X, S.T).T",
     [lambda: pins.test_maxvol_volume_grows_by_recorded_factor(),
      lambda: pins.test_exact_recovery_rank_l(60, 50, 5, 1)]),
    # maxvol: update with the wrong column of B
    ("maxvol", "np.outer(B[:, j], r)", "np.outer(B[:, (j + 1) % l], r)",
     [lambda: pins.test_maxvol_volume_grows_by_recorded_factor()]),
    # maxvol: position bookkeeping off (row stored in the wrong slot)
    ("maxvol", "I[j] = i", "I[(j + 1) % l] = i",
     [lambda: pins.test_maxvol_volume_grows_by_recorded_factor(),
      lambda: pins.test_maxvol_dominant_and_locally_maximal(5)]),
    # GEPP: wrong sign in the Schur complement update
    ("gepp_rows", "-= np.outer(mult", "+= np.outer(mult",
     [lambda: pins.test_gepp_pivots_match_lapack_getrf()]),
    # GEPP: pivot chosen by signed value instead of modulus
    ("gepp_rows", "np.abs(W[:, t])", "W[:, t]",
     [lambda: pins.test_gepp_pivots_match_lapack_getrf()]),
    # nucleus: left/right singular vectors swapped
    ("nucleus", "(QT[:k_eff].T / sigma[:k_eff]) @ P[:, :k_eff].T",
     "(P[:, :k_eff] / sigma[:k_eff]) @ QT[:k_eff]",
     [lambda: pins.test_nucleus_against_constructed_svd(5),
      lambda: pins.test_exact_recovery_rank_l(60, 50, 5, 1)]),
    # nucleus: sigma instead of 1/sigma
    ("nucleus", "/ sigma[:k_eff]", "* sigma[:k_eff]",
     [lambda: pins.test_nucleus_against_constructed_svd(5)]),
    # nucleus: truncation threshold ignored
    ("nucleus", "min(k, np.count_nonzero(sigma > rank_tol * sigma[0]))", "k",
     [lambda: pins.test_nucleus_against_constructed_svd(8)]),
    # Appendix F: nucleus dropped from the residual
    ("sampled_residual", "(np.asarray(C)[sr] @ U) @", "np.asarray(C)[sr] @",
     [lambda: pins.test_sampled_residual_on_whole_matrix_equals_full()]),
    # Appendix F: variance about zero instead of about the mean
    ("sampled_residual", "np.sum((E - mu) ** 2)", "np.sum(E ** 2)",
     [lambda: pins.test_sampled_residual_on_whole_matrix_equals_full()]),
    # runner-up: the winner's own value instead of the second largest (every
    # decision would then look unseparated)
    ("_runner_up", "return float(rest.max())", "return float(values[winner])",
     [lambda: pins.test_runner_up_of_gepp_decisions_is_second_largest_candidate(1),
      lambda: pins.test_runner_up_of_swap_decisions_is_second_largest_entry(5)]),
    # runner-up: the smallest remaining candidate instead of the largest
    ("_runner_up", "return float(rest.max())", "return float(rest.min())",
     [lambda: pins.test_runner_up_of_swap_decisions_is_second_largest_entry(6)]),
    # tolerance stop never taken
    ("cross_approximation", 'if estimate["rel"] <= tol:', 'if estimate["rel"] < 0.0:',
     [lambda: pins.test_tolerance_stop_at_the_first_sweep_whose_estimate_is_below_tol()]),
    # tolerance stop one sweep late (checks the estimate before the sweep)
    ("cross_approximation", 'if tol > 0.0 and sample_rows is not None:',
     'if tol > 0.0 and sample_rows is not None and s > 0:',
     [lambda: pins.test_tolerance_stop_at_the_first_sweep_whose_estimate_is_below_tol(),
      lambda: pins.test_tolerance_stop_on_exact_rank_after_one_sweep()]),
    # resume: the caller's row set ignored (restart from elimination)
    ("cross_approximation", "if s == 0 and I is None:", "if s == 0:",
     [lambda: pins.test_resume_from_checkpoint_equals_uninterrupted_run(1)]),
    # seed draw: last xor-shift of the mixer off by one bit
    ("splitmix64", "return state, z ^ (z >> 31)", "return state, z ^ (z >> 30)",
     [lambda: pins.test_splitmix64_published_outputs()]),
    # seed draw: Floyd's replacement step dropped (repeats possible)
    ("draw_columns", "v = c if t in seen else t", "v = t",
     [lambda: pins.test_draw_columns_distinct_in_range(0, 10, 10)]),
    # cynical: the submatrix's own row numbers returned instead of M's
    ("cynical", "I = [K[i] for i in inner.I]", "I = list(inner.I)",
     [lambda: pins.test_cynical_exact_on_rank_r("tests3"),
      lambda: pins.test_cynical_generator_lies_in_the_submatrix_and_is_dominant()]),
    # Tests 4: the inner step run on the initial columns instead of the outer loop's
    ("ca_cynical", "cynical(src, outer.I, outer.J,", "cynical(src, outer.I, L0,",
     [lambda: pins.test_tests4_outer_loop_is_one_ca_sweep_with_4r_generators()]),
    # refinement: inverse CDF taken with the wrong side at the interval ends
    ("exactly_sample", 'side="right"', 'side="left"',
     [lambda: pins.test_exactly_sample_maps_each_interval_to_its_index()]),
    # refinement: column and row scores swapped
    ("refine_by_leverage", "p_cols = sampling_scores(T)", "p_cols = sampling_scores(S[:len(T)])",
     [lambda: pins.test_refinement_reproduces_an_exact_rank_r_matrix(),
      lambda: pins.test_refinement_error_near_the_best_rank_r()]),
    # Algorithm D.1: the core without the nucleus
    ("top_svd_of_cur", "np.linalg.svd(Rc @ np.asarray(U, np.float64) @ Rr.T)", "np.linalg.svd(Rc @ Rr.T)",
     [lambda: pins.test_top_svd_of_cur_is_the_svd_of_the_product()]),
    # scores: norms instead of squared norms
    ("sampling_scores", "w = np.sum(V * V, axis=1)", "w = np.sqrt(np.sum(V * V, axis=1))",
     [lambda: pins.test_leverage_scores_of_an_exact_rank_r_matrix()]),
    # abridged Hadamard: the recursion's lower-right block without the minus
    ("abridged_hadamard", "H = np.block([[H, H], [H, -H]])", "H = np.block([[H, H], [H, H]])",
     [lambda: pins.test_abridged_hadamard_equals_the_printed_matrices()]),
    # recovery: H^T applied with the permutation instead of its inverse
    ("recover_lra", "Z[:, pre.pc] = Rbar * pre.sc[None, :]", "Z = Rbar[:, pre.pc] * pre.sc[None, pre.pc]",
     [lambda: pins.test_recovered_lra_error_is_the_preprocessed_error_over_2_to_d()]),
    ("recover_lra", "Y[pre.pr] = pre.sr[:, None] * Cbar", "Y = pre.sr[:, None] * Cbar[pre.pr]",
     [lambda: pins.test_recovered_lra_error_is_the_preprocessed_error_over_2_to_d()]),
    # recovery: the 2^d normalisation dropped on one side
    ("recover_lra", "for b in range(D)]).reshape(m, l) / D", "for b in range(D)]).reshape(m, l)",
     [lambda: pins.test_recovered_lra_error_is_the_preprocessed_error_over_2_to_d()]),
    # butterfly: a step that never subtracts
    ("butterfly", "vals = vals[0::2] + sig * vals[1::2]", "vals = vals[0::2] + vals[1::2]",
     [lambda: pins.test_preprocessed_entries_equal_F_M_H_exactly_on_small_integers()]),
    # butterfly: the sign of step k taken from the wrong bit of b
    ("butterfly", "(np.asarray(b) >> k) & 1", "(np.asarray(b) >> (d - 1 - k)) & 1",
     [lambda: pins.test_preprocessed_entries_equal_F_M_H_exactly_on_small_integers(),
      lambda: pins.test_butterfly_is_the_fast_walsh_transform_in_recursion_order()]),
    # butterfly: steps taken top bit first (the transform is the same, the order is not)
    ("butterfly", "vals = vals[0::2] + sig * vals[1::2]",
     "h = len(vals) // 2; sig = np.where((np.asarray(b) >> (d - 1 - k)) & 1, -1.0, 1.0); "
     "vals = vals[:h] + sig * vals[h:]",
     [lambda: pins.test_butterfly_is_the_fast_walsh_transform_in_recursion_order()]),
    # C-A: horizontal step chooses J inside R instead of R^T
    ("cross_approximation", "maxvol(R.T, J,", "maxvol(R[:, :l], J,",
     [lambda: pins.test_exact_recovery_rank_l(90, 120, 7, 3),
      lambda: pins.test_rank_one_picks_largest_factors()]),
]


@pytest.mark.parametrize("idx", range(len(MUTANTS)))
def test_mutant_is_caught(idx, monkeypatch):
    name, old, new, checks = MUTANTS[idx]
    bad = _mutant(getattr(ca, name), old, new)
    monkeypatch.setattr(ca, name, bad)
    monkeypatch.setattr(oracle, name, bad, raising=hasattr(oracle, name))
    assert _run_pins(checks), f"mutant {name}: {old!r} -> {new!r} survived"


def test_cauchy_sign_flip_is_caught(monkeypatch):
    """A sign flip of every entry leaves det unchanged at even n; the pin
    checks odd n too."""
    import numpy as np

    def flipped(self, rows, cols):
        xs, ys = self._pair(rows, cols)
        return (1.0 / (ys[..., 0] - xs[..., 0])).astype(np.float64)

    monkeypatch.setattr(ca.Cauchy, "block", flipped)
    assert _run_pins([lambda n=n: pins.test_cauchy_determinant_closed_form(n) for n in (3, 4, 5, 6)])


def test_cauchy_index_swap_is_caught(monkeypatch):
    import numpy as np

    def swapped(self, rows, cols):
        xs, ys = self._pair(cols, rows)
        return (1.0 / (xs[..., 0] - ys[..., 0])).T.astype(np.float64)

    monkeypatch.setattr(ca.Cauchy, "block", swapped)
    assert _run_pins([pins.test_cauchy_known_entries])
