"""Pins of the range finder (Algorithm 5.1a) and dual LSR (Algorithm 3.1 with
sparse orthogonal multipliers) oracle, and mutants that the pins must catch.
CPU only."""
import inspect
import os

import numpy as np
import pytest

import oracle.rf_lsr as rl
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rank_r(seed, m, n, r, noise=0.0):
    rng = W.rng_for(seed)
    M = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    return M + noise * rng.standard_normal((m, n))


def _printed():
    rows = {}
    for line in open(os.path.join(GOLDEN, "lsr_tables.txt")):
        if line.startswith("#") or not line.strip():
            continue
        cls, mult, k, m, n, mean, std = line.split()
        rows[(cls, mult, int(k), int(m), int(n))] = (float(mean), float(std))
    return rows


# ---------------------------------------------------------------------------
# Algorithm 5.1a
# ---------------------------------------------------------------------------

def test_range_finder_is_exact_on_a_rank_r_matrix():
    """Y = M[:, J] spans range(M) when rank M = r <= l: U V = M."""
    M = _rank_r(8001, 300, 250, 7)
    J = W.draw_indices(8002, 250, 12)
    res = rl.range_finder(M, J, 7)
    assert res.nrank == 7
    np.testing.assert_allclose(res.U.T @ res.U, np.eye(7), atol=1e-13)
    assert np.linalg.norm(M - res.U @ res.V) <= 1e-12 * np.linalg.norm(M)


def test_range_finder_fails_below_the_target_rank():
    """Stage 1: FAILURE when nrank(M H) < r."""
    M = _rank_r(8003, 200, 150, 4)
    with pytest.raises(rl.RangeFinderFailure):
        rl.range_finder(M, W.draw_indices(8004, 150, 10), 5)


def test_range_finder_V_is_the_least_squares_factor_and_error_is_above_optimal():
    """V = U^+ M solves min ||U V - M||; the error is at least the
    Eckart-Young optimum of rank r (Lemma 2.3)."""
    M = _rank_r(8005, 240, 200, 10, noise=1e-3)
    res = rl.range_finder(M, W.draw_indices(8006, 200, 16), 10)
    V_ls = np.linalg.lstsq(res.U, M, rcond=None)[0]
    np.testing.assert_allclose(res.V, V_ls, atol=1e-10 * np.abs(V_ls).max())
    s = np.linalg.svd(M, compute_uv=False)
    err = np.linalg.norm(M - res.U @ res.V)
    assert err >= np.sqrt(np.sum(s[10:] ** 2)) * (1 - 1e-12)


def test_range_finder_pivots_are_the_largest_remaining_column():
    """Businger-Golub pivoting: each pivot is the column of Y whose component
    orthogonal to the columns already chosen has the largest norm (computed
    here by explicit projection, independently of the QR)."""
    M = _rank_r(8007, 120, 90, 9, noise=1e-2)
    J = W.draw_indices(8008, 90, 14)
    res = rl.range_finder(M, J, 9)
    Y = M[:, J]
    chosen = []
    for step in range(9):
        if chosen:
            Q = np.linalg.qr(Y[:, chosen])[0]
            Rm = Y - Q @ (Q.T @ Y)
        else:
            Rm = Y
        norms = np.linalg.norm(Rm, axis=0)
        norms[chosen] = -1.0
        best = int(np.argmax(norms))
        assert res.piv[step] == best
        assert abs(abs(res.R[step, step]) - norms[best]) <= 1e-10 * norms[best]
        chosen.append(best)


def test_asph_multipliers_have_orthogonal_columns_and_rows():
    rng = W.rng_for(8009)
    H = rl.asph_columns(64, 3, rng.permutation(64), rng.choice([-1.0, 1.0], 64), 20)
    np.testing.assert_array_equal(H.T @ H, 8 * np.eye(20))
    F = rl.asph_rows(96, 2, rng.permutation(96), rng.choice([-1.0, 1.0], 96), 30)
    np.testing.assert_array_equal(F @ F.T, 4 * np.eye(30))


def test_range_finder_with_asph_multiplier_is_near_optimal():
    """An ASPH multiplier with l = r + 8 columns on a rank-r matrix plus
    noise: the error stays within 3x the optimum for most draws."""
    ok = 0
    for t in range(5):
        M = _rank_r(8010 + t, 256, 256, 12, noise=1e-4)
        rng = W.rng_for(8020 + t)
        H = rl.asph_columns(256, 3, rng.permutation(256), rng.choice([-1.0, 1.0], 256), 20)
        res = rl.range_finder(M, H, 12)
        s = np.linalg.svd(M, compute_uv=False)
        ok += np.linalg.norm(M - res.U @ res.V) <= 3 * np.sqrt(np.sum(s[12:] ** 2))
    assert ok >= 4


# ---------------------------------------------------------------------------
# Algorithm 3.1, dual LSR
# ---------------------------------------------------------------------------

def test_lsr_with_every_row_is_the_exact_solution():
    A, b = W.lsr_problem(8030, "gaussian", 300, 20)
    x = rl.dual_lsr(A, b, np.arange(300))
    np.testing.assert_allclose(x, np.linalg.solve(A.T @ A, A.T @ b), rtol=1e-10)
    assert rl.relative_residual(A, b, x) == pytest.approx(1.0, abs=1e-12)


def test_lsr_sub_identity_is_the_least_squares_solution_of_the_kept_rows():
    A, b = W.lsr_problem(8031, "gaussian", 500, 12)
    rows = W.draw_indices(8032, 500, 60)
    x = rl.dual_lsr(A, b, rows)
    np.testing.assert_allclose(x, np.linalg.solve(A[rows].T @ A[rows], A[rows].T @ b[rows]), rtol=1e-10)
    assert rl.relative_residual(A, b, x) >= 1.0


def test_gaussian_sketch_meets_its_expected_residual():
    """For a k x m Gaussian multiplier (entries N(0, 1/k)) the expected squared
    residual is (1 + n / (k - n - 1)) times the optimum (the exact expectation
    of a Gaussian sketch of a least squares problem); 40 draws at
    (k, m, n) = (600, 4096, 100), within 3 standard errors."""
    A, b = W.lsr_problem(8040, "gaussian", 4096, 100)
    r2 = []
    for t in range(40):
        F = W.rng_for(8041 + t).standard_normal((600, 4096)) / np.sqrt(600)
        r2.append(rl.relative_residual(A, b, rl.dual_lsr(A, b, F)) ** 2)
    r2 = np.array(r2)
    expect = 1 + 100 / (600 - 100 - 1)
    assert abs(r2.mean() - expect) <= 3 * r2.std() / np.sqrt(len(r2))


def test_lsr_means_against_the_printed_tables():
    """Table lsrRandom, (k, m, n) = (600, 4096, 100): sub-identity sampling of a
    Gaussian input behaves as a Gaussian multiplier (its rows are Gaussian);
    3-ASPH likewise.  Means over 20 draws within two printed standard
    deviations of the printed means."""
    P = _printed()
    sub, asph = [], []
    for t in range(20):
        A, b = W.lsr_problem(8100 + t, "gaussian", 4096, 100)
        rng = W.rng_for(8200 + t)
        sub.append(rl.relative_residual(A, b, rl.dual_lsr(A, b, rng.permutation(4096)[:600])))
        F = rl.asph_rows(4096, 3, rng.permutation(4096), rng.choice([-1.0, 1.0], 4096), 600)
        asph.append(rl.relative_residual(A, b, rl.dual_lsr(A, b, F)))
    mean_g, std_g = P[("gaussian", "gaussian", 600, 4096, 100)]
    mean_h, std_h = P[("gaussian", "asph3", 600, 4096, 100)]
    assert abs(np.mean(sub) - mean_g) <= 2 * std_g, np.mean(sub)
    assert abs(np.mean(asph) - mean_h) <= 2 * std_h, np.mean(asph)


def test_relative_residual_is_scale_invariant():
    A, b = W.lsr_problem(8050, "semicoherent", 400, 16)
    x = rl.dual_lsr(A, b, W.draw_indices(8051, 400, 96))
    assert rl.relative_residual(3 * A, 3 * b, x) == pytest.approx(rl.relative_residual(A, b, x), rel=1e-12)


# ---------------------------------------------------------------------------
# mutants
# ---------------------------------------------------------------------------

def _mutant(func, old, new):
    src = inspect.getsource(func)
    assert old in src, f"mutation anchor not found in {func.__name__}: {old!r}"
    ns = dict(vars(rl))
    exec(src.replace(old, new, 1), ns)
    return ns[func.__name__]


MUTANTS = [
    # U taken one column late
    ("range_finder", "U = Q[:, :r]", "U = Q[:, 1:r + 1]",
     [test_range_finder_is_exact_on_a_rank_r_matrix]),
    # V with a transposed role (least squares factor taken from Y instead of M)
    ("range_finder", "V = U.T @ M", "V = U.T @ (M @ np.eye(M.shape[1])[:, ::-1])",
     [test_range_finder_V_is_the_least_squares_factor_and_error_is_above_optimal]),
    # no pivoting
    ("range_finder", 'mode="economic", pivoting=True)', 'mode="economic", pivoting=False) + (np.arange(Y.shape[1]),)',
     [test_range_finder_pivots_are_the_largest_remaining_column]),
    # rank counted against the last diagonal entry
    ("numerical_rank", "a > rank_tol * a[0]", "a > rank_tol * a[-1]",
     [test_range_finder_fails_below_the_target_rank]),
    # sampled rows of A with the wrong entries of b
    ("dual_lsr", "return lsr_solution(A[F], b[F])", "return lsr_solution(A[F], b[:len(F)])",
     [test_lsr_sub_identity_is_the_least_squares_solution_of_the_kept_rows]),
    # dense multiplier applied to A only
    ("dual_lsr", "return lsr_solution(F @ A, F @ b)", "return lsr_solution(F @ A, b[:F.shape[0]])",
     [test_gaussian_sketch_meets_its_expected_residual]),
    # ASPH columns without their signs
    ("asph_columns", "return H * np.asarray(sign, np.float64)[None, :l]", "return H",
     [test_range_finder_with_asph_multiplier_is_near_optimal, test_asph_multipliers_have_orthogonal_columns_and_rows,
      lambda: _asph_sign_check()]),
    # relative residual against ||b|| instead of the optimum
    ("relative_residual", "best = np.linalg.norm(A @ lsr_solution(A, b) - b)", "best = np.linalg.norm(b)",
     [test_lsr_with_every_row_is_the_exact_solution]),
]


def _asph_sign_check():
    """Column j of the multiplier is sign[j] times column perm[j] of H_{n,d}."""
    rng = W.rng_for(8300)
    perm, sign = rng.permutation(32), rng.choice([-1.0, 1.0], 32)
    H = rl.asph_columns(32, 2, perm, sign, 8)
    from oracle.ca import abridged_hadamard
    Hd = abridged_hadamard(32, 2)
    for j in range(8):
        np.testing.assert_array_equal(H[:, j], sign[j] * Hd[:, perm[j]])


def test_asph_columns_are_signed_columns_of_the_abridged_hadamard():
    _asph_sign_check()


@pytest.mark.parametrize("idx", range(len(MUTANTS)))
def test_mutant_is_caught(idx, monkeypatch):
    name, old, new, checks = MUTANTS[idx]
    bad = _mutant(getattr(rl, name), old, new)
    monkeypatch.setattr(rl, name, bad)
    caught = False
    for check in checks:
        try:
            check()
        except (Exception, pytest.fail.Exception):
            caught = True
            break
    assert caught, f"mutant {name}: {old!r} -> {new!r} survived"


# ---------------------------------------------------------------------------
# The device's rank floor for the sampled LSR (a reading: the paper does not
# say how a numerical method detects a rank-deficient sample)
# ---------------------------------------------------------------------------

def _cholesky_qr_pivot_ratios(Wm, passes, shifted=True):
    """Shifted CholeskyQR in FP64 as the device runs it (the first
    passes - 2 passes, at least one, on Y^T Y + s_rel tr(Y^T Y) I): for each
    pass, whether it was shifted and the smallest pivot R_jj^2 over the
    column's squared norm (None where the matrix is not positive definite)."""
    import scipy.linalg as sl
    k, c = Wm.shape
    s_rel = 11.0 * (k * c + c * (c + 1)) * 2.0 ** -53
    Q, out = np.array(Wm, np.float64), []
    for s in range(passes):
        G = Q.T @ Q
        shift_here = shifted and s < max(1, passes - 2)
        try:
            R = np.linalg.cholesky(G + (s_rel * np.trace(G) if shift_here else 0.0) * np.eye(c)).T
        except np.linalg.LinAlgError:
            out.append((shift_here, None))
            break
        with np.errstate(divide="ignore", invalid="ignore"):
            out.append((shift_here, float(np.nanmin(np.diag(R) ** 2 / np.diag(G)))))
        Q = sl.solve_triangular(R, Q.T, trans="T", lower=False).T
    return s_rel, out


def test_lsr_rank_floor_separates_valid_and_deficient_samples():
    """In an unshifted pass the device reports ESINGULAR below a pivot of
    1e-3 s_rel times the column's squared norm.  In FP64 the valid samples'
    unshifted pivots stay at least 1e5 times above that floor (Gaussian rows
    with three passes; the condition-1e14 class with four, two shifted),
    while the rank-deficient samples (coherent rows missing rows of D, and
    the 6-ASPH coherent sample of rank 98) break the first unshifted pass."""
    k, m, n = 600, 4096, 100
    valid = []
    A, b = W.lsr_problem(9900, "gaussian", m, n)
    rows = W.rng_for(9901).permutation(m)[:k]
    valid.append((np.concatenate([A[rows], b[rows, None]], axis=1), 3))
    A, b = W.lsr_problem(9900, "ill", m, n)
    valid.append((np.concatenate([A[rows], b[rows, None]], axis=1), 4))
    for Wm, passes in valid:
        s_rel, out = _cholesky_qr_pivot_ratios(Wm, passes)
        assert len(out) == passes and all(r is not None for _, r in out)
        plain = [r for sh, r in out if not sh]
        assert plain and min(plain) >= 1e5 * (1e-3 * s_rel), out
    deficient = []
    A, b = W.lsr_problem(9950, "coherent", m, n)
    rows = W.rng_for(9951).permutation(m)[:k]
    deficient.append(np.concatenate([A[rows], b[rows, None]], axis=1))
    A, b = W.lsr_problem(9976, "coherent", m, n)
    rng = W.rng_for(9986)
    perm, sign = rng.permutation(m), rng.choice([-1.0, 1.0], m)
    F = rl.asph_rows(m, 6, perm, sign, k)
    deficient.append(np.concatenate([F @ A, (F @ b)[:, None]], axis=1))
    for Wm in deficient:
        assert np.linalg.matrix_rank(Wm[:, :n]) < n
        s_rel, out = _cholesky_qr_pivot_ratios(Wm, 3)
        first_plain = next(r for sh, r in out if not sh)
        assert first_plain is None or first_plain <= 1e-3 * s_rel, out
