"""Range finder (Algorithm 5.1a with a sub-identity multiplier) and superfast
dual LSR (Algorithm 3.1 with a sub-identity multiplier) through the C ABI,
against the FP64 oracle fed the same stored entries: the pivot order, the
subspace of U, V, the error and its Appendix F estimate; the LSR solution,
the sampled residual and the relative residual of the paper's tables."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import error_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1611_01391_gb300 as L  # noqa: E402

DEV = "cuda:0"
TAU = 1e-6


@pytest.fixture(scope="module")
def ctx():
    c = L.Context(0)
    yield c
    c.close()


def _rf(ctx, A32, J, r, rows=None, cols=None, **mult):
    m, n = A32.shape
    src = L.make_source("dense", a=torch.from_numpy(A32).to(DEV))
    U = torch.empty((m, r), dtype=torch.float32, device=DEV)
    V = torch.empty((r, n), dtype=torch.float32, device=DEV)
    res = L.lra_range_finder(ctx.ctx, src, J, r, U, V, rank_tol=TAU, resid_rows=rows, resid_cols=cols, **mult)
    torch.cuda.synchronize()
    return res, U.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("m,n,r,l,noise", [(3000, 2600, 10, 16, 1e-4), (4099, 1037, 24, 32, 1e-3),
                                           (20001, 513, 48, 64, 1e-4), (777, 6000, 5, 5, 1e-5)])
def test_range_finder_against_the_oracle(ctx, m, n, r, l, noise):
    A32 = W.factor_gaussian(9000 + m, m, n, r, noise)
    A = A32.astype(np.float64)
    J = W.draw_indices(9100 + n, n, l)
    rows, cols = W.draw_indices(9200, m, min(m, 500), sort=True), W.draw_indices(9300, n, min(n, 500), sort=True)
    res, U, V = _rf(ctx, A32, J, r, rows, cols)
    assert res["status"] == L.LRA_OK
    ref = O.range_finder(A, J, r, rank_tol=TAU)
    assert res["nrank"] == ref.nrank
    # the pivots of the leading r columns: the same wherever the remaining
    # norms are separated (always here: continuous random data)
    np.testing.assert_array_equal(res["piv"][:r], ref.piv[:r])
    # U: orthonormal to FP32 accuracy, spanning the oracle's subspace
    np.testing.assert_allclose(U.T @ U, np.eye(r), atol=1e-5)
    assert np.linalg.norm(U @ U.T @ ref.U - ref.U, 2) <= 1e-5
    # V against U^T M in FP64 from the device's own U (the GEMM's accuracy)
    V64 = U.T @ A
    assert np.abs(V - V64).max() <= 1e-5 * np.abs(V64).max()
    err = np.linalg.norm(A - U @ V) / np.linalg.norm(A)
    err_ref = np.linalg.norm(A - ref.U @ ref.V) / np.linalg.norm(A)
    assert error_ok(err, err_ref), (err, err_ref)
    est = O.sampled_residual(O.Dense(A32), U, np.eye(r), V, rows, cols)["rel"]
    assert res["est_rel_err"] == pytest.approx(est, rel=1e-4)
    assert res["gemm_mode"] in (0, 1)


@pytest.mark.parametrize("m,n,r,l,d", [(3000, 2048, 12, 20, 3), (1500, 4096, 24, 32, 6)])
def test_range_finder_with_an_asph_multiplier(ctx, m, n, r, l, d):
    """H = the first l columns of H_{n,d} P D (column t: sign[t] times column
    perm[t] of the abridged Hadamard matrix): the device forms Y = M H in
    FP32 butterfly sums, the oracle as the FP64 product with the dense H."""
    A32 = W.factor_gaussian(9050 + d, m, n, r, 1e-4)
    A = A32.astype(np.float64)
    rng = W.rng_for(9060 + d)
    perm, sign = rng.permutation(n), rng.choice([-1.0, 1.0], n)
    res, U, V = _rf(ctx, A32, perm[:l], r, mult_d=d, mult_sign=sign[:l])
    assert res["status"] == L.LRA_OK
    ref = O.range_finder(A, O.asph_columns(n, d, perm, sign, l), r, rank_tol=TAU)
    assert res["nrank"] == ref.nrank
    np.testing.assert_array_equal(res["piv"][:r], ref.piv[:r])
    assert np.linalg.norm(U @ U.T @ ref.U - ref.U, 2) <= 1e-5
    err = np.linalg.norm(A - U @ V) / np.linalg.norm(A)
    err_ref = np.linalg.norm(A - ref.U @ ref.V) / np.linalg.norm(A)
    assert error_ok(err, err_ref), (err, err_ref)


def test_range_finder_reports_failure_below_the_target_rank(ctx):
    """Stage 1 of Algorithm 5.1: FAILURE when nrank(M H) < r (a rank-5 matrix
    stored in FP32: its rounding is far below the rank tolerance)."""
    A32 = W.factor_gaussian(9400, 2000, 1500, 5, 0.0)
    res, _, _ = _rf(ctx, A32, W.draw_indices(9401, 1500, 12), 8)
    assert res["status"] == L.LRA_ESINGULAR
    assert res["nrank"] == 5
    assert res["nrank"] == O.range_finder(A32.astype(np.float64), W.draw_indices(9401, 1500, 12), 5,
                                          rank_tol=TAU).nrank


def test_range_finder_rejects_bad_arguments(ctx):
    A32 = W.factor_gaussian(9500, 300, 200, 4, 1e-3)
    src = L.make_source("dense", a=torch.from_numpy(A32).to(DEV))
    U = torch.empty((300, 8), dtype=torch.float32, device=DEV)
    V = torch.empty((8, 200), dtype=torch.float32, device=DEV)
    for J, r in (([0, 1, 2, 3, 4, 5, 6, 6], 4), (list(range(8)), 9), (list(range(97)), 8)):
        with pytest.raises(L.LraError) as e:
            L.lra_range_finder(ctx.ctx, src, J, r, U, V)
        assert e.value.code == L.LRA_EINVAL
    x, y = W.cauchy_points(9501, 300, 200)
    gen = L.make_source("cauchy", x=torch.from_numpy(x).to(DEV), y=torch.from_numpy(y).to(DEV))
    with pytest.raises(L.LraError) as e:
        L.lra_range_finder(ctx.ctx, gen, list(range(8)), 4, U, V)
    assert e.value.code == L.LRA_EINVAL


def _lsr(ctx, A, b, rows, passes=3, shifted=True, dtype=np.float64, **mult):
    Wm = np.ascontiguousarray(np.concatenate([A, b[:, None]], axis=1).astype(dtype))
    src = L.make_source("dense", a=torch.from_numpy(Wm).to(DEV))
    return L.lra_dual_lsr(ctx.ctx, src, rows, passes=passes, shifted=shifted, **mult)


@pytest.mark.parametrize("m,n,k", [(4096, 100, 600), (16384, 400, 2400), (3000, 37, 111)])
def test_dual_lsr_gaussian_against_the_oracle(ctx, m, n, k):
    A, b = W.lsr_problem(9600 + n, "gaussian", m, n)
    rows = W.rng_for(9700 + n).permutation(m)[:k]
    x, rho = _lsr(ctx, A, b, rows)
    xr = O.dual_lsr(A, b, rows)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-10 * np.abs(xr).max())
    assert rho == pytest.approx(np.linalg.norm(A[rows] @ xr - b[rows]), rel=1e-10)
    assert O.relative_residual(A, b, x) == pytest.approx(O.relative_residual(A, b, xr), rel=1e-10)


def test_dual_lsr_fp32_storage(ctx):
    """W stored in FP32: the rows are the FP32 values promoted to FP64."""
    A, b = W.lsr_problem(9800, "gaussian", 4096, 64)
    A32, b32 = A.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    rows = W.rng_for(9801).permutation(4096)[:400]
    x, _ = _lsr(ctx, A32, b32, rows, dtype=np.float32)
    xr = O.dual_lsr(A32, b32, rows)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-10 * np.abs(xr).max())


def test_dual_lsr_ill_conditioned_rows(ctx):
    """The ill-conditioned class (singular values 10^4 .. 10^-9, the rest
    10^-10, condition 1e14): four passes, two of them shifted, factor the sampled rows and
    its solution's residual on them is no larger than that of the oracle's
    least squares solution (which truncates singular values below its rcond;
    the device solves the full-rank problem, so x itself differs along the
    directions of the tiny singular values)."""
    A, b = W.lsr_problem(9900, "ill", 4096, 100)
    rows = W.rng_for(9901).permutation(4096)[:600]
    x, rho = _lsr(ctx, A, b, rows, passes=4)
    xr = O.dual_lsr(A, b, rows)
    rho_ref = np.linalg.norm(A[rows] @ xr - b[rows])
    assert np.linalg.norm(A[rows] @ x - b[rows]) <= (1 + 1e-6) * rho_ref
    # |x| reaches 1e10 along the tiny directions: A x carries ~1e-5 relative rounding
    assert rho == pytest.approx(np.linalg.norm(A[rows] @ x - b[rows]), rel=1e-3)


def test_dual_lsr_rank_deficient_sample_is_reported(ctx):
    """The coherent class A = [D_n; 0]: a row sample that misses rows of D
    leaves columns of the sampled A at zero (the hard inputs of the
    superfast recipe); the device reports a non-positive pivot."""
    A, b = W.lsr_problem(9950, "coherent", 4096, 100)
    rows = W.rng_for(9951).permutation(4096)[:600]
    assert np.linalg.matrix_rank(A[rows]) < 100
    with pytest.raises(L.LraError) as e:
        _lsr(ctx, A, b, rows)
    assert e.value.code == L.LRA_ESINGULAR


@pytest.mark.parametrize("kind,d", [("gaussian", 3), ("coherent", 8), ("semicoherent", 6)])
def test_dual_lsr_with_an_asph_multiplier(ctx, kind, d):
    """F = k rows of D P H_{m,d} (row t: sign[t] times row perm[t] of the
    abridged Hadamard matrix) at (k, m, n) = (600, 4096, 100): the device's
    FP64 butterfly sums against the oracle's dense F.  On the coherent and
    semi-coherent classes, where row sampling alone leaves the sampled
    problem rank-deficient, the ASPH rows mix the rows of D (Tables lsrsemi,
    lsrcoh use 6- and 8-ASPH)."""
    A, b = W.lsr_problem(9970 + d, kind, 4096, 100)
    rng = W.rng_for(9980 + d)
    perm, sign = rng.permutation(4096), rng.choice([-1.0, 1.0], 4096)
    x, rho = _lsr(ctx, A, b, perm[:600], mult_d=d, mult_sign=sign[:600])
    F = O.asph_rows(4096, d, perm, sign, 600)
    xr = O.dual_lsr(A, b, F)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-9 * np.abs(xr).max())
    assert rho == pytest.approx(np.linalg.norm(F @ A @ xr - F @ b), rel=1e-9)
    assert 1.0 <= O.relative_residual(A, b, x) <= 1.3


def test_dual_lsr_asph_sample_can_still_be_rank_deficient(ctx):
    """With d = 6 on the coherent class, rows 64 apart share an offset: two
    columns of D stay dependent when every sampled row of their offset has
    the same parity of its block index (here twice: rank 98), and the device
    reports it."""
    A, b = W.lsr_problem(9976, "coherent", 4096, 100)
    rng = W.rng_for(9986)
    perm, sign = rng.permutation(4096), rng.choice([-1.0, 1.0], 4096)
    assert np.linalg.matrix_rank(O.asph_rows(4096, 6, perm, sign, 600) @ A) < 100
    with pytest.raises(L.LraError) as e:
        _lsr(ctx, A, b, perm[:600], mult_d=6, mult_sign=sign[:600])
    assert e.value.code == L.LRA_ESINGULAR


def test_dual_lsr_rejects_bad_arguments(ctx):
    A, b = W.lsr_problem(9960, "gaussian", 500, 20)
    for rows, kw in ((np.arange(10), {}), (np.array([0] * 30), {}), (np.arange(30), {"passes": 5})):
        with pytest.raises(L.LraError) as e:
            _lsr(ctx, A, b, rows, **kw)
        assert e.value.code == L.LRA_EINVAL
