"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Pivot parity: the GPU's decision log must agree with the oracle's (fed the
same FP32 entries) on every decision up to the first genuine near-tie
(competing volume ratios within 1e-6).  Error parity: the GPU's CUR must have
a relative Frobenius error within 1.05x of the pure-FP64 oracle's, or 1e-5.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import GPU_TAU, check_nucleus, compare_traces, error_ok, rel_fro_error, sampled_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1611_01391_gb300 as L  # noqa: E402

DELTA = 1e-2
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    c = L.Context(0)
    yield c
    c.close()


def gpu_solve(ctx, src, m, n, J0, k, l, sweeps, rows=None, cols=None, trace_cap=8192,
              rank_tol=1e-6, tol=0.0, delta=DELTA):
    params, keep = L.make_params(k, l, sweeps, J0, delta=delta, rank_tol=rank_tol, tol=tol,
                                 resid_rows=rows, resid_cols=cols, trace_cap=trace_cap)
    res = ctx.solve(src, params, l, m, n, want_strips=True, trace_cap=trace_cap, device=DEV)
    assert res.info.status == 0, L.lra_status_str(res.info.status)
    res.C = res.C.cpu().numpy()
    res.R = res.R.cpu().numpy()
    return res


def as_oracle_trace(res):
    return [tuple(int(v) for v in row) for row in res.trace]


# ---------------------------------------------------------------------------
# Dense FP64 256 x 256, rank 8 + noise (std 1e-4), k = l = 8, 3 sweeps
# ---------------------------------------------------------------------------

def test_dense_f64_small_parity(ctx):
    A = W.lowrank_svd(W.BASE_SEED + 1)
    J0 = W.draw_indices(W.BASE_SEED + 101, 256, 8)
    a = torch.from_numpy(A).to(DEV)
    res = gpu_solve(ctx, L.make_source("dense", a=a), 256, 256, J0, 8, 8, 3)
    ref = O.cross_approximation(O.Dense(A.astype(np.float32)), J0, k=8, sweeps=3, delta=DELTA,
                                rank_tol=GPU_TAU)
    ncmp, div = compare_traces(res.trace, ref.trace, DELTA)
    assert ncmp > 8
    if div is None:
        assert list(res.I) == ref.I and list(res.J) == ref.J
        np.testing.assert_allclose(res.U, ref.U, rtol=0, atol=1e-9 * np.abs(ref.U).max())
        np.testing.assert_allclose(res.sigma, ref.sigma, rtol=1e-10, atol=1e-14 * ref.sigma[0])
    assert res.info.k_eff == ref.k_eff
    ref64 = O.cross_approximation(O.Dense(A), J0, k=8, sweeps=3, delta=DELTA)
    err64 = O.full_residual(O.Dense(A), ref64.C, ref64.U, ref64.R)[0]
    assert error_ok(rel_fro_error(A, res.C, res.U, res.R), err64)
    assert res.info.sweeps_done == 3 and res.info.converged == 1


# ---------------------------------------------------------------------------
# Generated Cauchy 1/(x_i - y_j), k = 16, l = 24, 4 sweeps, 1000 x 1000 sample
# ---------------------------------------------------------------------------

def _cauchy_case(ctx, m, n, seed):
    x, y = W.cauchy_points(seed, m, n)
    J0 = W.draw_indices(seed + 100, n, 24)
    rows = W.draw_indices(seed + 200, m, min(1000, m), sort=True)
    cols = W.draw_indices(seed + 300, n, min(1000, n), sort=True)
    xd, yd = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
    res = gpu_solve(ctx, L.make_source("cauchy", x=xd, y=yd), m, n, J0, 16, 24, 4, rows, cols)
    src32 = O.Cauchy(x, y, "fp32")
    ref = O.cross_approximation(src32, J0, k=16, sweeps=4, delta=DELTA, rank_tol=GPU_TAU,
                                sample_rows=rows, sample_cols=cols)
    ncmp, div = compare_traces(res.trace, ref.trace, DELTA)
    assert ncmp >= 24
    if div is None:
        assert list(res.I) == ref.I and list(res.J) == ref.J
        assert res.info.k_eff == ref.k_eff
    # U and sigma element by element against the FP64 nucleus of the same
    # cross (the Cauchy crosses have kappa ~ 1e8 in their FP32 entries)
    X32 = src32.block(res.I, res.J)
    s = np.linalg.svd(X32, compute_uv=False)
    assert s[0] / s[-1] > 1e6            # the ill-conditioned case this checks
    check_nucleus(res.U, res.sigma, res.info.k_eff, X32, 16)
    src64 = O.Cauchy(x, y, "fp64")
    ref64 = O.cross_approximation(src64, J0, k=16, sweeps=4, delta=DELTA,
                                  sample_rows=rows, sample_cols=cols)
    err_gpu = sampled_error(src64, res.C, res.U, res.R, rows, cols)
    assert error_ok(err_gpu, ref64.estimate["rel"]), (err_gpu, ref64.estimate["rel"])
    # the device's own Appendix F estimate matches the oracle's on the same factors
    est = O.sampled_residual(src32, res.C.astype(np.float64), res.U,
                             res.R.astype(np.float64), rows, cols)
    assert res.info.est_rel_err == pytest.approx(est["rel"], rel=1e-4)
    assert res.info.est_mu == pytest.approx(est["mu"], rel=1e-3, abs=1e-9 * abs(est["rel"]))
    assert res.info.est_var == pytest.approx(est["var"], rel=1e-3)
    return res, ref


def test_cauchy_reduced_parity(ctx):
    _cauchy_case(ctx, 6000, 7000, W.BASE_SEED + 12)


def test_cauchy_full_size_parity(ctx):
    """65536 x 65536 generated Cauchy in the launch configuration the
    benchmark times."""
    _cauchy_case(ctx, 65536, 65536, W.BASE_SEED + 2)


# ---------------------------------------------------------------------------
# Dense stored FP32, rank 64 + noise, k = 64, l = 96 (several CTAs per strip)
# ---------------------------------------------------------------------------

def test_dense_f32_l96_parity(ctx):
    m, n = 3000, 2500
    A = W.factor_gaussian(W.BASE_SEED + 33, m, n, 64, 1e-4)
    J0 = W.draw_indices(W.BASE_SEED + 133, n, 96)
    res = gpu_solve(ctx, L.make_source("dense", a=torch.from_numpy(A).to(DEV)), m, n, J0, 64, 96, 4)
    ref = O.cross_approximation(O.Dense(A), J0, k=64, sweeps=4, delta=DELTA, rank_tol=GPU_TAU)
    ncmp, div = compare_traces(res.trace, ref.trace, DELTA)
    assert ncmp >= 96
    if div is None:
        assert list(res.I) == ref.I and list(res.J) == ref.J
    A64 = A.astype(np.float64)
    assert error_ok(rel_fro_error(A64, res.C, res.U, res.R),
                    O.full_residual(O.Dense(A64), ref.C, ref.U, ref.R)[0])
    ref = O.cross_approximation(O.Dense(A64), J0, k=64, sweeps=4, delta=DELTA)
    err_ref = O.full_residual(O.Dense(A64), ref.C, ref.U, ref.R)[0]
    assert error_ok(rel_fro_error(A64, res.C, res.U, res.R), err_ref)


# ---------------------------------------------------------------------------
# Gathers are bit-exact copies / evaluations of the entries
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["dense32", "dense64", "cauchy", "invdist", "gauss"])
def test_strips_bit_exact(ctx, kind):
    m, n, l = 1037, 901, 7
    J0 = W.draw_indices(5, n, l)
    if kind.startswith("dense"):
        A = W.lowrank_svd(6, m, n, r=5, noise_std=1e-3)
        A = A.astype(np.float32) if kind == "dense32" else A
        src = L.make_source("dense", a=torch.from_numpy(A).to(DEV))
        ref = O.Dense(A.astype(np.float32))
    elif kind == "cauchy":
        x, y = W.cauchy_points(7, m, n)
        src = L.make_source("cauchy", x=torch.from_numpy(x).to(DEV), y=torch.from_numpy(y).to(DEV))
        ref = O.Cauchy(x, y, "fp32")
    else:
        x = W.cloud_points(8, m)
        y = W.cloud_points(9, n, lo=2.0, hi=3.0)
        xd, yd = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
        if kind == "invdist":
            src = L.make_source("invdist", x=xd, y=yd)
            ref = O.InvDist(x, y, "fp32")
        else:
            src = L.make_source("gauss", x=xd, y=yd, h=0.5 * np.sqrt(2.0) * 2.0)
            ref = O.Gauss(x, y, 0.5 * np.sqrt(2.0) * 2.0, "fp32")
    res = gpu_solve(ctx, src, m, n, J0, l, l, 2)
    C_ref = ref.block(np.arange(m), res.J)
    R_ref = ref.block(res.I, np.arange(n))
    if kind == "gauss":   # expf is not reproducible bit for bit: a few ulp
        np.testing.assert_allclose(res.C, C_ref, rtol=5e-7, atol=0)
        np.testing.assert_allclose(res.R, R_ref, rtol=5e-7, atol=0)
    else:
        np.testing.assert_array_equal(res.C.astype(np.float64), C_ref)
        np.testing.assert_array_equal(res.R.astype(np.float64), R_ref)


# ---------------------------------------------------------------------------
# Shapes: single CTA, ragged chunks, l = 1, l = min(m, n), k < l
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,n,l,k,sweeps", [
    (50, 40, 1, 1, 2), (64, 64, 3, 2, 3), (9, 300, 9, 9, 2), (777, 12, 12, 5, 3),
    (4099, 3001, 17, 11, 2), (20001, 513, 33, 20, 2), (1500, 1499, 96, 50, 2)])
def test_shapes_parity(ctx, m, n, l, k, sweeps):
    A = W.factor_gaussian(m * 7 + n, m, n, max(1, l // 2 + 1), 1e-3)
    J0 = W.draw_indices(m + 3 * n, n, l)
    res = gpu_solve(ctx, L.make_source("dense", a=torch.from_numpy(A).to(DEV)), m, n, J0, k, l, sweeps)
    ref = O.cross_approximation(O.Dense(A), J0, k=k, sweeps=sweeps, delta=DELTA, rank_tol=GPU_TAU)
    ncmp, div = compare_traces(res.trace, ref.trace, DELTA)
    if div is None:
        assert list(res.I) == ref.I and list(res.J) == ref.J
        assert res.info.k_eff == ref.k_eff
        np.testing.assert_allclose(res.sigma, ref.sigma, rtol=1e-9, atol=1e-12 * ref.sigma[0])
    check_nucleus(res.U, res.sigma, res.info.k_eff, A[np.ix_(res.I, res.J)], k)
    A64 = A.astype(np.float64)
    assert error_ok(rel_fro_error(A64, res.C, res.U, res.R),
                    O.full_residual(O.Dense(A64), ref.C, ref.U, ref.R)[0])
    ref = O.cross_approximation(O.Dense(A64), J0, k=k, sweeps=sweeps, delta=DELTA)
    err_ref = O.full_residual(O.Dense(A64), ref.C, ref.U, ref.R)[0]
    assert error_ok(rel_fro_error(A64, res.C, res.U, res.R), err_ref)


def test_invdist_and_gauss_error_parity(ctx):
    m, n = 3000, 2600
    x = W.cloud_points(41, m)
    y = W.cloud_points(42, n, lo=2.0, hi=3.0)
    J0 = W.draw_indices(43, n, 24)
    rows = W.draw_indices(44, m, 500, sort=True)
    cols = W.draw_indices(45, n, 500, sort=True)
    xd, yd = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
    # Truncation ranks sit at spectral gaps of the cross: where sigma_k ~
    # sigma_{k+1} (e.g. k = 16, l = 24, h = 1.5 on this cloud) the rank-k
    # truncation is ill posed and one-ulp changes of the entries move the
    # error by +-15% in the oracle itself.
    for kind, k, l, h in (("invdist", 16, 24, 0.0), ("gauss", 10, 16, 1.5), ("gauss", 12, 16, 1.0)):
        src = L.make_source(kind, x=xd, y=yd, h=h)
        res = gpu_solve(ctx, src, m, n, J0[:l], k, l, 3, rows, cols)
        src64 = O.InvDist(x, y, "fp64") if kind == "invdist" else O.Gauss(x, y, h, "fp64")
        err = sampled_error(src64, res.C, res.U, res.R, rows, cols)
        ref64 = O.cross_approximation(src64, J0[:l], k=k, sweeps=3, delta=DELTA,
                                      sample_rows=rows, sample_cols=cols)
        assert error_ok(err, ref64.estimate["rel"]), (kind, k, l, err, ref64.estimate["rel"])


# ---------------------------------------------------------------------------
# Status paths, early stop, determinism
# ---------------------------------------------------------------------------

def test_nonfinite_entry_is_reported(ctx):
    A = W.lowrank_svd(3, 200, 150, r=4, noise_std=1e-3).astype(np.float32)
    A[17, :] = np.nan
    params, keep = L.make_params(4, 4, 2, W.draw_indices(1, 150, 4))
    job = ctx.submit(L.make_source("dense", a=torch.from_numpy(A).to(DEV)), params)
    info = L.lra_cross_wait(ctx.ctx, job)
    assert info.status == L.LRA_ENONFINITE
    L.lra_cross_cancel(ctx.ctx, job)


def test_singular_strip_is_reported(ctx):
    A = np.zeros((100, 80), np.float32)
    A[:, 5] = 1.0
    params, keep = L.make_params(3, 3, 1, [5, 6, 7])
    job = ctx.submit(L.make_source("dense", a=torch.from_numpy(A).to(DEV)), params)
    info = L.lra_cross_wait(ctx.ctx, job)
    assert info.status == L.LRA_ESINGULAR
    L.lra_cross_cancel(ctx.ctx, job)


def test_tolerance_stops_early(ctx):
    A = W.factor_gaussian(77, 2000, 1800, 10, 0.0)
    rows = W.draw_indices(78, 2000, 300, sort=True)
    cols = W.draw_indices(79, 1800, 300, sort=True)
    res = gpu_solve(ctx, L.make_source("dense", a=torch.from_numpy(A).to(DEV)), 2000, 1800,
                    W.draw_indices(80, 1800, 12), 10, 12, 8, rows, cols, tol=1e-4)
    assert res.info.sweeps_done < 8
    assert res.info.est_rel_err <= 1e-4


def test_invalid_arguments_rejected(ctx):
    A = torch.zeros((10, 10), device=DEV)
    src = L.make_source("dense", a=A)
    for kw in (dict(k=5, l=4), dict(k=1, l=11), dict(k=1, l=0)):
        l = kw["l"]
        params, keep = L.make_params(kw["k"], max(l, 1), 1, list(range(max(l, 1))))
        params.l = l
        with pytest.raises(L.LraError) as e:
            ctx.submit(src, params)
        assert e.value.code == L.LRA_EINVAL
    params, keep = L.make_params(2, 2, 1, [3, 3])
    with pytest.raises(L.LraError):
        ctx.submit(src, params)


def test_repeat_is_bit_identical(ctx):
    x, y = W.cauchy_points(91, 20000, 15000)
    xd, yd = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
    rows = W.draw_indices(92, 20000, 400, sort=True)
    cols = W.draw_indices(93, 15000, 400, sort=True)
    src = L.make_source("cauchy", x=xd, y=yd)
    a = gpu_solve(ctx, src, 20000, 15000, W.draw_indices(94, 15000, 24), 16, 24, 3, rows, cols)
    b = gpu_solve(ctx, src, 20000, 15000, W.draw_indices(94, 15000, 24), 16, 24, 3, rows, cols)
    assert np.array_equal(a.I, b.I) and np.array_equal(a.J, b.J)
    assert np.array_equal(a.U, b.U)
    assert a.info.est_rel_err == b.info.est_rel_err


# ---------------------------------------------------------------------------
# Stored FP32 32768 x 32768 (the benchmark's stored workload, same bytes):
# decision log, index sets and the tensor-core full residual against FP64
# ---------------------------------------------------------------------------

def test_dense_32768_full_size_parity(ctx):
    import bench
    wl = bench.WORKLOADS["dense32768"]
    inp = bench.make_inputs(wl, 0)
    A = inp["a"]
    m, n, k, l, sw = wl["m"], wl["n"], wl["k"], wl["l"], wl["sweeps"]
    params, keep = L.make_params(k, l, sw, inp["J0"], trace_cap=8192, full_residual=True,
                                 resid_rows=inp["rows"], resid_cols=inp["cols"])
    res = ctx.solve(L.make_source("dense", a=torch.from_numpy(A).to(DEV)), params, l, m, n,
                    want_strips=True, trace_cap=8192, device=DEV)
    assert res.info.status == 0
    ref = O.cross_approximation(O.Dense(A), inp["J0"], k=k, sweeps=sw, delta=DELTA, rank_tol=GPU_TAU)
    ncmp, div = compare_traces(res.trace, ref.trace, DELTA)
    assert ncmp >= l
    if div is None:
        assert list(res.I) == ref.I and list(res.J) == ref.J
    check_nucleus(res.U, res.sigma, res.info.k_eff, A[np.ix_(res.I, res.J)], k)
    C, R = res.C.cpu().numpy(), res.R.cpu().numpy()
    full64 = O.full_residual(O.Dense(A), C.astype(np.float64), res.U, R.astype(np.float64))[0]
    assert res.info.full_rel_err == pytest.approx(full64, rel=2e-3)
    # the stored FP32 entries are exact in FP64, and sigma_k of the cross is
    # far above both truncation thresholds (1e-6 and the FP64 default
    # 1e-12), so this run is also the pure-FP64 error reference
    assert ref.sigma[k - 1] > 1e-4 * ref.sigma[0]
    err_ref = O.full_residual(O.Dense(A), ref.C, ref.U, ref.R)[0]
    assert error_ok(res.info.full_rel_err, err_ref)


def test_cancel_stops_a_running_job(ctx):
    """A long job cancelled right after submit ends well before it would have
    finished, and the context keeps working."""
    import time
    x, y = W.cauchy_points(95, 65536, 65536)
    xd, yd = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
    src = L.make_source("cauchy", x=xd, y=yd)
    J0 = W.draw_indices(96, 65536, 24)
    params, keep = L.make_params(16, 24, 40, J0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    full = ctx.solve(src, params, 24)
    t_full = time.perf_counter() - t0
    assert full.info.status == 0
    job = ctx.submit(src, params)
    t0 = time.perf_counter()
    L.lra_cross_cancel(ctx.ctx, job)
    t_cancel = time.perf_counter() - t0
    assert t_cancel < 0.5 * t_full, (t_cancel, t_full)
    again = ctx.solve(src, params, 24)
    assert again.info.status == 0
    np.testing.assert_array_equal(again.I, full.I)


def test_fixed_point_exit_keeps_the_whole_log(ctx):
    """A budget of 12 sweeps on a Cauchy matrix that reaches a fixed point
    after two or three: the device stops there, and its decision log, index
    sets, nucleus and sweep count are those of running every half-step (the
    oracle runs all 24)."""
    m, n, k, l = 3000, 4000, 12, 16
    x, y = W.cauchy_points(W.BASE_SEED + 900, m, n)
    src = L.make_source("cauchy", x=torch.from_numpy(x).to(DEV), y=torch.from_numpy(y).to(DEV))
    J0 = W.draw_indices(W.BASE_SEED + 901, n, l)
    res = gpu_solve(ctx, src, m, n, J0, k, l, 12)
    ref = O.cross_approximation(O.Cauchy(x, y, "fp32"), J0, k=k, sweeps=12, delta=DELTA, rank_tol=GPU_TAU)
    ncmp, div = compare_traces(res.trace, ref.trace, DELTA)
    assert div is None and ncmp == len(ref.trace)
    assert sum(1 for d in ref.trace if d[1] == O.STOP) == 24
    assert list(res.I) == ref.I and list(res.J) == ref.J
    assert res.info.sweeps_done == 12
    assert res.info.swaps_total == sum(1 for d in ref.trace if d[1] == O.SWAP)
    check_nucleus(res.U, res.sigma, res.info.k_eff, O.Cauchy(x, y, "fp32").block(res.I, res.J), k)


def test_fixed_point_exit_on_a_stored_matrix(ctx):
    """The same on a stored FP32 matrix (strips gathered between the
    half-steps, skipped once the job stops): a rank-10 matrix plus noise,
    budget of 10 sweeps, log, index sets and sweep count as the oracle's."""
    m, n, k, l = 2500, 1800, 10, 12
    A32 = W.factor_gaussian(W.BASE_SEED + 910, m, n, k, 1e-5)
    J0 = W.draw_indices(W.BASE_SEED + 911, n, l)
    res = gpu_solve(ctx, L.make_source("dense", a=torch.from_numpy(A32).to(DEV)), m, n, J0, k, l, 10)
    ref = O.cross_approximation(O.Dense(A32), J0, k=k, sweeps=10, delta=DELTA, rank_tol=GPU_TAU)
    ncmp, div = compare_traces(res.trace, ref.trace, DELTA)
    assert div is None and ncmp == len(ref.trace)
    assert sum(1 for d in ref.trace if d[1] == O.STOP) == 20
    assert list(res.I) == ref.I and list(res.J) == ref.J
    assert res.info.sweeps_done == 10
    # the returned strips are those of the final index sets
    np.testing.assert_array_equal(res.C, A32[:, res.J])
    np.testing.assert_array_equal(res.R, A32[res.I, :])
