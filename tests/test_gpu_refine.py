"""Refinement of a C-A CUR by leverage scores (Section 7.2, Algorithm 7.1,
Appendix C Algorithm C.1) through the C ABI, against the oracle fed the same
FP32 entries and the same uniform draws: the column and row scores element
by element, the sampled indices and their scales wherever the draw is not
within rounding of a boundary, the nucleus, and the error."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import GPU_TAU, U_DD, error_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1611_01391_gb300 as L  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = L.Context(0)
    yield c
    c.close()


def _separated_draws(p, u, tol=1e-9):
    """Draws whose uniform is farther than tol from every boundary of the
    cumulative scores (there both sides must pick the same index)."""
    cdf = np.cumsum(p)
    out = []
    for t, ut in enumerate(u):
        i = min(int(np.searchsorted(cdf, ut, side="right")), len(p) - 1)
        lo = cdf[i - 1] if i > 0 else 0.0
        out.append(ut - lo > tol and cdf[i] - ut > tol)
    return np.array(out)


def _refine_case(ctx, src, src32, src64, m, n, k, l, l_new, seed, rows, cols):
    J0 = W.draw_indices(seed, n, l)
    p, keep = L.make_params(k, l, 3, J0)
    ca = ctx.solve(src, p, l)
    assert ca.info.status == 0
    r = ca.info.k_eff
    rng = W.rng_for(seed + 1)
    uc, ur = rng.random(l_new), rng.random(l_new)
    dev = L.lra_cross_refine(ctx.ctx, src, ca.I, ca.J, r, l_new, uc, ur, rank_tol=GPU_TAU,
                             resid_rows=rows, resid_cols=cols, scores=True)
    assert dev["k_eff"] == r
    X32 = src32.block(ca.I, ca.J)
    Ur, kr, sx = O.nucleus(X32, r, GPU_TAU)
    assert kr == r
    ref = O.refine_by_leverage(src32, list(ca.I), list(ca.J), Ur, r, l_new, l_new, uc, ur, rank_tol=GPU_TAU)
    # scores: the subspaces come from the double-float SVD of the cross
    # (about 2^-48 kappa_r relative) and FP64 products
    kappa = sx[0] / sx[r - 1]
    tol = 64 * l * U_DD * kappa
    np.testing.assert_allclose(dev["p_cols"], ref.p_cols, rtol=0, atol=tol * ref.p_cols.max())
    np.testing.assert_allclose(dev["p_rows"], ref.p_rows, rtol=0, atol=tol * ref.p_rows.max())
    # sampled indices: the same wherever the draw is separated from a boundary
    sc = _separated_draws(ref.p_cols, uc)
    sr = _separated_draws(ref.p_rows, ur)
    assert sc.mean() > 0.9 and sr.mean() > 0.9
    np.testing.assert_array_equal(dev["cols"][sc], ref.cols[sc])
    np.testing.assert_array_equal(dev["rows"][sr], ref.rows[sr])
    if sc.all() and sr.all():
        np.testing.assert_allclose(dev["d"], ref.d, rtol=tol)
        np.testing.assert_allclose(dev["dbar"], ref.dbar, rtol=tol)
        # the nucleus of the same scaled generator, element by element
        Mk = ref.dbar[:, None] * src32.block(ref.rows, ref.cols) * ref.d[None, :]
        s = np.linalg.svd(Mk, compute_uv=False)
        bound = 64 * l_new * U_DD * s[0] / s[r - 1]
        err_u = np.abs(dev["U"] - ref.U).max() / np.abs(ref.U).max()
        assert err_u <= bound, (err_u, bound)
    # the error of the refined CUR against the FP64 entries, on the sample
    A = src64.block(rows, cols)

    def err(cl, U, rw):
        return np.linalg.norm(A - src64.block(rows, cl) @ U @ src64.block(rw, cols)) / np.linalg.norm(A)

    e_dev = err(dev["cols"], dev["U"], dev["rows"])
    e_ref = err(ref.cols, ref.U, ref.rows)
    assert error_ok(e_dev, e_ref), (e_dev, e_ref)
    # the device's Appendix F estimate of its refined CUR, on the FP32 entries
    est = O.sampled_residual(src32, src32.block(np.arange(m), dev["cols"]), dev["U"],
                             src32.block(dev["rows"], np.arange(n)), rows, cols)["rel"]
    assert dev["est_rel_err"] == pytest.approx(est, rel=1e-4)
    return e_dev, err(ca.J, ca.U, ca.I)


def test_refine_dense_rank_plus_noise(ctx):
    m, n = 3000, 2600
    A = W.factor_gaussian(2001, m, n, 10, 1e-4)
    src = L.make_source("dense", a=torch.from_numpy(A).cuda())
    rows, cols = W.draw_indices(2002, m, 400, sort=True), W.draw_indices(2003, n, 400, sort=True)
    s32 = O.Dense(A)
    e_ref, e_ca = _refine_case(ctx, src, s32, O.Dense(A.astype(np.float64)), m, n, 10, 16, 48, 2004, rows, cols)
    assert e_ref < 1e-3


def test_refine_generated_cauchy(ctx):
    m, n = 20000, 15000
    x, y = W.cauchy_points(2005, m, n)
    src = L.make_source("cauchy", x=torch.from_numpy(x).cuda(), y=torch.from_numpy(y).cuda())
    rows, cols = W.draw_indices(2006, m, 500, sort=True), W.draw_indices(2007, n, 500, sort=True)
    _refine_case(ctx, src, O.Cauchy(x, y, "fp32"), O.Cauchy(x, y, "fp64"), m, n, 16, 24, 48, 2008, rows, cols)


def test_refine_rejects_bad_arguments(ctx):
    A = W.factor_gaussian(2009, 300, 200, 4, 1e-3)
    src = L.make_source("dense", a=torch.from_numpy(A).cuda())
    I, J = np.arange(8), np.arange(8)
    u = np.full(16, 0.5)
    for kw in (dict(I=[0, 0, 1, 2, 3, 4, 5, 6]), dict(l_new=97, uc=np.full(97, 0.5), ur=np.full(97, 0.5)),
               dict(uc=np.full(16, 1.0)), dict(r=9)):
        args = dict(I=I, J=J, r=4, l_new=16, uc=u, ur=u)
        args.update(kw)
        with pytest.raises(L.LraError) as e:
            L.lra_cross_refine(ctx.ctx, src, args["I"], args["J"], args["r"], args["l_new"], args["uc"], args["ur"])
        assert e.value.code == L.LRA_EINVAL


def test_refine_with_repeated_draws(ctx):
    """Exactly(l) draws with replacement: repeated columns and rows make the
    sampled generator exactly rank-deficient (n = 1024, r = 16, l = 24,
    64 draws, 3 repeated columns, 4 repeated rows); the trailing columns of
    its pivoted QR are then zero up to rounding, which must not break the
    nucleus (a reflector scalar overflowed here before)."""
    n, r, lc, ln = 1024, 16, 24, 64
    rng = W.rng_for(W.BASE_SEED + 12000)
    rng.standard_normal((n, r)), rng.standard_normal((r, n)), rng.standard_normal((n, n))
    B64 = rng.standard_normal((n, r)) @ rng.standard_normal((r, n)) + 1e-4 * rng.standard_normal((n, n))
    B32 = B64.astype(np.float32)
    src = L.make_source("dense", a=torch.from_numpy(B32).cuda())
    p, keep = L.make_params(r, lc, 3, W.draw_indices(W.BASE_SEED + 12500, n, lc))
    ca = ctx.solve(src, p, lc)
    assert ca.info.status == 0 and ca.info.k_eff == r
    u = W.rng_for(W.BASE_SEED + 12600)
    uc, ur = u.random(ln), u.random(ln)
    dev = L.lra_cross_refine(ctx.ctx, src, ca.I, ca.J, r, ln, uc, ur, rank_tol=GPU_TAU)
    assert dev["k_eff"] == r
    s32 = O.Dense(B32)
    Ur, kr, _ = O.nucleus(s32.block(ca.I, ca.J), r, GPU_TAU)
    ref = O.refine_by_leverage(s32, list(ca.I), list(ca.J), Ur, r, ln, ln, uc, ur, rank_tol=GPU_TAU)
    B = B32.astype(np.float64)

    def err(cl, U, rw):
        return np.linalg.norm(B - B[:, cl] @ U @ B[rw, :]) / np.linalg.norm(B)

    assert error_ok(err(dev["cols"], dev["U"], dev["rows"]), err(ref.cols, ref.U, ref.rows))
