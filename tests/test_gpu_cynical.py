"""Cynical algorithms (Section 6.5) in the forms of Tests 3 and 4 of Section
12.2, through the C ABI, against the oracle fed the same FP32 entries: the
outer C-A loop's index sets, the generator, the nucleus and the error."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import GPU_TAU, check_nucleus, error_ok, separated

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1611_01391_gb300 as L  # noqa: E402

DELTA = 1e-2


@pytest.fixture(scope="module")
def ctx():
    c = L.Context(0)
    yield c
    c.close()


def _tb_ranrc(seed, n, r):
    """W = G1 G2 + 1e-10 G3 of Table tb_ranrc, stored in FP32."""
    rng = W.rng_for(seed)
    A = rng.standard_normal((n, r)) @ rng.standard_normal((r, n)) + 1e-10 * rng.standard_normal((n, n))
    return A.astype(np.float32)


def _check(ctx, A32, res, ref, r):
    I, J, U, K, Lq = res
    A64 = A32.astype(np.float64)
    outer_sep = ref.outer is None or all(separated(d, DELTA) for d in ref.outer.trace)
    if outer_sep:
        assert list(K) == ref.K and list(Lq) == ref.L
        if all(separated(d, DELTA) for d in ref.inner.trace):
            assert list(I) == ref.I and list(J) == ref.J
    check_nucleus(U, np.linalg.svd(A32[np.ix_(I, J)].astype(np.float64), compute_uv=False), r,
                  A32[np.ix_(I, J)], r)
    err = np.linalg.norm(A64 - A64[:, J] @ U @ A64[I, :]) / np.linalg.norm(A64)
    oerr = np.linalg.norm(A64 - A64[:, ref.J] @ ref.U @ A64[ref.I, :]) / np.linalg.norm(A64)
    assert error_ok(err, oerr), (err, oerr)
    return err


@pytest.mark.parametrize("n,r", [(1024, 8), (1024, 16), (2048, 24)])
def test_tests4_against_the_oracle(ctx, n, r):
    A32 = _tb_ranrc(1200 + n + r, n, r)
    src = L.make_source("dense", a=torch.from_numpy(A32).cuda())
    L0 = W.draw_indices(1300 + r, n, 4 * r)
    res = L.lra_cross_cynical(ctx.ctx, src, r, L0, outer_loops=1, inner_sweeps=2, rank_tol=GPU_TAU)
    ref = O.ca_cynical(O.Dense(A32), L0, r, outer_loops=1, inner_sweeps=2, rank_tol=GPU_TAU)
    err = _check(ctx, A32, res, ref, r)
    assert err < 1e-6


@pytest.mark.parametrize("n,r", [(1024, 8), (2048, 16)])
def test_tests3_against_the_oracle(ctx, n, r):
    A32 = _tb_ranrc(1400 + n + r, n, r)
    src = L.make_source("dense", a=torch.from_numpy(A32).cuda())
    K0, L0 = W.draw_indices(1500 + r, n, 4 * r), W.draw_indices(1600 + r, n, 4 * r)
    res = L.lra_cross_cynical(ctx.ctx, src, r, L0, K=K0, outer_loops=0, inner_sweeps=2, rank_tol=GPU_TAU)
    ref = O.cynical(O.Dense(A32), K0, L0, r, inner_sweeps=2, rank_tol=GPU_TAU)
    assert list(res[3]) == list(K0) and list(res[4]) == list(L0)
    _check(ctx, A32, res, ref, r)


def test_cynical_on_a_generator(ctx):
    """Tests 4 on the generated Cauchy matrix (no stored matrix at all)."""
    x, y = W.cauchy_points(1700, 20000, 30000)
    src = L.make_source("cauchy", x=torch.from_numpy(x).cuda(), y=torch.from_numpy(y).cuda())
    L0 = W.draw_indices(1701, 30000, 48)
    I, J, U, K, Lq = L.lra_cross_cynical(ctx.ctx, src, 12, L0, outer_loops=1, inner_sweeps=2, rank_tol=GPU_TAU)
    ref = O.ca_cynical(O.Cauchy(x, y, "fp32"), L0, 12, outer_loops=1, inner_sweeps=2, rank_tol=GPU_TAU)
    if all(separated(d, DELTA) for d in ref.outer.trace):
        assert list(K) == ref.K and list(Lq) == ref.L
    assert set(I) <= set(K) and set(J) <= set(Lq)
    rows, cols = W.draw_indices(1702, 20000, 400, sort=True), W.draw_indices(1703, 30000, 400, sort=True)
    s64 = O.Cauchy(x, y, "fp64")
    A = s64.block(rows, cols)
    err = np.linalg.norm(A - s64.block(rows, J) @ U @ s64.block(I, cols)) / np.linalg.norm(A)
    oerr = np.linalg.norm(A - s64.block(rows, ref.J) @ ref.U @ s64.block(ref.I, cols)) / np.linalg.norm(A)
    assert error_ok(err, oerr), (err, oerr)


def test_cynical_rejects_bad_arguments(ctx):
    A32 = _tb_ranrc(1800, 300, 4)
    src = L.make_source("dense", a=torch.from_numpy(A32).cuda())
    for kw in (dict(r=5, L=list(range(4))),                       # r > q
               dict(r=4, L=list(range(97))),                      # q > 96
               dict(r=4, L=[1, 2, 3, 3, 5, 6, 7, 8]),             # repeated column
               dict(r=4, L=list(range(8)), K=None, outer_loops=0)):  # Tests 3 without K
        with pytest.raises(L.LraError) as e:
            L.lra_cross_cynical(ctx.ctx, src, **kw)
        assert e.value.code == L.LRA_EINVAL
