"""Pre-processing with abridged Hadamard multipliers (Section 8.1, family (i))
and recovery of the LRA of M (Section 6.6) through the C ABI, against the
oracle: the materialised H_{m,d} M H_{n,d}, the entry-by-entry M_bar and the
recovered factors bit for bit; C-A on M_bar decision by decision; the
recovered error against the oracle's; Appendix E's delta matrix."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import GPU_TAU, compare_traces, error_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1611_01391_gb300 as L  # noqa: E402

DEV = "cuda:0"
DELTA = 1e-2


@pytest.fixture(scope="module")
def ctx():
    c = L.Context(0)
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


class _Pre:
    """Device tensors of one pre-processed source (kept alive together)."""

    def __init__(self, A32, d, mult, lda_pad=0):
        m, n = A32.shape
        self.m, self.n, self.d = m, n, d
        buf = torch.zeros((m, n + lda_pad), dtype=torch.float32, device=DEV)
        buf[:, :n] = _dev(A32)
        self.a = buf[:, :n]
        self.mult = [_dev(v) for v in mult]
        self.src = L.make_source("preprocessed", a=self.a, d=d, perm_rows=self.mult[0], sign_rows=self.mult[1],
                                 perm_cols=self.mult[2], sign_cols=self.mult[3])
        self.oracle = O.Preprocessed(O.Dense(A32), d, *[np.asarray(v) for v in mult], precision="fp32")

    def materialized(self, ldg_pad=0):
        G = torch.empty((self.m, self.n + ldg_pad), dtype=torch.float32, device=DEV)[:, :self.n]
        L.lra_preprocess_materialize(self.src, G)
        torch.cuda.synchronize()
        self.G = G
        self.src_mat = L.make_source("preprocessed", a=G, d=self.d, perm_rows=self.mult[0],
                                     sign_rows=self.mult[1], perm_cols=self.mult[2], sign_cols=self.mult[3],
                                     materialized=True)
        return G


def _identity(m, n):
    return (np.arange(m, dtype=np.int32), np.ones(m, np.float32), np.arange(n, dtype=np.int32),
            np.ones(n, np.float32))


def _gather(src, rows, cols):
    out = torch.empty((len(rows), len(cols)), dtype=torch.float32, device=DEV)
    L.lra_gather_entries(src, _dev(np.asarray(rows, np.int32)), _dev(np.asarray(cols, np.int32)), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("m,n,d,pad", [(96, 80, 1, 0), (200, 136, 3, 5), (64, 96, 5, 0), (1024, 1056, 2, 4), (1000, 1056, 3, 3),
                                       (3008, 2080, 4, 0), (512, 160, 5, 1), (48, 40, 0, 0), (4096, 32, 5, 0)])
def test_materialized_transform_is_bit_exact(m, n, d, pad):
    """G = H_{m,d} M H_{n,d}: every entry (small cases) or every entry of a
    row sample (large ones) equal to the oracle's butterfly sums in FP32."""
    A32 = W.factor_gaussian(4000 + m + d, m, n, 6, 1e-3)
    pre = _Pre(A32, d, _identity(m, n), lda_pad=pad)
    G = pre.materialized(ldg_pad=pad).cpu().numpy()
    rows = np.arange(m) if m * n * (4 ** d) <= 30_000_000 else W.draw_indices(4100 + m, m, 48, sort=True)
    ref = pre.oracle.block(rows, np.arange(n)).astype(np.float32)
    np.testing.assert_array_equal(G[rows], ref)


@pytest.mark.parametrize("m,n,d", [(96, 80, 1), (320, 272, 3), (128, 64, 6), (2048, 1536, 2)])
def test_entries_on_the_fly_equal_the_oracle_and_the_materialized_source(m, n, d):
    A32 = W.factor_gaussian(4200 + m, m, n, 5, 1e-3)
    pre = _Pre(A32, d, W.hadamard_multipliers(4300 + m, m, n))
    rows = W.draw_indices(4400 + m, m, min(m, 64))
    cols = W.draw_indices(4500 + n, n, min(n, 80))
    got = _gather(pre.src, rows, cols)
    np.testing.assert_array_equal(got, pre.oracle.block(rows, cols).astype(np.float32))
    if d <= 5:
        pre.materialized()
        np.testing.assert_array_equal(_gather(pre.src_mat, rows, cols), got)


def _solve(ctx, src, m, n, J0, k, l, sweeps):
    params, keep = L.make_params(k, l, sweeps, J0, delta=DELTA, rank_tol=GPU_TAU, trace_cap=8192)
    res, A, B = L.solve_preprocessed(ctx, src, params, l, m, n, trace_cap=8192, device=DEV)
    assert res.info.status == 0, L.lra_status_str(res.info.status)
    torch.cuda.synchronize()
    return res, A.cpu().numpy(), B.cpu().numpy()


@pytest.mark.parametrize("m,n,d,k,l", [(2048, 1536, 3, 12, 16), (1000, 1200, 2, 8, 8), (4096, 1024, 1, 20, 24)])
def test_ca_on_preprocessed_source_and_recovery(ctx, m, n, d, k, l):
    A32 = W.factor_gaussian(4600 + m + d, m, n, k, 1e-4)
    pre = _Pre(A32, d, W.hadamard_multipliers(4700 + m, m, n))
    J0 = W.draw_indices(4800 + n, n, l)
    res, A, B = _solve(ctx, pre.src, m, n, J0, k, l, 3)
    ref = O.cross_approximation(pre.oracle, J0, k=k, sweeps=3, delta=DELTA, rank_tol=GPU_TAU)
    ncmp, div = compare_traces(res.trace, ref.trace, DELTA)
    assert ncmp >= l
    Cbar, Rbar = res.C.cpu().numpy(), res.R.cpu().numpy()
    # the strips are entries of M_bar: bit for bit
    np.testing.assert_array_equal(Cbar, pre.oracle.block(np.arange(m), res.J).astype(np.float32))
    np.testing.assert_array_equal(Rbar, pre.oracle.block(res.I, np.arange(n)).astype(np.float32))
    if div is None:
        assert list(res.I) == ref.I and list(res.J) == ref.J
    # recovery from the device's own strips: bit for bit
    Ar, Br = O.recover_lra(pre.oracle, Cbar, Rbar)
    np.testing.assert_array_equal(A, Ar.astype(np.float32))
    np.testing.assert_array_equal(B, Br.astype(np.float32))
    # the error of the recovered LRA of M; Section 6.6: it is the error on
    # M_bar over 2^d (up to the FP32 rounding of A and B)
    M64 = A32.astype(np.float64)
    err = np.linalg.norm(M64 - A.astype(np.float64) @ res.U @ B.astype(np.float64))
    Mbar = pre.oracle.block(np.arange(m), np.arange(n))
    err_bar = np.linalg.norm(Mbar - Cbar.astype(np.float64) @ res.U @ Rbar.astype(np.float64))
    assert err == pytest.approx(err_bar / (1 << d), rel=1e-2)
    pre64 = O.Preprocessed(O.Dense(M64), d, *[np.asarray(v) for v in W.hadamard_multipliers(4700 + m, m, n)])
    r64 = O.cross_approximation(pre64, J0, k=k, sweeps=3, delta=DELTA)
    A64, B64 = O.recover_lra(pre64, r64.C, r64.R)
    err64 = np.linalg.norm(M64 - A64 @ r64.U @ B64)
    assert error_ok(err / np.linalg.norm(M64), err64 / np.linalg.norm(M64)), (err, err64)


def test_materialized_source_gives_the_same_solve(ctx):
    """The two forms of M_bar have the same entries, so the whole solve (log,
    index sets, nucleus, recovered factors) is bit-identical."""
    m, n, d, k, l = 3072, 2048, 4, 10, 12
    A32 = W.factor_gaussian(4900, m, n, k, 1e-4)
    pre = _Pre(A32, d, W.hadamard_multipliers(4901, m, n))
    pre.materialized()
    J0 = W.draw_indices(4902, n, l)
    r1, A1, B1 = _solve(ctx, pre.src, m, n, J0, k, l, 3)
    r2, A2, B2 = _solve(ctx, pre.src_mat, m, n, J0, k, l, 3)
    np.testing.assert_array_equal(r1.trace, r2.trace)
    assert list(r1.I) == list(r2.I) and list(r1.J) == list(r2.J)
    np.testing.assert_array_equal(r1.U, r2.U)
    np.testing.assert_array_equal(A1, A2)
    np.testing.assert_array_equal(B1, B2)


def test_laplacian_preprocessed_against_the_oracle(ctx):
    """Class (i) of the paper's inputs (single-layer Laplacian, n = 1024,
    r = 15) after abridged Hadamard pre-processing: error within the bar of
    the FP64 oracle run on the same multipliers and initial columns."""
    n, d, k = 1024, 3, 15
    M64 = W.laplacian_single_layer(n)
    M32 = M64.astype(np.float32)
    mult = W.hadamard_multipliers(5000, n, n)
    pre = _Pre(M32, d, mult)
    J0 = W.draw_indices(5001, n, k)
    res, A, B = _solve(ctx, pre.src, n, n, J0, k, k, 3)
    err = np.linalg.norm(M64 - A.astype(np.float64) @ res.U @ B.astype(np.float64)) / np.linalg.norm(M64)
    pre64 = O.Preprocessed(O.Dense(M64), d, *[np.asarray(v) for v in mult])
    r64 = O.cross_approximation(pre64, J0, k=k, sweeps=3, delta=DELTA)
    A64, B64 = O.recover_lra(pre64, r64.C, r64.R)
    err64 = np.linalg.norm(M64 - A64 @ r64.U @ B64) / np.linalg.norm(M64)
    assert error_ok(err, err64), (err, err64)
    assert err < 1e-2


@pytest.mark.parametrize("n,d,materialize", [(64, 6, False), (32, 5, True), (256, 8, False)])
def test_full_hadamard_preprocessing_finds_the_delta_matrix(ctx, n, d, materialize):
    """Appendix E's single nonzero entry: after pre-processing with
    d = log2 n every entry of M_bar is +-1, and the recovered rank-1 LRA is
    exact from any initial column."""
    A32 = W.delta_matrix(n, n, 37 % n, 11).astype(np.float32)
    for seed in range(3):
        pre = _Pre(A32, d, W.hadamard_multipliers(5100 + seed, n, n))
        src = pre.src
        if materialize:
            pre.materialized()
            src = pre.src_mat
        J0 = W.draw_indices(5200 + seed, n, 1)
        res, A, B = _solve(ctx, src, n, n, J0, 1, 1, 1)
        E = A32.astype(np.float64) - A.astype(np.float64) @ res.U @ B.astype(np.float64)
        assert np.abs(E).max() <= 1e-6


def test_preprocessing_rejects_bad_arguments(ctx):
    m, n = 96, 80
    A32 = W.factor_gaussian(5300, m, n, 4, 1e-3)
    pre = _Pre(A32, 3, W.hadamard_multipliers(5301, m, n))
    G = torch.empty((m, n), dtype=torch.float32, device=DEV)
    cases = []
    for kw in (dict(d=11), dict(d=5), dict(d=-1)):   # 2^5 does not divide 80
        cases.append(L.make_source("preprocessed", a=pre.a, perm_rows=pre.mult[0], sign_rows=pre.mult[1],
                                   perm_cols=pre.mult[2], sign_cols=pre.mult[3], **kw))
    nullp = L.make_source("preprocessed", a=pre.a, d=3, perm_rows=pre.mult[0], sign_rows=pre.mult[1],
                          perm_cols=pre.mult[2], sign_cols=pre.mult[3])
    nullp.pre_perm_cols = None
    cases.append(nullp)
    for src in cases:
        with pytest.raises(L.LraError) as e:
            L.lra_preprocess_materialize(src, G)
        assert e.value.code == L.LRA_EINVAL
        with pytest.raises(L.LraError) as e:
            _gather(src, [0], [0])
        assert e.value.code == L.LRA_EINVAL
    # materialise: depth above 5, G overlapping M, ldg < n, a materialised source
    A64 = np.zeros((128, 128), np.float32)
    deep = _Pre(A64, 6, W.hadamard_multipliers(5302, 128, 128))
    with pytest.raises(L.LraError):
        L.lra_preprocess_materialize(deep.src, torch.empty((128, 128), dtype=torch.float32, device=DEV))
    with pytest.raises(L.LraError):
        L.lra_preprocess_materialize(pre.src, pre.a)
    with pytest.raises(L.LraError):
        L.lra_preprocess_materialize(pre.src, torch.empty((m * n,), dtype=torch.float32, device=DEV)
                                     .as_strided((m, n), (n - 1, 1)))
    pre.materialized()
    with pytest.raises(L.LraError):
        L.lra_preprocess_materialize(pre.src_mat, G)
    # recovery on a source of another kind
    dense = L.make_source("dense", a=pre.a.contiguous())
    C = torch.zeros((m, 4), dtype=torch.float32, device=DEV)
    R = torch.zeros((4, n), dtype=torch.float32, device=DEV)
    with pytest.raises(L.LraError) as e:
        L.lra_preprocessed_recover(dense, C, R, C.clone(), R.clone())
    assert e.value.code == L.LRA_EINVAL
