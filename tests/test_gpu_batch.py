"""Batched C-A (one persistent launch over many far-field blocks of the
1/|x - y| kernel, Section 9) against the FP64 oracle's rank-adaptive rule:
l starts at 12 (1.5 x 8) and doubles (up to 96) while the cross has full
numerical rank at 1e-6, k <= 64, stop on the sampled estimate or after the
sweep budget."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import SubSource, check_nucleus, compare_traces, error_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1611_01391_gb300 as L  # noqa: E402
from paper_1611_01391_gb300.api import make_batch_params, solve_batch  # noqa: E402

L_INIT, L_MAX, K_MAX, SWEEPS, TOL, Q = 12, 96, 64, 2, 1e-6, 32


@pytest.fixture(scope="module")
def ctx():
    c = L.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def case():
    pts, blocks = W.octree_block_pairs(W.BASE_SEED + 4, npoints=1 << 17, leaf=512, n_pairs=40)
    jc, sr, sc = W.block_candidates(W.BASE_SEED + 5, blocks, L_MAX, Q)
    return pts, blocks, jc, sr, sc


def _run(ctx, pts, blocks, jc, sr, sc):
    d = torch.from_numpy(pts).cuda()
    src = L.make_source("invdist", x=d, y=d)
    p, keep = make_batch_params(L_INIT, L_MAX, K_MAX, SWEEPS, TOL, jc, sr, sc)
    return solve_batch(ctx, src, blocks, p, L_MAX)


def _nucleus(r, b):
    l = int(r.l[b])
    return r.I[b, :l], r.J[b, :l], r.U[b].ravel()[: l * l].reshape(l, l).astype(np.float64)


@pytest.fixture(scope="module")
def tree4096():
    """The 2^20-point octree (leaf <= 2048) of the batched workload, and a
    subset of its 4096 far-field blocks: the 12 largest and 24 drawn at
    random."""
    pts, blocks = W.octree_block_pairs(W.BASE_SEED + 4, npoints=1 << 20, leaf=2048, n_pairs=4096)
    side = np.maximum(blocks[:, 1], blocks[:, 3])
    big = np.argsort(-side, kind="stable")[:12]
    rest = np.setdiff1d(np.arange(len(blocks)), big)
    pick = np.concatenate([big, np.random.default_rng(5).choice(rest, 24, replace=False)])
    sel = blocks[pick]
    jc, sr, sc = W.block_candidates(W.BASE_SEED + 5, sel, L_MAX, Q)
    return pts, sel, jc, sr, sc


def _decision_parity(r, b, sub32, jc_b, sr_b, sc_b, A64):
    """Block b of a batched run against the oracle's rank-adaptive rule fed
    the same FP32 entries: decision logs agree up to the first unseparated
    decision; with no divergence, the same l, I, J, kept rank and nucleus;
    the error within 1.05x of that oracle's.  Returns True when the logs
    agree to the end."""
    trace = []
    oI, oJ, oU, ok, osig, ol, osw = O.cross_approximation_adaptive(
        sub32, jc_b, L_INIT, L_MAX, K_MAX, SWEEPS, TOL, sample_rows=sr_b, sample_cols=sc_b, trace=trace)
    dt, dv = r.block_trace(b)
    assert len(dt) < r.trace.shape[1], "device log truncated"
    ncmp, div = compare_traces([tuple(t) for t in dt], trace, 1e-2)
    assert ncmp >= min(L_INIT, sub32.m, sub32.n), (b, ncmp)
    I, J, U = _nucleus(r, b)
    if div is None:
        assert int(r.l[b]) == ol and list(I) == list(oI) and list(J) == list(oJ), b
        assert int(r.k_eff[b]) == ok, (b, r.k_eff[b], ok)
        # the recorded values are the oracle's |B| to double-float accuracy
        ov = np.array([d[4] for d in trace])
        np.testing.assert_allclose(dv, ov, rtol=1e-6)
    X32 = sub32.block(I, J)
    check_nucleus(U, r.sigma[b], int(r.k_eff[b]), X32, K_MAX, tau=TOL, sigma_rel=2.0 ** -23)
    err = np.linalg.norm(A64 - A64[:, J] @ U @ A64[I, :]) / np.linalg.norm(A64)
    oerr = np.linalg.norm(A64 - A64[:, oJ] @ oU @ A64[oI, :]) / np.linalg.norm(A64)
    assert error_ok(err, oerr), (b, err, oerr)
    return div is None


def test_batch_decision_logs_on_the_4096_block_tree(ctx, tree4096):
    """Blocks of the batched workload's own tree (sides up to 2048) through
    the persistent launch, each against the oracle fed the same FP32 entries
    of 1/|x - y| (reproduced bit for bit)."""
    pts, blocks, jc, sr, sc = tree4096
    d = torch.from_numpy(pts).cuda()
    src = L.make_source("invdist", x=d, y=d)
    p, keep = make_batch_params(L_INIT, L_MAX, K_MAX, SWEEPS, TOL, jc, sr, sc, trace_cap=8192)
    r = solve_batch(ctx, src, blocks, p, L_MAX)
    assert np.all(r.status == 0)
    s32 = O.InvDist(pts, pts, "fp32")
    s64 = O.InvDist(pts, pts, "fp64")
    full = 0
    for b, (r0, m, c0, n) in enumerate(blocks):
        A64 = SubSource(s64, r0, m, c0, n).block(np.arange(m), np.arange(n))
        full += _decision_parity(r, b, SubSource(s32, r0, m, c0, n), jc[b], sr[b], sc[b], A64)
    # most blocks agree to the last decision (the rest diverge only at a near-tie)
    assert full >= 0.8 * len(blocks), full


def test_batch_error_vs_oracle(ctx, case):
    """40 blocks of a 2^17-point tree: decision logs, index sets, kept ranks
    and nuclei against the oracle fed the same FP32 entries, errors within
    1.05x, and the device's Appendix F estimate against the FP64 one on the
    device's own factors."""
    pts, blocks, jc, sr, sc = case
    d = torch.from_numpy(pts).cuda()
    src = L.make_source("invdist", x=d, y=d)
    p, keep = make_batch_params(L_INIT, L_MAX, K_MAX, SWEEPS, TOL, jc, sr, sc, trace_cap=8192)
    r = solve_batch(ctx, src, blocks, p, L_MAX)
    assert np.all(r.status == 0)
    s64 = O.InvDist(pts, pts, "fp64")
    s32 = O.InvDist(pts, pts, "fp32")
    full = 0
    for b, (r0, m, c0, n) in enumerate(blocks):
        A64 = SubSource(s64, r0, m, c0, n).block(np.arange(m), np.arange(n))
        sub32 = SubSource(s32, r0, m, c0, n)
        full += _decision_parity(r, b, sub32, jc[b], sr[b], sc[b], A64)
        I, J, U = _nucleus(r, b)
        # the residual is ~1e-7 |M|, so FP32 rounding of M alone moves it by
        # percents: compare on the same FP32 entries
        est = O.sampled_residual(sub32, sub32.block(np.arange(m), J), U, sub32.block(I, np.arange(n)),
                                 sr[b], sc[b])["rel"]
        assert r.est_err[b] == pytest.approx(est, rel=1e-3, abs=1e-9)
    assert full >= 0.8 * len(blocks), full


def test_batch_subset_is_bit_identical(ctx, case):
    """Each block's result does not depend on which other blocks share the
    launch or which cluster picked it up."""
    pts, blocks, jc, sr, sc = case
    a = _run(ctx, pts, blocks, jc, sr, sc)
    sel = np.arange(0, len(blocks), 3)
    b = _run(ctx, pts, blocks[sel], jc[sel], sr[sel], sc[sel])
    for name in ("l", "k_eff", "I", "J", "U", "est_err"):
        np.testing.assert_array_equal(getattr(a, name)[sel], getattr(b, name))


def test_batch_rejects_invalid_blocks(ctx, case):
    pts, blocks, jc, sr, sc = case
    bad = blocks.copy()
    bad[0, 1] = 4096                     # side above 2048
    with pytest.raises(L.LraError) as e:
        _run(ctx, pts, bad, jc, sr, sc)
    assert e.value.code == L.LRA_EINVAL
    jbad = jc.copy()
    jbad[1, 1] = jbad[1, 0]              # repeated candidate column
    with pytest.raises(L.LraError):
        _run(ctx, pts, blocks, jbad, sr, sc)


def test_blocks_that_need_the_cluster_pass(ctx):
    """Blocks of 2048 x 2048 whose rank exceeds what one CTA's shared memory
    holds (l > 24 at that side) finish in the 4-CTA pass; small blocks in the
    same launch finish in the first.  Errors against the oracle's rule, and
    the same results when the large blocks run alone."""
    x = W.cloud_points(W.BASE_SEED + 70, 6144)
    d = torch.from_numpy(x).cuda()
    h = 0.6
    src = L.make_source("gauss", x=d, y=d, h=h)
    blocks = np.array([[0, 2048, 2048, 2048], [2048, 2048, 4096, 2048], [0, 300, 4096, 260],
                       [4096, 2048, 0, 2048], [100, 200, 5000, 190]], np.int64)
    jc, sr, sc = W.block_candidates(W.BASE_SEED + 71, blocks, L_MAX, Q)
    p, keep = make_batch_params(L_INIT, L_MAX, K_MAX, SWEEPS, TOL, jc, sr, sc, trace_cap=16384)
    r = solve_batch(ctx, src, blocks, p, L_MAX)
    assert np.all(r.status == 0)
    assert r.l[0] > 12 and r.l[1] > 12 and r.l[3] > 12     # went through a cluster pass
    s64 = O.Gauss(x, x, h, "fp64")
    for b, (r0, m, c0, n) in enumerate(blocks):
        A64 = SubSource(s64, r0, m, c0, n).block(np.arange(m), np.arange(n))
        # numpy's float32 exp is not CUDA's expf: the oracle takes the
        # device's own FP32 entries of the block (lra_gather_entries)
        rows = torch.arange(r0, r0 + m, dtype=torch.int32, device="cuda")
        cols = torch.arange(c0, c0 + n, dtype=torch.int32, device="cuda")
        ent = torch.empty((m, n), dtype=torch.float32, device="cuda")
        L.lra_gather_entries(src, rows, cols, ent)
        sub32 = O.Dense(ent.cpu().numpy())
        _decision_parity(r, b, sub32, jc[b], sr[b], sc[b], A64)
    sel = np.array([0, 3])
    p2, keep2 = make_batch_params(L_INIT, L_MAX, K_MAX, SWEEPS, TOL, jc[sel], sr[sel], sc[sel])
    r2 = solve_batch(ctx, src, blocks[sel], p2, L_MAX)
    for name in ("l", "k_eff", "I", "J", "U", "est_err"):
        np.testing.assert_array_equal(getattr(r, name)[sel], getattr(r2, name))


def test_tiny_and_degenerate_blocks(ctx):
    """Blocks smaller than the first cross (the cross is capped by the block),
    a 1 x 1 block, a single row, and no error sample."""
    pts = W.cloud_points(W.BASE_SEED + 72, 600)
    d = torch.from_numpy(pts).cuda()
    src = L.make_source("invdist", x=d, y=d)
    blocks = np.array([[0, 1, 300, 1], [10, 5, 400, 3], [20, 1, 500, 40], [100, 64, 200, 64],
                       [0, 7, 590, 9]], np.int64)
    jc, _, _ = W.block_candidates(W.BASE_SEED + 73, blocks, L_MAX, 1)
    p, keep = make_batch_params(L_INIT, L_MAX, K_MAX, SWEEPS, TOL, jc)
    r = solve_batch(ctx, src, blocks, p, L_MAX)
    assert np.all(r.status == 0)
    s64 = O.InvDist(pts, pts, "fp64")
    for b, (r0, m, c0, n) in enumerate(blocks):
        assert r.l[b] <= min(m, n)
        sub = SubSource(s64, r0, m, c0, n)
        A = sub.block(np.arange(m), np.arange(n))
        I, J, U = _nucleus(r, b)
        assert len(set(I.tolist())) == len(I) and I.max() < m and J.max() < n
        err = np.linalg.norm(A - A[:, J] @ U @ A[I, :]) / np.linalg.norm(A)
        oI, oJ, oU, ok, osig, ol, osw = O.cross_approximation_adaptive(sub, jc[b], L_INIT, L_MAX, K_MAX,
                                                                       SWEEPS, TOL)
        oerr = np.linalg.norm(A - A[:, oJ] @ oU @ A[oI, :]) / np.linalg.norm(A)
        assert error_ok(err, oerr), (b, err, oerr)
        assert r.l[b] == ol, (b, r.l[b], ol)


def test_launch_shapes_and_tuner_give_identical_results(ctx, tree4096, tmp_path):
    """Every launch shape (cluster chain, cut-over side, queue order) gives
    each block the same result bit for bit, U included; the tuner checks
    l, k_eff, I, J and the estimate on each of its 30 candidates itself,
    stores its choice in the cache and finds it there the second time."""
    pts, blocks, jc, sr, sc = tree4096
    d = torch.from_numpy(pts).cuda()
    src = L.make_source("invdist", x=d, y=d)
    p, keep = make_batch_params(L_INIT, L_MAX, K_MAX, SWEEPS, TOL, jc, sr, sc)
    ref = solve_batch(ctx, src, blocks, p, L_MAX)
    assert np.all(ref.status == 0)
    fields = ("status", "l", "k_eff", "swaps", "I", "J", "U", "sigma", "est_err")
    for mask, cut, order in ((15, 512, 1), (2 | 4 | 8, 0, 0), (1 | 8, 1024, 1), (8, 0, 1)):
        q, keep2 = make_batch_params(L_INIT, L_MAX, K_MAX, SWEEPS, TOL, jc, sr, sc)
        q.cluster_mask, q.cutover_side, q.order = mask, cut, order
        r = solve_batch(ctx, src, blocks, q, L_MAX)
        for name in fields:
            np.testing.assert_array_equal(getattr(r, name), getattr(ref, name), err_msg=f"{name} {mask} {cut} {order}")
    cache = tmp_path / "tuning.json"
    b64 = np.ascontiguousarray(blocks, np.int64)
    tuned, ms_def, ms_tuned = L.lra_cross_tune_batch(ctx.ctx, src, b64, p, cache)
    assert ms_def > 0 and 0 < ms_tuned <= ms_def
    r = solve_batch(ctx, src, blocks, tuned, L_MAX)
    for name in fields:
        np.testing.assert_array_equal(getattr(r, name), getattr(ref, name), err_msg=name)
    again, md2, mt2 = L.lra_cross_tune_batch(ctx.ctx, src, b64, p, cache)
    assert md2 == -1.0 and (again.cluster_mask, again.cutover_side, again.order) == \
        (tuned.cluster_mask, tuned.cutover_side, tuned.order)
    gpu = torch.cuda.get_device_properties(0).name
    hit = L.lra_batch_tuning_lookup(cache, gpu, src, b64, p)
    assert hit is not None and hit.cluster_mask == tuned.cluster_mask
