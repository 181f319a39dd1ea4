"""Boundary features through the C ABI: resume from a checkpoint (init_I),
the seeded initial column set, the tolerance stop against the oracle, entry
access (lra_gather_entries), and fetch / submit / poll from two threads."""
import threading
import time

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import GPU_TAU, compare_traces

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


def _cauchy(seed, m, n):
    x, y = W.cauchy_points(seed, m, n)
    xd, yd = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
    return x, y, (xd, yd), L.make_source("cauchy", x=xd, y=yd)


@pytest.mark.parametrize("cut", [1, 3])
def test_resume_from_checkpoint_is_bit_identical(ctx, cut):
    """A solve checkpointed after `cut` sweeps as (I, J) and resubmitted with
    init_I = I, init_J = J for the remaining sweeps returns the I, J, U and
    estimate of the uninterrupted solve, bit for bit."""
    x, y, keep, src = _cauchy(W.BASE_SEED + 60, 30000, 25000)
    J0 = W.draw_indices(W.BASE_SEED + 61, 25000, 24)
    rows = W.draw_indices(W.BASE_SEED + 62, 30000, 500, sort=True)
    cols = W.draw_indices(W.BASE_SEED + 63, 25000, 500, sort=True)
    total = 4
    p, k1 = L.make_params(16, 24, total, J0, resid_rows=rows, resid_cols=cols, trace_cap=4096)
    whole = ctx.solve(src, p, 24, trace_cap=4096)
    p, k2 = L.make_params(16, 24, cut, J0, resid_rows=rows, resid_cols=cols)
    first = ctx.solve(src, p, 24)
    p, k3 = L.make_params(16, 24, total - cut, first.J, init_I=first.I, resid_rows=rows, resid_cols=cols,
                          trace_cap=4096)
    rest = ctx.solve(src, p, 24, trace_cap=4096)
    for r in (whole, first, rest):
        assert r.info.status == 0
    assert rest.info.sweeps_done == total - cut
    np.testing.assert_array_equal(rest.I, whole.I)
    np.testing.assert_array_equal(rest.J, whole.J)
    np.testing.assert_array_equal(rest.U, whole.U)
    assert rest.info.est_rel_err == whole.info.est_rel_err
    # the resumed decision log is the uninterrupted one's tail, shifted by 2 cut half-steps
    tail = [tuple(t[1:]) for t in whole.trace if t[0] >= 2 * cut]
    assert [tuple(t[1:]) for t in rest.trace] == tail
    np.testing.assert_array_equal(rest.trace_val, whole.trace_val[len(whole.trace) - len(tail):])
    # and the oracle's resumed run agrees with the device's resumed run
    ref = O.cross_approximation(O.Cauchy(x, y, "fp32"), first.J, k=16, sweeps=total - cut, delta=DELTA,
                                rank_tol=GPU_TAU, I0=first.I)
    ncmp, div = compare_traces(rest.trace, ref.trace, DELTA)
    assert ncmp >= 2
    if div is None:
        assert list(rest.I) == ref.I and list(rest.J) == ref.J


def test_seeded_initial_columns(ctx):
    """init_J = NULL: the library draws J0 from the seed exactly as the
    oracle's SplitMix64 + Floyd sampling does (same result as passing the
    oracle's draw)."""
    x, y, keep, src = _cauchy(W.BASE_SEED + 64, 9000, 11000)
    seed = 0xC0FFEE
    p, k1 = L.make_params(16, 24, 2, None, seed=seed)
    a = ctx.solve(src, p, 24)
    p, k2 = L.make_params(16, 24, 2, O.draw_columns(seed, 11000, 24))
    b = ctx.solve(src, p, 24)
    assert a.info.status == 0 and b.info.status == 0
    np.testing.assert_array_equal(a.I, b.I)
    np.testing.assert_array_equal(a.J, b.J)
    np.testing.assert_array_equal(a.U, b.U)


def test_resume_and_seed_validation(ctx):
    x, y, keep, src = _cauchy(W.BASE_SEED + 65, 500, 400)
    J0 = W.draw_indices(1, 400, 8)
    for bad_I in ([0, 1, 2, 3, 4, 5, 6, 6], [0, 1, 2, 3, 4, 5, 6, 500]):
        p, k = L.make_params(8, 8, 1, J0, init_I=bad_I)
        with pytest.raises(L.LraError) as e:
            ctx.submit(src, p)
        assert e.value.code == L.LRA_EINVAL


def test_tolerance_stop_matches_the_oracle(ctx):
    """Step 6 of the C-A iterations: the device stops after the first sweep
    whose Appendix F estimate is <= tol, at the same sweep and with the same
    index sets as the oracle fed the same FP32 entries.  tol is placed
    between two consecutive per-sweep estimates of the oracle, far from both,
    so the device's estimate (equal to the oracle's within 1e-4) decides the
    same way."""
    m, n = 6000, 7000
    x, y, keep, src = _cauchy(W.BASE_SEED + 66, m, n)
    J0 = W.draw_indices(W.BASE_SEED + 67, n, 24)
    rows = W.draw_indices(W.BASE_SEED + 68, m, 600, sort=True)
    cols = W.draw_indices(W.BASE_SEED + 69, n, 600, sort=True)
    s32 = O.Cauchy(x, y, "fp32")
    full = O.cross_approximation(s32, J0, k=16, sweeps=6, delta=DELTA, rank_tol=GPU_TAU, keep_trace=False)
    ests = []
    for I, J in full.history:
        U, _, _ = O.nucleus(s32.block(I, J), 16, GPU_TAU)
        ests.append(O.sampled_residual(s32, O.columns(s32, J), U, O.rows(s32, I), rows, cols)["rel"])
    # the first sweep where the estimate drops by > 2x: stop right there
    stop_at = next((s for s in range(1, len(ests)) if ests[s] < 0.5 * min(ests[:s])), None)
    if stop_at is None:
        tols = [ests[0] * 2.0]
        expect = [1]
    else:
        tols = [float(np.sqrt(ests[stop_at] * min(ests[:stop_at]))), ests[0] * 2.0, min(ests) * 0.1]
        expect = [stop_at + 1, 1, 6]
    for tol, want in zip(tols, expect):
        p, kp = L.make_params(16, 24, 6, J0, resid_rows=rows, resid_cols=cols, tol=tol, trace_cap=8192)
        res = ctx.solve(src, p, 24, trace_cap=8192)
        assert res.info.status == 0
        ref = O.cross_approximation(s32, J0, k=16, sweeps=6, delta=DELTA, rank_tol=GPU_TAU, tol=tol,
                                    sample_rows=rows, sample_cols=cols)
        assert ref.sweeps_done == want, (tol, ests)
        assert res.info.sweeps_done == want, (tol, ests, res.info.sweeps_done)
        ncmp, div = compare_traces(res.trace, ref.trace, DELTA)
        if div is None:
            assert list(res.I) == ref.I and list(res.J) == ref.J


@pytest.mark.parametrize("kind", ["dense32", "dense64", "cauchy", "invdist", "gauss"])
def test_gather_entries_equal_the_strips(ctx, kind):
    """Entry access returns the same FP32 values as the solve's strips C and R
    (bit for bit), and NaN for an index outside M."""
    m, n, l = 700, 650, 9
    J0 = W.draw_indices(11, n, l)
    if kind.startswith("dense"):
        A = W.lowrank_svd(12, m, n, r=5, noise_std=1e-3)
        A = A.astype(np.float32) if kind == "dense32" else A
        keep = torch.from_numpy(A).to(DEV)
        src = L.make_source("dense", a=keep)
    elif kind == "cauchy":
        x, y, keep, src = _cauchy(13, m, n)
    else:
        x = torch.from_numpy(W.cloud_points(14, m)).to(DEV)
        y = torch.from_numpy(W.cloud_points(15, n, lo=2.0, hi=3.0)).to(DEV)
        keep = (x, y)
        src = L.make_source(kind, x=x, y=y, h=0.7)
    p, kp = L.make_params(l, l, 2, J0)
    res = ctx.solve(src, p, l, m, n, want_strips=True, device=DEV)
    assert res.info.status == 0
    rows = torch.arange(m, dtype=torch.int32, device=DEV)
    cols = torch.from_numpy(res.J.astype(np.int32)).to(DEV)
    out = torch.empty((m, l), dtype=torch.float32, device=DEV)
    L.lra_gather_entries(src, rows, cols, out)
    torch.cuda.synchronize()
    assert torch.equal(out, res.C)
    rows = torch.from_numpy(res.I.astype(np.int32)).to(DEV)
    cols = torch.arange(n, dtype=torch.int32, device=DEV)
    out = torch.empty((l, n), dtype=torch.float32, device=DEV)
    L.lra_gather_entries(src, rows, cols, out)
    torch.cuda.synchronize()
    assert torch.equal(out, res.R)
    rows = torch.tensor([0, -1, m], dtype=torch.int32, device=DEV)
    cols = torch.tensor([n - 1, 0], dtype=torch.int32, device=DEV)
    out = torch.zeros((3, 2), dtype=torch.float32, device=DEV)
    L.lra_gather_entries(src, rows, cols, out)
    v = out.cpu().numpy()
    assert np.isfinite(v[0]).all() and np.isnan(v[1:]).all()


def test_fetch_of_a_long_job_does_not_block_other_threads():
    """One thread waits in fetch_cur for a long solve; meanwhile another
    thread submits a short solve and polls it to completion.  The short
    solve must finish while the long one is still being waited for."""
    x, y, keep, src = _cauchy(W.BASE_SEED + 70, 32768, 32768)
    A = torch.from_numpy(W.lowrank_svd(W.BASE_SEED + 71).astype(np.float32)).to(DEV)
    small = L.make_source("dense", a=A)
    with L.Context(0, n_streams=2) as c:
        # a tolerance no estimate reaches keeps the long solve running every
        # sweep (a fixed budget alone would end it at the fixed point)
        rr, rc = W.draw_indices(74, 32768, 64, sort=True), W.draw_indices(75, 32768, 64, sort=True)
        p_long, k1 = L.make_params(64, 96, 60, W.draw_indices(72, 32768, 96), tol=1e-300,
                                   resid_rows=rr, resid_cols=rc)
        p_small, k2 = L.make_params(8, 8, 1, W.draw_indices(73, 256, 8))
        c.solve(small, p_small, 8)          # warm-up (kernel modules loaded)
        t0 = time.perf_counter()
        alone = c.solve(src, p_long, 96)
        t_long = time.perf_counter() - t0
        assert alone.info.status == 0
        assert t_long > 0.1, t_long          # long enough to overlap with
        job = c.submit(src, p_long)
        t = {}
        waiting = threading.Event()

        def fetch_long():
            t["fetch_start"] = time.perf_counter()
            waiting.set()
            r = c.fetch(job, 96)
            t["long_done"] = time.perf_counter()
            t["long_status"] = r.info.status

        th = threading.Thread(target=fetch_long)
        th.start()
        waiting.wait()
        time.sleep(0.005)                    # the fetching thread is inside fetch_cur
        t0 = time.perf_counter()
        j2 = c.submit(small, p_small)
        t["submitted"] = time.perf_counter()
        while True:
            code, info = L.lra_cross_poll(c.ctx, j2)
            if code == L.LRA_OK:
                break
        t["small_done"] = time.perf_counter()
        r2 = c.fetch(j2, 8)
        th.join()
        assert r2.info.status == 0 and info.status == 0 and t["long_status"] == 0
        assert t["small_done"] < t["long_done"], (t, t_long)
        assert t["submitted"] - t0 < 0.25 * t_long, (t, t_long)


@pytest.mark.parametrize("m,n,lda,l", [
    (5000, 96, 96, 96),        # every column: all sectors shared, l % 4 == 0
    (4099, 90, 92, 90),        # every column, padded rows, partial last sector, l % 4 != 0
    (20001, 4096, 4100, 24),   # ragged last row tile, padded rows
    (1037, 3000, 3000, 7),     # odd l: scalar stores
    (33, 200, 256, 1),         # one column, fewer rows than two tiles
])
def test_stored_column_gather_is_bit_exact(ctx, m, n, lda, l):
    """C = M[:, J] of a stored FP32 matrix (TMA row tiles of the distinct
    32-byte sectors of J, transposed in shared memory) is an exact copy, for
    padded row pitches, ragged row tiles, shared and partial sectors."""
    rng = np.random.default_rng(m + n + l)
    full = rng.standard_normal((m, lda)).astype(np.float32)
    dev = torch.from_numpy(full).to(DEV)[:, :n]
    assert dev.stride(0) == lda
    src = L.make_source("dense", a=dev)
    J0 = W.draw_indices(m + l, n, l)
    p, kp = L.make_params(l, l, 2, J0)
    res = ctx.solve(src, p, l, m, n, want_strips=True, device=DEV)
    assert res.info.status == 0
    A = full[:, :n]
    np.testing.assert_array_equal(res.C.cpu().numpy(), A[:, res.J])
    np.testing.assert_array_equal(res.R.cpu().numpy(), A[res.I, :])
    if l == n:
        assert sorted(res.J.tolist()) == list(range(n))
