"""Served form: requests of different sizes, ranks and generators admitted
while others run (several context streams, memory-budget admission).  Each
result must be identical alone and in the mix, and agree with the FP64
oracle within the error bar."""
import time

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import GPU_TAU, compare_traces, error_ok, sampled_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1611_01391_gb300 as L  # noqa: E402


def _prepare(reqs):
    """Device-resident inputs and argument structs of each request."""
    out = []
    for r in reqs:
        xd = torch.from_numpy(r["x"]).cuda()
        yd = torch.from_numpy(r["y"]).cuda()
        src = L.make_source(r["kind"], x=xd, y=yd, h=r["h"])
        p, keep = L.make_params(r["k"], r["l"], r["sweeps"], r["J0"], resid_rows=r["rows"],
                                resid_cols=r["cols"])
        out.append((src, p, (xd, yd, keep)))
    return out


def _oracle_src(r, prec):
    if r["kind"] == "cauchy":
        return O.Cauchy(r["x"], r["y"], prec)
    if r["kind"] == "gauss":
        return O.Gauss(r["x"], r["y"], r["h"], prec)
    return O.InvDist(r["x"], r["y"], prec)


def test_same_alone_and_in_the_mix():
    reqs = W.serving_requests(W.BASE_SEED + 50, 10, min_side=256, max_side=4096)
    prep = _prepare(reqs)
    # alone: one request at a time on a single stream
    alone = []
    with L.Context(0, n_streams=1) as ctx:
        for (src, p, _), r in zip(prep, reqs):
            alone.append(ctx.solve(src, p, r["l"]))
    # in the mix: everything admitted at once on 8 streams, maxvol grids
    # capped at 56 CTAs as in the served configuration (the decisions do not
    # depend on how the strip is split over CTAs)
    with L.Context(0, n_streams=8, max_grid=56) as ctx:
        jobs = [ctx.submit(src, p) for (src, p, _) in prep]
        mixed = [ctx.fetch(j, r["l"]) for j, r in zip(jobs, reqs)]
    for a, b, r in zip(alone, mixed, reqs):
        assert a.info.status == 0 and b.info.status == 0
        np.testing.assert_array_equal(a.I, b.I)
        np.testing.assert_array_equal(a.J, b.J)
        np.testing.assert_array_equal(a.U, b.U)
        assert a.info.est_rel_err == b.info.est_rel_err


def _device_entries(src, m, n):
    """The FP32 entries of the whole m x n matrix as the device sees them."""
    rows = torch.arange(m, dtype=torch.int32, device="cuda")
    cols = torch.arange(n, dtype=torch.int32, device="cuda")
    out = torch.empty((m, n), dtype=torch.float32, device="cuda")
    L.lra_gather_entries(src, rows, cols, out)
    return out.cpu().numpy()


def test_mix_against_input_matched_oracle():
    """Requests solved in the mix against the oracle fed the device's own FP32
    entries (lra_gather_entries), generator by generator: the decision logs
    agree up to the first unseparated decision, and the error (against the
    FP64 entries, on the request's Appendix F sample) is within 1.05x of that
    oracle's (or 1e-5).  For the Gaussian kernel numpy's float32 exp is not
    CUDA's expf, so only input matching removes the spread that FP32
    rounding of the entries causes where the rank-k truncation is ill posed."""
    reqs = W.serving_requests(W.BASE_SEED + 51, 8, min_side=256, max_side=2048)
    kinds = {r["kind"] for r in reqs}
    assert {"gauss", "cauchy"} <= kinds or len(kinds) >= 2
    prep = []
    for r in reqs:
        xd = torch.from_numpy(r["x"]).cuda()
        yd = torch.from_numpy(r["y"]).cuda()
        src = L.make_source(r["kind"], x=xd, y=yd, h=r["h"])
        p, keep = L.make_params(r["k"], r["l"], r["sweeps"], r["J0"], resid_rows=r["rows"],
                                resid_cols=r["cols"], trace_cap=16384)
        prep.append((src, p, (xd, yd, keep)))
    with L.Context(0, n_streams=3) as ctx:
        jobs = [ctx.submit(src, p) for (src, p, _) in prep]
        res = [ctx.fetch(j, r["l"], r["m"], r["n"], want_strips=True, device="cuda", trace_cap=16384)
               for j, r in zip(jobs, reqs)]
        ents = [_device_entries(src, r["m"], r["n"]) for (src, _, _), r in zip(prep, reqs)]
    for g, r, A32 in zip(res, reqs, ents):
        assert g.info.status == 0
        matched = O.cross_approximation(O.Dense(A32), r["J0"], k=r["k"], sweeps=r["sweeps"],
                                        rank_tol=GPU_TAU, sample_rows=r["rows"], sample_cols=r["cols"])
        ncmp, div = compare_traces(g.trace, matched.trace, 1e-2)
        assert ncmp >= min(r["l"], 8)
        if div is None:
            assert list(g.I) == matched.I and list(g.J) == matched.J
        s64 = _oracle_src(r, "fp64")
        err = sampled_error(s64, g.C.cpu().numpy(), g.U, g.R.cpu().numpy(), r["rows"], r["cols"])
        err_m = sampled_error(s64, matched.C, matched.U, matched.R, r["rows"], r["cols"])
        assert error_ok(err, err_m), (r["kind"], r["m"], r["n"], r["k"], err, err_m)
        if r["kind"] != "gauss":
            # generators whose FP32 entries the oracle reproduces bit for bit:
            # also within 1.05x of the pure-FP64 oracle
            ref = O.cross_approximation(s64, r["J0"], k=r["k"], sweeps=r["sweeps"],
                                        sample_rows=r["rows"], sample_cols=r["cols"])
            assert error_ok(err, ref.estimate["rel"]), (r["kind"], err, ref.estimate["rel"])


def test_memory_budget_admission():
    reqs = W.serving_requests(W.BASE_SEED + 52, 3, min_side=2000, max_side=2001)
    prep = _prepare(reqs)
    budget = L.lra_cross_footprint(prep[0][0], prep[0][1]) + 4096
    with L.Context(0, mem_budget_bytes=budget, n_streams=2) as ctx:
        j0 = ctx.submit(prep[0][0], prep[0][1])
        with pytest.raises(L.LraError) as e:
            ctx.submit(prep[1][0], prep[1][1])
        assert e.value.code == L.LRA_EBUSY
        ctx.fetch(j0, reqs[0]["l"])             # frees the budget
        j1 = ctx.submit(prep[1][0], prep[1][1])
        assert ctx.fetch(j1, reqs[1]["l"]).info.status == 0


def test_poll_is_nonblocking_and_completes():
    reqs = W.serving_requests(W.BASE_SEED + 53, 2, min_side=4096, max_side=8192)
    prep = _prepare(reqs)
    with L.Context(0, n_streams=2) as ctx:
        jobs = [ctx.submit(src, p) for (src, p, _) in prep]
        t0 = time.perf_counter()
        done = set()
        while len(done) < len(jobs) and time.perf_counter() - t0 < 60:
            for j in jobs:
                if j not in done:
                    code, info = L.lra_cross_poll(ctx.ctx, j)
                    if code == L.LRA_OK:
                        assert info.status == 0
                        done.add(j)
        assert len(done) == len(jobs)
        for j, r in zip(jobs, reqs):
            ctx.fetch(j, r["l"])
