"""The seeded input generators against the recipes they state (CPU only).

Every GPU test, the oracle pins and bench.py draw their inputs from
workloads/; these checks pin what those inputs are: value ranges, spectra,
the admissibility of the far-field blocks, the request mix of the served
form and the arrival process, and that a seed fixes the bytes."""
import math

import numpy as np

import workloads as W


def test_seed_fixes_the_bytes():
    a = W.factor_gaussian(5, 300, 200, 7, 1e-3)
    b = W.factor_gaussian(5, 300, 200, 7, 1e-3)
    c = W.factor_gaussian(6, 300, 200, 7, 1e-3)
    assert a.dtype == np.float32 and a.tobytes() == b.tobytes() and a.tobytes() != c.tobytes()
    x1, y1 = W.cauchy_points(9, 100, 50)
    x2, y2 = W.cauchy_points(9, 100, 50)
    assert x1.tobytes() == x2.tobytes() and y1.tobytes() == y2.tobytes()


def test_haar_orthogonal_is_orthogonal():
    q = W.haar_orthogonal(W.rng_for(3), 64)
    np.testing.assert_allclose(q.T @ q, np.eye(64), atol=1e-12)


def test_lowrank_svd_spectrum():
    """U[:, :8] V[:, :8]^T + E with E ~ N(0, 1e-8): eight singular values at
    1 (up to the noise), the rest at the noise level."""
    m = n = 256
    a = W.lowrank_svd(W.BASE_SEED + 1, m, n, r=8, noise_std=1e-4)
    s = np.linalg.svd(a, compute_uv=False)
    noise_top = 1e-4 * (math.sqrt(m) + math.sqrt(n))    # largest singular value of E, about
    assert np.all(np.abs(s[:8] - 1.0) < 2 * noise_top)
    assert s[8] < 1.5 * noise_top and s[8] > 0.5 * noise_top


def test_factor_gaussian_rank_plus_noise():
    a = W.factor_gaussian(11, 400, 300, 12, 1e-4, dtype=np.float64)
    s = np.linalg.svd(a, compute_uv=False)
    assert s[11] > 100 * s[12]                            # rank 12 ...
    assert s[12] < 1e-4 * (math.sqrt(400) + math.sqrt(300)) * 1.5   # ... plus N(0, 1e-8) noise


def test_cauchy_points_ranges():
    x, y = W.cauchy_points(W.BASE_SEED, 10000, 8000)
    assert x.dtype == np.float32 and y.dtype == np.float32
    # y = U[0,1) + 2 in FP32 can round up to 3 exactly
    assert x.min() >= 0.0 and x.max() < 1.0 and y.min() >= 2.0 and y.max() <= 3.0
    assert abs(float(x.mean()) - 0.5) < 0.02 and abs(float(y.mean()) - 2.5) < 0.02


def test_draw_indices_distinct_in_range():
    idx = W.draw_indices(4, 1000, 96)
    assert idx.dtype == np.int32 and len(set(idx.tolist())) == 96
    assert idx.min() >= 0 and idx.max() < 1000
    s = W.draw_indices(4, 1000, 96, sort=True)
    assert np.all(np.diff(s) > 0)


def _bbox(p):
    return p.min(axis=0), p.max(axis=0)


def _admissible_sets(px, py, eta):
    (lx, hx), (ly, hy) = _bbox(px), _bbox(py)
    gap = np.maximum(0.0, np.maximum(lx - hy, ly - hx))
    dist = float(np.sqrt(np.sum(gap.astype(np.float64) ** 2)))
    diam = max(float(np.linalg.norm(hx - lx)), float(np.linalg.norm(hy - ly)))
    return dist > 0.0 and diam <= eta * dist


def test_octree_blocks_are_admissible_far_field_pairs():
    """The batched workload: 4096 pairs of boxes of a z-order octree over
    2^20 points, each side between 64 and 2048 points, each pair
    eta-admissible (eta = 1).  Each side's points lie inside its box, so
    their bounding boxes are admissible too, which is what is checked here;
    the ranges of a pair do not overlap."""
    pts, blocks = W.octree_block_pairs(W.BASE_SEED + 4)
    assert pts.shape == (1 << 20, 3) and pts.dtype == np.float32
    assert blocks.shape == (4096, 4)
    r0, m, c0, n = blocks.T
    assert m.min() >= 64 and n.min() >= 64 and m.max() <= 2048 and n.max() <= 2048
    assert np.all(r0 + m <= len(pts)) and np.all(c0 + n <= len(pts))
    assert np.all((r0 + m <= c0) | (c0 + n <= r0))
    for b in range(0, 4096, 16):
        a0, am, b0, bn = (int(v) for v in blocks[b])
        assert _admissible_sets(pts[a0:a0 + am], pts[b0:b0 + bn], 1.0), b
    # the candidate columns and samples of every block are local and distinct
    jc, sr, sc = W.block_candidates(W.BASE_SEED + 5, blocks[:64], 96, 32)
    for b in range(64):
        _, mb, _, nb = (int(v) for v in blocks[b])
        assert len(set(jc[b].tolist())) == min(96, nb) and jc[b].max() < nb
        assert np.all(np.diff(sr[b]) > 0) and sr[b].max() < mb
        assert np.all(np.diff(sc[b]) > 0) and sc[b].max() < nb


def test_serving_request_mix():
    """The served form's stream: generator uniform over three kinds, m and n
    log-uniform in [256, 16384], k uniform over {8, 16, 32, 64},
    l = min(96, ceil(1.5 k)), points in the stated boxes."""
    reqs = W.serving_requests(W.BASE_SEED + 50, 600)
    kinds = [r["kind"] for r in reqs]
    for kind in ("cauchy", "gauss", "invdist"):
        assert abs(kinds.count(kind) / len(reqs) - 1 / 3) < 0.07
    logs = np.log([r["m"] for r in reqs] + [r["n"] for r in reqs])
    assert abs(float(logs.mean()) - 0.5 * (math.log(256) + math.log(16384))) < 0.15
    for r in reqs:
        assert 256 <= r["m"] <= 16384 and 256 <= r["n"] <= 16384
        assert r["k"] in (8, 16, 32, 64) and r["l"] == min(96, math.ceil(1.5 * r["k"]))
        assert len(set(r["J0"].tolist())) == r["l"] and r["J0"].max() < r["n"]
        assert np.all(np.diff(r["rows"]) > 0) and r["rows"].max() < r["m"]
        assert np.all(np.diff(r["cols"]) > 0) and r["cols"].max() < r["n"]
        x, y = r["x"], r["y"]
        if r["kind"] == "cauchy":
            assert x.shape == (r["m"],) and y.shape == (r["n"],)
            assert x.min() >= 0 and x.max() < 1 and y.min() >= 2 and y.max() <= 3
        elif r["kind"] == "gauss":
            assert x.shape == (r["m"], 3) and y.shape == (r["n"], 3) and r["h"] == 0.5
            assert x.min() >= 0 and x.max() < 1 and y.min() >= 0 and y.max() < 1
        else:   # U[0,1) + 2 in FP32 can round up to 3 exactly
            assert x.min() >= 0 and x.max() < 1 and y.min() >= 2 and y.max() <= 3


def test_poisson_arrivals():
    t = W.poisson_arrivals(7, 20000, 250.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(float(gaps.mean()) * 250.0 - 1.0) < 0.03
    # exponential gaps: coefficient of variation 1
    assert abs(float(gaps.std() / gaps.mean()) - 1.0) < 0.05


def test_delta_matrix():
    a = W.delta_matrix(5, 7, 2, 3)
    assert a.shape == (5, 7) and a[2, 3] == 1 and np.count_nonzero(a) == 1
